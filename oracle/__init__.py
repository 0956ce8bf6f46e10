"""FP64 CPU oracle for the free-energy D3Q27 lattice Boltzmann step (arXiv 2504.03819).

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, obviously-checkable
restatement of the method in double precision on the CPU (PyTorch CPU ops in
float64; autograd of the same code is the discrete adjoint).  Only the test
suite, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` / ``--impl
reference`` legs of ``bench.py`` may import it.  The CUDA library and its Python
binding never import, link or execute anything here, and nothing here imports
them: the two implementations share no code.

Equation numbers follow the paper's numbered displays in order (Eq. 1 is the
free-energy functional, Eq. 38 the contact-line surface density).

Modules
  lattice  -- D3Q27 velocity set and weights (Sec. II B, Eq. 17), Hermite
              polynomials, the phase-space generalized equilibrium
              (Eqs. 13-16), the raw/central-moment definitions (Eqs. 18-19)
              and the equilibrium central-moment table (Eq. 20).
  thermo   -- van der Waals EOS, critical point, free energy and chemical
              potential (Sec. III, Eqs. 29-32), Maxwell equal-area
              construction, flat-interface surface tension (Eq. 33) and the
              Young-Laplace droplet densities (Sec. III B).
  step     -- one time step: moments (Eq. 11), wetting boundary (Eqs. 36-38),
              chemical potential (Eqs. 2, 32), force (Eq. 12), corrections
              (Eqs. 27-28), central-moment collision (Eqs. 21-26) and
              streaming (Eq. 10) with halfway bounce-back (Sec. III C);
              plus initialisation and the diagnostics used by the tests.

Pinned against the paper and the mathematics by tests/test_oracle_*.py.
Functions whose result has no such pin say "parity unpinned" in their docstring.
"""
