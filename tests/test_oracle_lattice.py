"""Pins for oracle/lattice.py: D3Q27 set, Hermite reading, generalized
equilibrium and the central-moment table (Sec. II B, Eqs. 13-20).

Each check compares against a fact fixed by the paper or by the mathematics,
computed by code paths independent of the function under test (explicit
Python loops over the 27 velocities instead of the matrix routines).
"""
import itertools
import math

import pytest
import torch

from oracle import lattice as L

DT = torch.float64
CS2 = 1.0 / 3.0


def brute_central_moment(f, u, a, b, c):
    """sum_i f_i (c_ix-u_x)^a (c_iy-u_y)^b (c_iz-u_z)^c by explicit loops (Eq. 19)."""
    s = 0.0
    for cz, cy, cx in itertools.product((-1, 0, 1), repeat=3):
        i = (cx + 1) + 3 * (cy + 1) + 9 * (cz + 1)
        s += float(f[i]) * (cx - u[0]) ** a * (cy - u[1]) ** b * (cz - u[2]) ** c
    return s


def test_velocity_set_and_weights():
    c = L.velocities()
    w = L.weights()
    assert c.shape == (27, 3)
    assert len({tuple(v) for v in c.tolist()}) == 27
    # Eq. 17 by speed class
    for i in range(27):
        n2 = int((c[i] ** 2).sum())
        assert float(w[i]) == pytest.approx({0: 8 / 27, 1: 2 / 27, 2: 1 / 54, 3: 1 / 216}[n2], abs=1e-16)
    assert float(w.sum()) == pytest.approx(1.0, abs=1e-15)
    # lattice isotropy up to fourth order: sum w c_a c_b = c_s^2 d_ab,
    # sum w c_a^2 c_b^2 = c_s^4 (a != b), odd moments vanish
    for a in range(3):
        assert float((w * c[:, a]).sum()) == pytest.approx(0.0, abs=1e-16)
        for b in range(3):
            assert float((w * c[:, a] * c[:, b]).sum()) == pytest.approx(CS2 if a == b else 0.0, abs=1e-16)
            if a != b:
                assert float((w * c[:, a] ** 2 * c[:, b] ** 2).sum()) == pytest.approx(CS2 ** 2, abs=1e-16)
    # rest vector at 13, opposite = 26 - i
    assert torch.equal(c[13], torch.zeros(3, dtype=DT))
    assert L.opposite() == [26 - i for i in range(27)]


def test_hermite_orthogonality():
    """Tensor-product Hermite polynomials are orthogonal under the D3Q27 weights,
    with norms prod(1, c_s^2, 2 c_s^4) -- the defining property of the
    lattice Hermite basis the paper refers to."""
    w = L.weights()
    norms = {0: 1.0, 1: CS2, 2: 2 * CS2 ** 2}
    exps = L.moment_exponents()
    for m in exps:
        for n in exps:
            v = float((w * L.hermite(*m) * L.hermite(*n)).sum())
            ref = norms[m[0]] * norms[m[1]] * norms[m[2]] if m == n else 0.0
            assert v == pytest.approx(ref, abs=1e-15)


def test_isotropic_operator_moments():
    """E_i (Eq. 16) carries zero mass and momentum and adds the identity to the
    second moment, so that f^eq has second moment p_m I at rest."""
    E = L.isotropic_operator()
    c = L.velocities()
    assert float(E.sum()) == pytest.approx(0.0, abs=1e-15)
    for a in range(3):
        assert float((E * c[:, a]).sum()) == pytest.approx(0.0, abs=1e-15)
        for b in range(3):
            assert float((E * c[:, a] * c[:, b]).sum()) == pytest.approx(1.0 if a == b else 0.0, abs=1e-14)
    assert float(E[13]) == pytest.approx(-19.0 / 9.0, abs=1e-14)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_equilibrium_central_moments_match_table(seed):
    """Pin (Eq. 20): brute-force central moments of the phase-space
    equilibrium of Eqs. 13-16 equal the table -- rho, p_m, p_m c_s^2,
    p_m c_s^4, all others zero -- at arbitrary velocity."""
    g = torch.Generator().manual_seed(seed)
    for _ in range(4):
        rho = float(torch.rand(1, generator=g, dtype=DT)) * 7 + 0.3
        pm = float(torch.rand(1, generator=g, dtype=DT)) * 1.5 - 0.2
        u = ((torch.rand(3, generator=g, dtype=DT) - 0.5) * 0.6).tolist()
        feq = L.f_eq_phase_space(torch.tensor(rho, dtype=DT), torch.tensor(u, dtype=DT), torch.tensor(pm, dtype=DT))
        for (a, b, c) in L.moment_exponents():
            k = brute_central_moment(feq, u, a, b, c)
            order = sorted((a, b, c))
            if (a, b, c) == (0, 0, 0):
                ref = rho
            elif order == [0, 0, 2]:
                ref = pm
            elif order == [0, 2, 2]:
                ref = pm * CS2
            elif (a, b, c) == (2, 2, 2):
                ref = pm * CS2 ** 2
            else:
                ref = 0.0
            assert k == pytest.approx(ref, abs=2e-13), (a, b, c)


def test_equilibrium_raw_second_moment():
    """Sec. II B requirement: sum_i f_i^eq c_a c_b = p_m d_ab + rho u_a u_b,
    and mass / momentum are rho and rho u."""
    c = L.velocities()
    rho, pm = 3.7, 0.41
    u = torch.tensor([0.07, -0.05, 0.11], dtype=DT)
    feq = L.f_eq_phase_space(torch.tensor(rho, dtype=DT), u, torch.tensor(pm, dtype=DT))
    assert float(feq.sum()) == pytest.approx(rho, abs=1e-13)
    for a in range(3):
        assert float((feq * c[:, a]).sum()) == pytest.approx(rho * float(u[a]), abs=1e-13)
        for b in range(3):
            ref = pm * (a == b) + rho * float(u[a] * u[b])
            assert float((feq * c[:, a] * c[:, b]).sum()) == pytest.approx(ref, abs=1e-13)


def test_equilibrium_at_rest_ideal_gas():
    """With p_m = rho c_s^2 and u = 0 the equilibrium is w_i rho."""
    rho = torch.tensor(2.5, dtype=DT)
    feq = L.f_eq_phase_space(rho, torch.zeros(3, dtype=DT), rho * CS2)
    assert torch.allclose(feq, L.weights() * 2.5, atol=1e-15)


def test_sixth_order_equilibrium_is_maxwellian_product():
    """g^{eq,6} (Eq. 14) has the central moments of the lattice Maxwellian
    (rho, rho c_s^2, rho c_s^4, rho c_s^6 on the diagonal orders), i.e. it is
    the p_m = rho c_s^2 member of the family of Eq. 20."""
    rho = 1.9
    u = [0.13, -0.21, 0.05]
    g = L.g_eq6(torch.tensor(rho, dtype=DT), torch.tensor(u, dtype=DT))
    assert brute_central_moment(g, u, 2, 2, 2) == pytest.approx(rho * CS2 ** 3, abs=1e-13)
    assert brute_central_moment(g, u, 2, 0, 2) == pytest.approx(rho * CS2 ** 2, abs=1e-13)
    assert brute_central_moment(g, u, 1, 2, 0) == pytest.approx(0.0, abs=1e-13)


def test_central_moment_roundtrip_and_matrix():
    g = torch.Generator().manual_seed(7)
    f = torch.rand(5, 27, generator=g, dtype=DT)
    u = (torch.rand(5, 3, generator=g, dtype=DT) - 0.5) * 0.5
    k = L.central_moments(f, u)
    for n in range(5):
        for (a, b, c) in [(0, 0, 0), (1, 0, 0), (2, 1, 0), (2, 2, 2), (1, 1, 1), (0, 2, 1)]:
            assert float(k[n, L.midx(a, b, c)]) == pytest.approx(
                brute_central_moment(f[n], u[n].tolist(), a, b, c), abs=1e-13)
    f2 = L.from_central_moments(k, u)
    assert torch.allclose(f2, f, atol=1e-13)
    # raw moments are the central moments about u = 0
    assert torch.allclose(L.raw_moment_matrix(), L.central_moment_matrix(torch.zeros(3, dtype=DT)))
