"""D3Q27 lattice, generalized equilibrium and moment definitions (FP64, CPU).

Test infrastructure only (see ``oracle/__init__.py``).

Conventions
  * Velocity index i runs over the 27 vectors c_i in {-1,0,1}^3 in tensor order
    i = (c_x+1) + 3 (c_y+1) + 9 (c_z+1); the rest vector is i = 13 and the
    opposite of i is 26 - i.
  * Moment index m = a + 3 b + 9 c stands for the exponents (a, b, c) of
    (alpha, beta, gamma) in Eqs. 18-19, each 0, 1 or 2.
  * c_s^2 = 1/3 (Sec. II B).
"""
from __future__ import annotations

import itertools

import torch

DT = torch.float64
CS2 = 1.0 / 3.0


def velocities() -> torch.Tensor:
    """The 27 D3Q27 velocity vectors (Sec. II B, Fig. 1) as a (27, 3) tensor."""
    c = torch.zeros(27, 3, dtype=DT)
    for cz, cy, cx in itertools.product((-1, 0, 1), repeat=3):
        i = (cx + 1) + 3 * (cy + 1) + 9 * (cz + 1)
        c[i] = torch.tensor([cx, cy, cz], dtype=DT)
    return c


def weights() -> torch.Tensor:
    """Lattice weights by |c_i|^2 = 0, 1, 2, 3: 8/27, 2/27, 1/54, 1/216 (Eq. 17)."""
    table = {0: 8.0 / 27.0, 1: 2.0 / 27.0, 2: 1.0 / 54.0, 3: 1.0 / 216.0}
    c = velocities()
    return torch.tensor([table[int(n)] for n in (c * c).sum(1).tolist()], dtype=DT)


def opposite() -> list[int]:
    """Index of -c_i for each i."""
    c = velocities()
    out = []
    for i in range(27):
        out.append(next(k for k in range(27) if torch.equal(c[k], -c[i])))
    return out


def moment_exponents() -> list[tuple[int, int, int]]:
    """(a, b, c) for each moment index m = a + 3b + 9c."""
    return [(m % 3, (m // 3) % 3, m // 9) for m in range(27)]


def midx(a: int, b: int, c: int) -> int:
    """Moment index of k_{abc}."""
    return a + 3 * b + 9 * c


# ---------------------------------------------------------------------------
# Hermite polynomials.  The paper defines H_{i abc} only by reference to
# Appendix B of Saito et al. (2023), which is not reproduced.  Reading used
# here: the tensor-product (separable) Hermite polynomials of the D3Q27 lattice,
#   H_{i abc} = h_a(c_ix) h_b(c_iy) h_c(c_iz),  h_0 = 1, h_1 = c, h_2 = c^2 - c_s^2.
# Pinned by tests: under this reading the central moments of Eqs. 13-16 equal
# the table of Eq. 20 at any velocity.
# ---------------------------------------------------------------------------
def _h1d(n: int, c: torch.Tensor) -> torch.Tensor:
    if n == 0:
        return torch.ones_like(c)
    if n == 1:
        return c
    return c * c - CS2


def hermite(a: int, b: int, c: int) -> torch.Tensor:
    """H_{i abc} for all 27 i as a (27,) tensor (reading of the paper's H)."""
    v = velocities()
    return _h1d(a, v[:, 0]) * _h1d(b, v[:, 1]) * _h1d(c, v[:, 2])


def g_eq6(rho: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """Sixth-order Hermite equilibrium g_i^{eq,6} (Eq. 14), written term by term.

    rho: (...,) density, u: (..., 3) velocity.  Returns (..., 27).
    """
    w = weights()
    H = {(a, b, c): hermite(a, b, c) for a in range(3) for b in range(3) for c in range(3)}
    ux, uy, uz = u[..., 0:1], u[..., 1:2], u[..., 2:3]
    cs2 = CS2
    t1 = (ux * H[1, 0, 0] + uy * H[0, 1, 0] + uz * H[0, 0, 1]) / cs2
    t2 = (ux**2 * H[2, 0, 0] + uy**2 * H[0, 2, 0] + uz**2 * H[0, 0, 2]
          + 2.0 * (ux * uy * H[1, 1, 0] + uy * uz * H[0, 1, 1] + ux * uz * H[1, 0, 1])) / (2.0 * cs2**2)
    t3 = (ux**2 * uy * H[2, 1, 0] + ux**2 * uz * H[2, 0, 1] + ux * uy**2 * H[1, 2, 0]
          + ux * uz**2 * H[1, 0, 2] + uy * uz**2 * H[0, 1, 2] + uy**2 * uz * H[0, 2, 1]
          + 2.0 * ux * uy * uz * H[1, 1, 1]) / (2.0 * cs2**3)
    t4 = (ux**2 * uy**2 * H[2, 2, 0] + ux**2 * uz**2 * H[2, 0, 2] + uy**2 * uz**2 * H[0, 2, 2]
          + 2.0 * (ux * uy * uz**2 * H[1, 1, 2] + ux * uy**2 * uz * H[1, 2, 1]
                   + ux**2 * uy * uz * H[2, 1, 1])) / (4.0 * cs2**4)
    t5 = (ux**2 * uy * uz**2 * H[2, 1, 2] + ux**2 * uy**2 * uz * H[2, 2, 1]
          + ux * uy**2 * uz**2 * H[1, 2, 2]) / (4.0 * cs2**5)
    t6 = ux**2 * uy**2 * uz**2 * H[2, 2, 2] / (8.0 * cs2**6)
    return rho[..., None] * w * (1.0 + t1 + t2 + t3 + t4 + t5 + t6)


def isotropic_operator() -> torch.Tensor:
    """E_i of Eq. 16 as a (27,) tensor."""
    w = weights()
    cs2 = CS2
    return w * ((hermite(2, 0, 0) + hermite(0, 2, 0) + hermite(0, 0, 2)) / (2.0 * cs2**2)
                - (hermite(2, 2, 0) + hermite(0, 2, 2) + hermite(2, 0, 2)) / (4.0 * cs2**3)
                + hermite(2, 2, 2) / (8.0 * cs2**4))


def correction_operator(u: torch.Tensor) -> torch.Tensor:
    """Phi_i of Eq. 15 for velocity u (..., 3).  Returns (..., 27)."""
    w = weights()
    H = {(a, b, c): hermite(a, b, c) for a in range(3) for b in range(3) for c in range(3)}
    ux, uy, uz = u[..., 0:1], u[..., 1:2], u[..., 2:3]
    cs2 = CS2
    t3 = (ux * (H[1, 2, 0] + H[1, 0, 2]) + uy * (H[2, 1, 0] + H[0, 1, 2])
          + uz * (H[2, 0, 1] + H[0, 2, 1])) / (2.0 * cs2**3)
    t4 = ((ux**2 + uy**2) * H[2, 2, 0] + (uy**2 + uz**2) * H[0, 2, 2] + (ux**2 + uz**2) * H[2, 0, 2]
          + 2.0 * (uy * uz * H[2, 1, 1] + ux * uz * H[1, 2, 1] + ux * uy * H[1, 1, 2])) / (4.0 * cs2**4)
    t5 = (ux * (uy**2 + uz**2 - cs2) * H[1, 2, 2] + uy * (ux**2 + uz**2 - cs2) * H[2, 1, 2]
          + uz * (ux**2 + uy**2 - cs2) * H[2, 2, 1]) / (4.0 * cs2**5)
    t6 = ((ux**2 * uy**2 + uy**2 * uz**2 + ux**2 * uz**2 - cs2 * (ux**2 + uy**2 + uz**2))
          * H[2, 2, 2]) / (8.0 * cs2**6)
    return isotropic_operator() + w * (t3 + t4 + t5 + t6)


def f_eq_phase_space(rho: torch.Tensor, u: torch.Tensor, pm: torch.Tensor) -> torch.Tensor:
    """Generalized equilibrium f_i^eq = g_i^{eq,6} + (p_m - rho c_s^2) Phi_i (Eq. 13)."""
    return g_eq6(rho, u) + (pm - rho * CS2)[..., None] * correction_operator(u)


# ---------------------------------------------------------------------------
# Moments
# ---------------------------------------------------------------------------
def raw_moment_matrix() -> torch.Tensor:
    """(27, 27) matrix with rows m and columns i: c_ix^a c_iy^b c_iz^c (Eq. 18)."""
    v = velocities()
    rows = [v[:, 0] ** a * v[:, 1] ** b * v[:, 2] ** c for (a, b, c) in moment_exponents()]
    return torch.stack(rows)


def central_moment_matrix(u: torch.Tensor) -> torch.Tensor:
    """(..., 27, 27) matrix M(u) with rows m and columns i (Eq. 19):

    M_{m i} = (c_ix - u_x)^a (c_iy - u_y)^b (c_iz - u_z)^c,  so that k = M(u) f.
    """
    v = velocities()
    d = v - u[..., None, :]                       # (..., 27 velocities, 3)
    rows = [d[..., 0] ** a * d[..., 1] ** b * d[..., 2] ** c for (a, b, c) in moment_exponents()]
    return torch.stack(rows, dim=-2)              # (..., 27 moments, 27 velocities)


def central_moments(f: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """k_{abc} = sum_i f_i (c_ix-u_x)^a (c_iy-u_y)^b (c_iz-u_z)^c (Eq. 19).  f: (..., 27)."""
    return (central_moment_matrix(u) @ f[..., None])[..., 0]


def from_central_moments(k: torch.Tensor, u: torch.Tensor) -> torch.Tensor:
    """Populations with central moments k about u: solves M(u) f = k (inverse of Eq. 19)."""
    return torch.linalg.solve(central_moment_matrix(u), k[..., None])[..., 0]


def equilibrium_central_moments(rho: torch.Tensor, pm: torch.Tensor) -> torch.Tensor:
    """Equilibrium central moments (Eq. 20); all entries not listed there are zero."""
    k = torch.zeros(*rho.shape, 27, dtype=DT)
    k[..., midx(0, 0, 0)] = rho
    for (a, b, c) in ((2, 0, 0), (0, 2, 0), (0, 0, 2)):
        k[..., midx(a, b, c)] = pm
    for (a, b, c) in ((2, 2, 0), (2, 0, 2), (0, 2, 2)):
        k[..., midx(a, b, c)] = pm * CS2
    k[..., midx(2, 2, 2)] = pm * CS2 * CS2
    return k
