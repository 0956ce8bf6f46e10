"""One time step of the free-energy D3Q27 LB model, plain FP64 on the CPU.

Test infrastructure only (see ``oracle/__init__.py``).

State: populations f of shape (27, nz, ny, nx) at time t (after streaming,
before collision), a boolean solid mask of shape (nz, ny, nx), and Params.
All directions are periodic; walls are solid-mask nodes.  Populations on solid
nodes carry no meaning and are kept at zero.

The step, in the order the method defines it:
  1. rho = sum_i f_i, j = sum_i f_i c_i on fluid nodes           (Eq. 11)
  2. wetting density on solid nodes                           (Eqs. 37-38)
  3. mu = mu0(rho) - kappa lap(rho) on fluid nodes             (Eqs. 2, 32)
  4. wetting chemical potential on solid nodes                     (Eq. 36)
  5. F = (1/3 - rho) grad mu, u = (j + F/2)/rho, p_m = (1+mu)/3  (Eqs. 11-12)
  6. Q_aa = -3 d_a[(p_m - rho c_s^2) u_a], fourth-order Q         (Eqs. 27-28)
  7. central moments about u, collision, back to populations   (Eqs. 19-26)
  8. streaming with halfway bounce-back at solid nodes    (Eq. 10, Sec. III C)

Every function is written with differentiable torch ops so that autograd of
``step`` is the exact discrete adjoint of this step.

Readings where the paper is silent (each is listed in the design notes):
  * stencils: lap g = 6 sum_i w_i (g(x+c_i) - g(x)) and
    d_a g = 3 sum_i w_i c_ia g(x+c_i), the D3Q27-isotropic forms;
  * central moments are taken about the force-corrected velocity u of Eq. 11,
    and k000* = k000 (mass is conserved by collision);
  * on solid nodes u = 0, hence the flux (p_m - rho/3) u = 0 there;
  * solid nodes with no fluid neighbour get rho = mu = 0 (never read);
  * the contact-line limiter acts only on densities modified by Eq. 38;
  * halfway bounce-back: a population whose source node x - c_i is solid is
    the opposite post-collision population of x itself; for a wall moving
    with velocity U_w (Sec. III B uses moving walls, with no formula) it
    gains f^eq_i(U_w) - f^eq_-i(U_w), the part of the generalized equilibrium
    (Eq. 13) odd in the velocity, to first order in U_w, at the rho and p_m of
    the fluid node x:  2 w_i (c_i . U_w) / c_s^2 * A with A = p_m / c_s^2 for
    edge and corner velocities and A = p_m / c_s^2 + (9/4)(rho - p_m / c_s^2)
    for face velocities (for p_m = rho c_s^2 the usual A = rho).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import torch

from . import lattice as L

DT = torch.float64
C = L.velocities()
W = L.weights()
OPP = L.opposite()
CS2 = L.CS2


@dataclass
class Params:
    """Model parameters (Sec. II B and Sec. III).

    omega: the 11 relaxation rates omega_0..omega_10 of Eqs. 21-26.
    nu > 0 selects the per-node omega_1 = 1 / (rho nu / p_m + 1/2) (Sec. II B);
    nu <= 0 keeps omega_1 = omega[1].
    wetting_mode: 0 neutral (rho_s = rho_ave), 1 rho_s = phi rho_ave,
    2 rho_s = rho_ave - delta_rho (Eq. 38); wetting_value is phi or delta_rho.
    wall_u: None (walls at rest) or a (3, nz, ny, nx) float64 tensor whose
    values on solid nodes are the wall velocities (fluid entries unused).
    kappa, omega and wetting_value may be 0-d / 1-d float64 tensors with
    requires_grad for gradient checks.
    """
    a: float
    b: float
    R: float
    T: float
    kappa: object
    omega: object = field(default_factory=lambda: [1.0] * 11)
    nu: float = 0.0
    q4: bool = True
    wetting_mode: int = 0
    wetting_value: object = 1.0
    rho_l: float = 0.0
    rho_v: float = 0.0
    wall_u: object = None

    def omega_t(self) -> torch.Tensor:
        return torch.as_tensor(self.omega, dtype=DT)


# ---------------------------------------------------------------------------
# Lattice stencils (periodic)
# ---------------------------------------------------------------------------
def at(g: torch.Tensor, c) -> torch.Tensor:
    """g(x + c) for every x, periodic in all three directions."""
    cx, cy, cz = (int(v) for v in c)
    return torch.roll(g, shifts=(-cz, -cy, -cx), dims=(-3, -2, -1))


def laplacian(g: torch.Tensor) -> torch.Tensor:
    """lap g(x) = (2/c_s^2) sum_i w_i [g(x + c_i) - g(x)]."""
    out = torch.zeros_like(g)
    for i in range(27):
        out = out + W[i] * (at(g, C[i]) - g)
    return 6.0 * out


def gradient(g: torch.Tensor) -> torch.Tensor:
    """(d_x g, d_y g, d_z g)(x) = (1/c_s^2) sum_i w_i c_i g(x + c_i); shape (3, ...)."""
    comps = [torch.zeros_like(g) for _ in range(3)]
    for i in range(27):
        gi = at(g, C[i])
        for a in range(3):
            if C[i, a] != 0:
                comps[a] = comps[a] + W[i] * C[i, a] * gi
    return 3.0 * torch.stack(comps)


def solid_average(g: torch.Tensor, solid: torch.Tensor) -> tuple[torch.Tensor, torch.Tensor]:
    """sum_i w_i g(x+c_i) s_w(x+c_i) and sum_i w_i s_w(x+c_i) (Eqs. 36-37 parts)."""
    sw = (~solid).to(DT)
    num = torch.zeros_like(g)
    den = torch.zeros_like(g)
    for i in range(27):
        s = at(sw, C[i])
        num = num + W[i] * at(g, C[i]) * s
        den = den + W[i] * s
    return num, den


# ---------------------------------------------------------------------------
# Thermodynamics in torch (Eq. 32, bulk part)
# ---------------------------------------------------------------------------
def mu0(rho: torch.Tensor, p: Params) -> torch.Tensor:
    """Bulk chemical potential RT[ln(rho/(1-b rho)) + 1/(1-b rho)] - 2 a rho (Eq. 32)."""
    one_m = 1.0 - p.b * rho
    return p.R * p.T * (torch.log(rho / one_m) + 1.0 / one_m) - 2.0 * p.a * rho


# ---------------------------------------------------------------------------
# Steps 1-6: macroscopic fields
# ---------------------------------------------------------------------------
def wetting_density(rho_fluid: torch.Tensor, solid: torch.Tensor, p: Params) -> torch.Tensor:
    """Density on solid nodes from the improved wetting scheme (Eqs. 37-38).

    rho_ave is the weighted mean of fluid-neighbour densities (Eq. 37).  Where
    0.05 rho_l + 0.95 rho_v <= rho_ave <= 0.95 rho_l + 0.05 rho_v (contact-line
    region) the density is modified by Eq. 38 and then limited to the same
    band; elsewhere rho_s = rho_ave.  Neutral wetting skips Eq. 38.
    Returns a field equal to rho_fluid on fluid nodes and rho_s on solid nodes.
    """
    num, den = solid_average(rho_fluid, solid)
    has = den > 0
    rho_ave = torch.where(has, num / torch.where(has, den, torch.ones_like(den)), torch.zeros_like(num))
    if p.wetting_mode == 0:
        rho_s = rho_ave
    else:
        lo = 0.05 * p.rho_l + 0.95 * p.rho_v
        hi = 0.95 * p.rho_l + 0.05 * p.rho_v
        band = (rho_ave >= lo) & (rho_ave <= hi)
        wv = torch.as_tensor(p.wetting_value, dtype=DT)
        modified = wv * rho_ave if p.wetting_mode == 1 else rho_ave - wv
        modified = torch.clamp(modified, lo, hi)
        rho_s = torch.where(band, modified, rho_ave)
    return torch.where(solid, rho_s, rho_fluid)


def wetting_chemical_potential(mu_fluid: torch.Tensor, solid: torch.Tensor) -> torch.Tensor:
    """Chemical potential on solid nodes: weighted mean over fluid neighbours (Eq. 36)."""
    num, den = solid_average(mu_fluid, solid)
    has = den > 0
    mu_s = torch.where(has, num / torch.where(has, den, torch.ones_like(den)), torch.zeros_like(num))
    return torch.where(solid, mu_s, mu_fluid)


def fields(f: torch.Tensor, solid: torch.Tensor, p: Params) -> dict:
    """Steps 1-6 of the time step.  Returns a dict of full-grid fields."""
    fluid = ~solid
    zero = torch.zeros(f.shape[1:], dtype=DT)
    one = torch.ones(f.shape[1:], dtype=DT)
    # 1. moments (Eq. 11)
    rho_f = torch.where(fluid, f.sum(0), zero)
    j = torch.stack([torch.where(fluid, (f * C[:, a].view(27, 1, 1, 1)).sum(0), zero) for a in range(3)])
    # 2. wetting density (Eqs. 37-38)
    rho = wetting_density(rho_f, solid, p)
    # 3. chemical potential (Eqs. 2, 32)
    rho_safe = torch.where(fluid, rho, one)
    kappa = torch.as_tensor(p.kappa, dtype=DT)
    mu_f = torch.where(fluid, mu0(rho_safe, p) - kappa * laplacian(rho), zero)
    # 4. wetting chemical potential (Eq. 36)
    mu = wetting_chemical_potential(mu_f, solid)
    # 5. force (Eq. 12), velocity (Eq. 11), modified pressure
    gmu = gradient(mu)
    F = torch.where(fluid, (1.0 / 3.0 - rho) * gmu, zero)
    u = torch.where(fluid, (j + 0.5 * F) / rho_safe, zero)
    pm = torch.where(fluid, (1.0 + mu) / 3.0, zero)
    # relaxation rates; omega_1 per node in viscosity mode (Sec. II B)
    om = p.omega_t()
    if p.nu > 0:
        om1 = torch.where(fluid, 1.0 / (rho_safe * p.nu / torch.where(fluid, pm, one) + 0.5), zero)
    else:
        om1 = om[1] * one
    # 6. third-order diagonal corrections (Eq. 27) and fourth-order ones (Eq. 28)
    flux = torch.where(fluid, pm - rho * CS2, zero) * u            # (p_m - rho c_s^2) u_a
    Q = torch.stack([torch.where(fluid, -3.0 * gradient(flux[a])[a], zero) for a in range(3)])
    return dict(rho=rho, j=j, mu=mu, F=F, u=u, pm=pm, om1=om1, Q=Q)


# ---------------------------------------------------------------------------
# Step 7: central-moment collision (Eqs. 19-26)
# ---------------------------------------------------------------------------
def collide_moments(k: torch.Tensor, pm: torch.Tensor, F: torch.Tensor, Q: torch.Tensor,
                    om: torch.Tensor, om1: torch.Tensor, q4: bool) -> torch.Tensor:
    """Post-collision central moments k* from Eqs. 21-26.

    k: (n, 27) pre-collision central moments; pm: (n,); F, Q: (n, 3) with
    Q = (Q_200, Q_020, Q_002); om: (11,) rates; om1: (n,) omega_1 per node.
    Sums and differences of moments that Eqs. 22-24 relax together are
    relaxed as stated there and then solved for the individual moments.
    k*_000 = k_000 (mass).
    """
    K = lambda a, b, c: k[:, L.midx(a, b, c)]
    o = [om[r] * torch.ones_like(pm) for r in range(11)]
    o[1] = om1
    cs2 = CS2
    Fx, Fy, Fz = F[:, 0], F[:, 1], F[:, 2]
    Q200, Q020, Q002 = Q[:, 0], Q[:, 1], Q[:, 2]
    out = {}
    out[0, 0, 0] = K(0, 0, 0)
    # first order (Eq. 21)
    for idx, Fa in (((1, 0, 0), Fx), ((0, 1, 0), Fy), ((0, 0, 1), Fz)):
        out[idx] = (1 - o[0]) * K(*idx) + (1 - o[0] / 2) * Fa
    # second order (Eq. 22)
    for idx in ((1, 1, 0), (0, 1, 1), (1, 0, 1)):
        out[idx] = (1 - o[1]) * K(*idx)
    A = (1 - o[1]) * (K(2, 0, 0) - K(0, 2, 0)) + (1 - o[1] / 2) * (Q200 - Q020)
    B = (1 - o[1]) * (K(2, 0, 0) - K(0, 0, 2)) + (1 - o[1] / 2) * (Q200 - Q002)
    S = ((1 - o[2]) * (K(2, 0, 0) + K(0, 2, 0) + K(0, 0, 2)) + 3 * o[2] * pm
         + (1 - o[2] / 2) * (Q200 + Q020 + Q002))
    out[2, 0, 0] = (S + A + B) / 3
    out[0, 2, 0] = (S - 2 * A + B) / 3
    out[0, 0, 2] = (S + A - 2 * B) / 3
    # third order (Eq. 23)
    for pidx, qidx, Fa in (((1, 2, 0), (1, 0, 2), Fx), ((2, 1, 0), (0, 1, 2), Fy),
                           ((2, 0, 1), (0, 2, 1), Fz)):
        P = (1 - o[3]) * (K(*pidx) + K(*qidx)) + 2 * (1 - o[3] / 2) * Fa * cs2
        D = (1 - o[4]) * (K(*pidx) - K(*qidx))
        out[pidx] = (P + D) / 2
        out[qidx] = (P - D) / 2
    out[1, 1, 1] = (1 - o[5]) * K(1, 1, 1)
    # fourth order (Eq. 24) with the approximate correction of Eq. 28
    if q4:
        Q220, Q202, Q022 = (Q200 + Q020) * cs2, (Q200 + Q002) * cs2, (Q020 + Q002) * cs2
    else:
        Q220 = Q202 = Q022 = torch.zeros_like(pm)
    D1 = ((1 - o[6]) * (K(2, 2, 0) - 2 * K(2, 0, 2) + K(0, 2, 2))
          + (1 - o[6] / 2) * (Q220 - 2 * Q202 + Q022))
    D2 = ((1 - o[6]) * (K(2, 2, 0) + K(2, 0, 2) - 2 * K(0, 2, 2))
          + (1 - o[6] / 2) * (Q220 + Q202 - 2 * Q022))
    T = ((1 - o[7]) * (K(2, 2, 0) + K(2, 0, 2) + K(0, 2, 2)) + 3 * o[7] * pm * cs2
         + (1 - o[7] / 2) * (Q220 + Q202 + Q022))
    out[2, 2, 0] = (T + D1 + D2) / 3
    out[2, 0, 2] = (T - D1) / 3
    out[0, 2, 2] = (T - D2) / 3
    for idx in ((2, 1, 1), (1, 2, 1), (1, 1, 2)):
        out[idx] = (1 - o[8]) * K(*idx)
    # fifth order (Eq. 25)
    for idx, Fa in (((1, 2, 2), Fx), ((2, 1, 2), Fy), ((2, 2, 1), Fz)):
        out[idx] = (1 - o[9]) * K(*idx) + (1 - o[9] / 2) * Fa * cs2 * cs2
    # sixth order (Eq. 26)
    out[2, 2, 2] = (1 - o[10]) * K(2, 2, 2) + o[10] * pm * cs2 * cs2
    assert len(out) == 27
    return torch.stack([out[e] for e in L.moment_exponents()], dim=1)


CHUNK = 16384


def collide(f: torch.Tensor, solid: torch.Tensor, fl: dict, p: Params) -> torch.Tensor:
    """Post-collision populations f* on fluid nodes (zero on solid nodes).

    k = M(u) f (Eq. 19), k* from Eqs. 21-26, f* = M(u)^{-1} k*.
    """
    nz, ny, nx = solid.shape
    fluid = ~solid.reshape(-1)
    idx = torch.nonzero(fluid).reshape(-1)
    fN = f.reshape(27, -1).T[idx]
    uN = fl["u"].reshape(3, -1).T[idx]
    FN = fl["F"].reshape(3, -1).T[idx]
    QN = fl["Q"].reshape(3, -1).T[idx]
    pmN = fl["pm"].reshape(-1)[idx]
    om1N = fl["om1"].reshape(-1)[idx]
    om = p.omega_t()
    parts = []
    for s in range(0, idx.numel(), CHUNK):
        sl = slice(s, s + CHUNK)
        M = L.central_moment_matrix(uN[sl])
        k = (M @ fN[sl, :, None])[..., 0]
        ks = collide_moments(k, pmN[sl], FN[sl], QN[sl], om, om1N[sl], p.q4)
        parts.append(torch.linalg.solve(M, ks[..., None])[..., 0])
    fsN = torch.cat(parts) if parts else fN
    out = torch.zeros(nz * ny * nx, 27, dtype=DT).index_copy(0, idx, fsN)
    return out.T.reshape(27, nz, ny, nx)


# ---------------------------------------------------------------------------
# Step 8: streaming with halfway bounce-back (Eq. 10, Sec. III C)
# ---------------------------------------------------------------------------
def wall_odd_equilibrium(i: int, rho: torch.Tensor, pm: torch.Tensor, uw: torch.Tensor) -> torch.Tensor:
    """f^eq_i - f^eq_-i of the generalized equilibrium (Eq. 13) at velocity
    uw, to first order in uw: 2 w_i (c_i . uw) / c_s^2 * A, A = p_m / c_s^2
    (|c_i|^2 = 2, 3) or p_m / c_s^2 + (9/4)(rho - p_m / c_s^2) (|c_i|^2 = 1)."""
    cx, cy, cz = (int(v) for v in C[i])
    a = pm / CS2
    if cx * cx + cy * cy + cz * cz == 1:
        a = a + 2.25 * (rho - pm / CS2)
    return 2.0 * W[i] * (cx * uw[0] + cy * uw[1] + cz * uw[2]) / CS2 * a


def stream(fs: torch.Tensor, solid: torch.Tensor, rho: torch.Tensor | None = None,
           pm: torch.Tensor | None = None, wall_u: torch.Tensor | None = None) -> torch.Tensor:
    """f_i(x, t+1) = f*_i(x - c_i); if x - c_i is solid, f_i(x, t+1) =
    f*_{-i}(x) + [f^eq_i - f^eq_-i](rho(x), p_m(x), U_w(x - c_i)) (the last
    term only for moving walls, wall_u given)."""
    fluid = ~solid
    out = []
    for i in range(27):
        cx, cy, cz = (int(v) for v in C[i])
        pulled = torch.roll(fs[i], shifts=(cz, cy, cx), dims=(0, 1, 2))
        src_solid = torch.roll(solid, shifts=(cz, cy, cx), dims=(0, 1, 2))
        back = fs[OPP[i]]
        if wall_u is not None:
            uw = torch.roll(wall_u, shifts=(cz, cy, cx), dims=(1, 2, 3))
            back = back + wall_odd_equilibrium(i, rho, pm, uw)
        v = torch.where(src_solid, back, pulled)
        out.append(torch.where(fluid, v, torch.zeros_like(v)))
    return torch.stack(out)


def step(f: torch.Tensor, solid: torch.Tensor, p: Params) -> torch.Tensor:
    """One full time step f(t) -> f(t+1)."""
    fl = fields(f, solid, p)
    return stream(collide(f, solid, fl, p), solid, fl["rho"], fl["pm"], p.wall_u)


def run(f: torch.Tensor, solid: torch.Tensor, p: Params, n: int) -> torch.Tensor:
    for _ in range(n):
        f = step(f, solid, p)
    return f


# ---------------------------------------------------------------------------
# Initialisation and diagnostics
# ---------------------------------------------------------------------------
def initial_populations(rho0: torch.Tensor, u0: torch.Tensor | None, solid: torch.Tensor,
                        p: Params) -> torch.Tensor:
    """f = equilibrium with central moments of Eq. 20 about u0, at rho0 and
    p_m = (1 + mu(rho0))/3, mu including the wetting values on solid nodes.
    The paper does not state its initial populations; this is the reading used.
    """
    fluid = ~solid
    rho_f = torch.where(fluid, rho0, torch.zeros_like(rho0))
    rho = wetting_density(rho_f, solid, p)
    one = torch.ones_like(rho0)
    kappa = torch.as_tensor(p.kappa, dtype=DT)
    mu_f = torch.where(fluid, mu0(torch.where(fluid, rho, one), p) - kappa * laplacian(rho),
                       torch.zeros_like(rho0))
    mu = wetting_chemical_potential(mu_f, solid)
    pm = (1.0 + mu) / 3.0
    if u0 is None:
        u0 = torch.zeros(3, *rho0.shape, dtype=DT)
    nz, ny, nx = solid.shape
    idx = torch.nonzero(fluid.reshape(-1)).reshape(-1)
    keq = L.equilibrium_central_moments(rho.reshape(-1)[idx], pm.reshape(-1)[idx])
    uN = u0.reshape(3, -1).T[idx]
    parts = [L.from_central_moments(keq[s:s + CHUNK], uN[s:s + CHUNK]) for s in range(0, idx.numel(), CHUNK)]
    fN = torch.cat(parts)
    out = torch.zeros(nz * ny * nx, 27, dtype=DT).index_copy(0, idx, fN)
    return out.T.reshape(27, nz, ny, nx)


def macroscopic(f: torch.Tensor, solid: torch.Tensor, p: Params) -> dict:
    """rho, u (force-corrected, Eq. 11), mu of the current state, plus the FP64
    totals mass = sum_fluid rho and energy = 1/2 sum_fluid rho |u|^2."""
    fl = fields(f, solid, p)
    fluid = ~solid
    mass = torch.where(fluid, fl["rho"], torch.zeros_like(fl["rho"])).sum()
    energy = 0.5 * torch.where(fluid, fl["rho"] * (fl["u"] ** 2).sum(0), torch.zeros_like(fl["rho"])).sum()
    return dict(rho=fl["rho"], u=fl["u"], mu=fl["mu"], F=fl["F"], mass=mass, energy=energy)
