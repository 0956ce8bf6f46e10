"""van der Waals thermodynamics for the free-energy model (FP64, CPU).

Test infrastructure only (see ``oracle/__init__.py``).

Sec. III: the EOS p0 = rho R T / (1 - b rho) - a rho^2 (Eq. 29), its critical
point (Eq. 30), free energy psi (Eq. 31) and bulk chemical potential mu0 (the
bulk part of Eq. 32).  Sec. II A: p0 = rho mu0 - psi (Eq. 4) and the flat
interface surface tension sigma = kappa * int (d rho/dz)^2 dz (Eq. 33).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

from scipy.optimize import brentq


@dataclass(frozen=True)
class VdW:
    """van der Waals parameters a, b, R and absolute temperature T (Eq. 29)."""
    a: float
    b: float
    R: float
    T: float

    # --- Eq. 29 -----------------------------------------------------------
    def p0(self, rho: float) -> float:
        return rho * self.R * self.T / (1.0 - self.b * rho) - self.a * rho * rho

    def dp0(self, rho: float) -> float:
        return self.R * self.T / (1.0 - self.b * rho) ** 2 - 2.0 * self.a * rho

    # --- Eq. 31 -----------------------------------------------------------
    def psi(self, rho: float) -> float:
        return rho * self.R * self.T * math.log(rho / (1.0 - self.b * rho)) - self.a * rho * rho

    # --- bulk part of Eq. 32 ------------------------------------------------
    def mu0(self, rho: float) -> float:
        return (self.R * self.T * (math.log(rho / (1.0 - self.b * rho)) + 1.0 / (1.0 - self.b * rho))
                - 2.0 * self.a * rho)


def critical_point(a: float, b: float, R: float = 1.0) -> tuple[float, float, float]:
    """(rho_c, T_c, p_c) = (1/(3b), 8a/(27 R b), a/(27 b^2))  (Eq. 30)."""
    return 1.0 / (3.0 * b), 8.0 * a / (27.0 * R * b), a / (27.0 * b * b)


def at_reduced_temperature(a: float, b: float, R: float, t_over_tc: float) -> VdW:
    """EOS at T = t_over_tc * T_c."""
    return VdW(a, b, R, t_over_tc * critical_point(a, b, R)[1])


def spinodal(eos: VdW) -> tuple[float, float]:
    """Densities where dp0/drho = 0 below the critical temperature (low, high)."""
    rc = 1.0 / (3.0 * eos.b)
    lo = brentq(eos.dp0, 1e-12, rc)
    hi = brentq(eos.dp0, rc, (1.0 - 1e-12) / eos.b)
    return lo, hi


def maxwell(eos: VdW) -> tuple[float, float]:
    """Coexistence densities (rho_l, rho_v) by Maxwell's equal-area rule.

    Equivalent conditions used: mu0(rho_l) = mu0(rho_v) and p0(rho_l) = p0(rho_v).
    The coexistence pressure is found by bisection between the spinodal
    pressures; for each trial pressure the outer roots of p0(rho) = p give the
    two phases, and the chemical-potential difference changes sign at the
    coexistence pressure.
    """
    s_lo, s_hi = spinodal(eos)
    p_min, p_max = eos.p0(s_hi), eos.p0(s_lo)
    rmax = (1.0 - 1e-13) / eos.b

    def phases(p: float) -> tuple[float, float]:
        rv = brentq(lambda r: eos.p0(r) - p, 1e-14, s_lo, xtol=1e-15, rtol=1e-15)
        rl = brentq(lambda r: eos.p0(r) - p, s_hi, rmax, xtol=1e-15, rtol=1e-15)
        return rl, rv

    def gap(p: float) -> float:
        rl, rv = phases(p)
        return eos.mu0(rl) - eos.mu0(rv)

    lo = max(p_min, 1e-14) * (1 + 1e-12) if p_min > 0 else 1e-14
    hi = p_max * (1 - 1e-12)
    p_coex = brentq(gap, lo, hi, xtol=1e-16, rtol=1e-15, maxiter=500)
    return phases(p_coex)


def coexistence_chemical_potential(eos: VdW) -> float:
    rl, rv = maxwell(eos)
    return 0.5 * (eos.mu0(rl) + eos.mu0(rv))


def surface_tension_continuum(eos: VdW, kappa: float, n: int = 20000) -> float:
    """sigma = int_{rho_v}^{rho_l} sqrt(2 kappa w(rho)) d rho for a flat interface,

    w(rho) = psi(rho) - mu_c rho + p_c >= 0 (grand-potential excess density).
    This is the continuum value of Eq. 33 with kappa/2 rho'^2 = w(rho) across
    the profile.  Composite Simpson rule in rho.
    """
    rl, rv = maxwell(eos)
    mu_c = 0.5 * (eos.mu0(rl) + eos.mu0(rv))
    p_c = 0.5 * (eos.p0(rl) + eos.p0(rv))

    def integrand(r: float) -> float:
        w = eos.psi(r) - mu_c * r + p_c
        return math.sqrt(max(2.0 * kappa * w, 0.0))

    if n % 2:
        n += 1
    h = (rl - rv) / n
    s = integrand(rv) + integrand(rl)
    for k in range(1, n):
        s += (4.0 if k % 2 else 2.0) * integrand(rv + k * h)
    return s * h / 3.0


def surface_tension_profile(rho_z, kappa: float) -> float:
    """Eq. 33 on a lattice profile rho(z), z = 0 .. Nz-1 (periodic), integrated
    over z in [0, Nz/2] with central differences and the trapezoid rule.
    """
    n = len(rho_z)
    d = [(rho_z[(z + 1) % n] - rho_z[(z - 1) % n]) * 0.5 for z in range(n)]
    half = n // 2
    s = 0.0
    for z in range(half):
        s += 0.5 * (d[z] ** 2 + d[z + 1] ** 2)
    return kappa * s


def young_laplace(eos: VdW, sigma: float, radius: float) -> tuple[float, float]:
    """Inside/outside densities of a droplet of radius R at equilibrium:

    mu0(rho_in) = mu0(rho_out) and p0(rho_in) - p0(rho_out) = 2 sigma / R.
    Newton iteration started from the Maxwell densities.
    """
    ri, ro = maxwell(eos)
    for _ in range(100):
        g1 = eos.mu0(ri) - eos.mu0(ro)
        g2 = eos.p0(ri) - eos.p0(ro) - 2.0 * sigma / radius
        a11, a12 = eos.dp0(ri) / ri, -eos.dp0(ro) / ro
        a21, a22 = eos.dp0(ri), -eos.dp0(ro)
        det = a11 * a22 - a12 * a21
        dri = (g1 * a22 - a12 * g2) / det
        dro = (a11 * g2 - a21 * g1) / det
        ri, ro = ri - dri, ro - dro
        if abs(dri) + abs(dro) < 1e-15:
            break
    return ri, ro
