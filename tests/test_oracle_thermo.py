"""Pins for oracle/thermo.py (Sec. III, Eqs. 29-33)."""
import json
import math
import os

import pytest
from scipy.integrate import quad

from oracle import thermo as T

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
A_PAPER, B, R = 9.0 / 392.0, 2.0 / 21.0, 1.0


def test_critical_point_printed():
    g = GOLD["critical_point_paper_eos"]
    rc, tc, pc = T.critical_point(g["a"], g["b"], g["R"])
    assert rc == pytest.approx(g["rho_c"], rel=1e-14)
    assert tc == pytest.approx(g["T_c"], rel=1e-14)
    assert pc == pytest.approx(g["p_c"], rel=1e-14)
    # Eq. 30 is where dp0/drho and d2p0/drho2 vanish
    eos = T.VdW(g["a"], g["b"], g["R"], tc)
    assert eos.dp0(rc) == pytest.approx(0.0, abs=1e-14)
    h = 1e-4
    assert (eos.p0(rc + h) - 2 * eos.p0(rc) + eos.p0(rc - h)) / h ** 2 == pytest.approx(0.0, abs=1e-6)
    assert eos.p0(rc) == pytest.approx(pc, rel=1e-13)


def test_maxwell_printed_values():
    g = GOLD["maxwell_0p7Tc"]
    rl, rv = T.maxwell(T.at_reduced_temperature(A_PAPER, B, R, g["t_over_tc"]))
    assert abs(rl - g["rho_l"]) <= g["printed_digits"]["rho_l"]
    assert abs(rv - g["rho_v"]) <= g["printed_digits"]["rho_v"]
    assert abs(rl / rv - g["ratio"]) <= g["printed_digits"]["ratio"]


@pytest.mark.parametrize("t", [0.6, 0.7, 0.85, 0.95])
def test_equal_area_in_pv_plane(t):
    """Maxwell's rule in its original form: in the p-V plane (V = 1/rho) the
    isotherm encloses equal areas above and below the coexistence pressure,
    int_{V_l}^{V_v} (p(V) - p_coex) dV = 0, by adaptive quadrature."""
    eos = T.at_reduced_temperature(A_PAPER, B, R, t)
    rl, rv = T.maxwell(eos)
    p_co = eos.p0(rl)
    assert eos.p0(rv) == pytest.approx(p_co, rel=1e-10, abs=1e-14)
    area, _ = quad(lambda V: eos.p0(1.0 / V) - p_co, 1.0 / rl, 1.0 / rv, limit=200, epsabs=1e-14)
    scale = p_co * (1.0 / rv - 1.0 / rl)
    assert abs(area) < 1e-9 * max(scale, 1e-3)


def test_reduced_form_is_universal():
    """vdW in reduced variables is parameter free: b*rho_l and b*rho_v at the
    same T/Tc do not depend on a (so a = 9/49 and a = 9/392 share them)."""
    for t in (0.7, 0.85):
        r1 = T.maxwell(T.at_reduced_temperature(9.0 / 392.0, B, R, t))
        r2 = T.maxwell(T.at_reduced_temperature(9.0 / 49.0, B, R, t))
        assert r1[0] == pytest.approx(r2[0], rel=1e-11)
        assert r1[1] == pytest.approx(r2[1], rel=1e-11)


def test_near_critical_scaling():
    """Mean-field vdW: (rho_l - rho_v)/rho_c -> 4 sqrt(1 - T/Tc) as T -> Tc."""
    eps = 1e-4
    rl, rv = T.maxwell(T.at_reduced_temperature(A_PAPER, B, R, 1.0 - eps))
    rc = 1.0 / (3.0 * B)
    assert (rl - rv) / rc / math.sqrt(eps) == pytest.approx(4.0, rel=2e-3)


def test_free_energy_identities():
    """mu0 = d psi / d rho and p0 = rho mu0 - psi (Eq. 4) for the vdW forms
    (Eqs. 29, 31, 32)."""
    eos = T.at_reduced_temperature(A_PAPER, B, R, 0.7)
    for rho in (0.3, 1.0, 3.5, 7.0, 9.5):
        h = 1e-6
        dpsi = (eos.psi(rho + h) - eos.psi(rho - h)) / (2 * h)
        assert eos.mu0(rho) == pytest.approx(dpsi, rel=1e-7, abs=1e-9)
        assert eos.p0(rho) == pytest.approx(rho * eos.mu0(rho) - eos.psi(rho), rel=1e-12, abs=1e-14)
        dp = (eos.p0(rho + h) - eos.p0(rho - h)) / (2 * h)
        assert eos.dp0(rho) == pytest.approx(dp, rel=1e-6, abs=1e-8)


def test_young_laplace_limits():
    """Young-Laplace droplet densities tend to Maxwell's as R -> infinity, and
    the pressure jump of the solution is 2 sigma / R at equal mu0."""
    eos = T.at_reduced_temperature(A_PAPER, B, R, 0.7)
    rl, rv = T.maxwell(eos)
    ri, ro = T.young_laplace(eos, 0.204, 1e9)
    assert ri == pytest.approx(rl, rel=1e-8) and ro == pytest.approx(rv, rel=1e-7)
    ri, ro = T.young_laplace(eos, 0.204, 20.0)
    assert eos.p0(ri) - eos.p0(ro) == pytest.approx(2 * 0.204 / 20.0, rel=1e-10)
    assert eos.mu0(ri) == pytest.approx(eos.mu0(ro), rel=1e-12)
    assert ri > rl and ro > rv   # curvature raises both densities


def test_surface_tension_continuum_quadrature():
    """The Simpson quadrature of the continuum flat-interface tension agrees
    with an independent adaptive integral of the same integrand."""
    eos = T.at_reduced_temperature(A_PAPER, B, R, 0.7)
    rl, rv = T.maxwell(eos)
    mu_c, p_c = eos.mu0(rl), eos.p0(rl)
    ref, _ = quad(lambda r: math.sqrt(max(2 * 0.02 * (eos.psi(r) - mu_c * r + p_c), 0.0)), rv, rl, limit=400)
    assert T.surface_tension_continuum(eos, 0.02) == pytest.approx(ref, rel=1e-6)
