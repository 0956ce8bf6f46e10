"""Results the paper prints for its own runs, reproduced with the CUDA path
(paper EOS a = 9/392, b = 2/21, R = 1, kappa = 0.02):

* Sec. III A, Fig. 2: flat-interface coexistence densities agree with
  Maxwell's equal-area construction for nu = 0.15 and nu = 0.03.  The bulk
  densities after 10 000 steps are held to 2e-4 relative (measured <= 6e-5
  at 0.7 T_c and <= 2e-6 at 0.8 and 0.9 T_c).  At 0.6 T_c the run from a
  width-5 interface goes non-finite (the paper does not print its
  temperatures).
* Sec. III B, Fig. 5: stationary droplets of radius R in 64^3 (the
  stationary-droplet workload's domain) obey the Young-Laplace law.  With
  the workload's a = 9/49, kappa = 0.01 a width-5 drop of R >= 12 goes
  non-finite, so the check runs the paper's EOS at 0.7 T_c (nu = 0.15).
* Sec. III C, Eq. 38, Fig. 7: the contact angle of a drop on a wall follows
  the wetting parameter.  The paper's own setup (0.7 T_c) grows a wall mode
  on the GPU and in the oracle, and the workload's a = 9/49, kappa = 0.01
  leaves the angle at 90 degrees for every phi and delta_rho and goes
  non-finite within 40 000 steps, so the check runs the paper's EOS at
  0.8 T_c.
* Sec. III B, Fig. 4(a): without the fourth-order correction (Eq. 28) the
  r = 30 droplet in 128^3 (0.7 T_c, nu = 0.15) diverges shortly after t = 86
  (FP64); with it the droplet stays finite.  In FP32 the uncorrected run
  goes non-finite between steps 50 and 60, so the check is: non-finite
  within 150 steps without the correction, finite and slow after 300 steps
  with it.
"""
import json
import os

import numpy as np
import pytest
import torch

from oracle import thermo as T
from paper_2504_03819_gb300 import Domain
from paper_2504_03819_gb300 import inputs as I
from paper_2504_03819_gb300.binding import Params

pytestmark = pytest.mark.gpu
GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
A392, B, KAPPA = 9.0 / 392.0, 2.0 / 21.0, 0.02


def paper_params(t_over_tc, **kw):
    eos = T.at_reduced_temperature(A392, B, 1.0, t_over_tc)
    rl, rv = T.maxwell(eos)
    return Params(a=A392, b=B, R=1.0, T=eos.T, kappa=KAPPA, rho_l=rl, rho_v=rv, **kw), rl, rv


@pytest.mark.parametrize("nu", [0.15, 0.03])
@pytest.mark.parametrize("t_over_tc", [0.7, 0.8, 0.9])
def test_coexistence_curve_matches_maxwell(t_over_tc, nu):
    """4 x 4 x 128 periodic, liquid slab of width 64 (Sec. III A setup)."""
    p, rl, rv = paper_params(t_over_tc, nu=nu)
    nz = 128
    prof = I.slab(1, 1, nz, 64, rl, rv).astype(np.float32)
    d = Domain(4, 4, nz, "f32")
    d.set_params(p)
    d.set_state(torch.from_numpy(np.repeat(np.repeat(prof, 4, axis=1), 4, axis=2)))
    d.step(10000)
    assert d.sync_status() == 0
    m = d.moments()
    r = m["rho"][:, 0, 0].double().cpu()
    assert float(r.max()) == pytest.approx(rl, rel=2e-4)
    assert float(r.min()) == pytest.approx(rv, rel=2e-4)
    # equilibrium: the chemical potential is uniform (spread below 1 % of the
    # coexistence value; measured 0.1 % at 0.7 T_c) and the flow has died out
    mu = m["mu"].double().cpu()
    assert float(mu.max() - mu.min()) < 0.01 * abs(float(mu.mean()))
    # residual flow: 3e-6 at nu = 0.15, 2e-5 at nu = 0.03 (five times slower
    # viscous decay) after 10 000 steps
    assert float(m["u"].abs().max()) < 1e-4


@pytest.mark.parametrize("q4", [0, 1])
def test_fourth_order_correction_ablation(q4):
    g = GOLD["q4_ablation"]
    n, r = g["n"], float(g["radius"])
    p, rl, rv = paper_params(0.7, nu=0.15, q4_correction=q4)
    d = Domain(n, n, n, "f32")
    d.set_params(p)
    d.set_state(torch.from_numpy(I.droplet(n, n, n, r, rl, rv).astype(np.float32)))
    if q4:
        d.step(300)
        assert d.sync_status() == 0
        assert float(d.moments()["u"].abs().max()) < 0.02
    else:
        failed = False
        for _ in range(15):
            d.step(10)
            if d.sync_status() != 0:
                failed = True
                break
        assert failed, "the droplet without the fourth-order correction stayed finite for 150 steps"
    d.close()


@pytest.mark.parametrize("radius", [12, 16, 20])
def test_laplace_law_of_stationary_droplets(radius):
    """After 10 000 steps the droplet is at equilibrium: one chemical
    potential inside and outside, and the pressure jump Delta p =
    p0(rho_in) - p0(rho_out) over the equimolar radius R_eq gives a surface
    tension sigma = Delta p R_eq / 2 that does not depend on R (measured
    0.2161 - 0.2166 for R = 12, 16, 20), within 3 % of the continuum value
    int sqrt(2 kappa w) d rho = 0.2183 and 6 % of the flat-interface 0.204
    the paper prints (a lattice effect of the ~3-node interface).
    Spurious currents stay below 1e-4 (measured 6e-6 - 3e-5; the
    paper's 2.4e-11 is FP64 after 100 000 steps).  R = 12 shrinks to R_eq
    ~ 10.3 by evaporating into the vapour, as small drops do."""
    import math
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from _wetting import equimolar_radius
    n = 64
    p, rl, rv = paper_params(0.7, nu=0.15)
    eos = T.at_reduced_temperature(A392, B, 1.0, 0.7)
    d = Domain(n, n, n, "f32")
    d.set_params(p)
    d.set_state(torch.from_numpy(I.droplet(n, n, n, float(radius), rl, rv).astype(np.float32)))
    d.step(10000)
    assert d.sync_status() == 0
    m = d.moments()
    rho = m["rho"].double().cpu().numpy()
    c = n // 2
    rin, rout = float(rho[c - 1:c + 1, c - 1:c + 1, c - 1:c + 1].mean()), float(rho[0, 0, 0])
    req = equimolar_radius(rho, rin, rout)
    sigma = (eos.p0(rin) - eos.p0(rout)) * req / 2.0
    sigma_c = T.surface_tension_continuum(eos, KAPPA)
    assert sigma == pytest.approx(sigma_c, rel=0.03)
    assert sigma == pytest.approx(GOLD["surface_tension_flat_0p7Tc"]["sigma"], rel=0.08)
    # one chemical potential: both phases moved off coexistence by the same
    # Kelvin shift (to 2 % of it; measured 0.1 - 1.5 %)
    kelvin = eos.mu0(rin) - T.coexistence_chemical_potential(eos)
    assert kelvin > 0 and abs(eos.mu0(rin) - eos.mu0(rout)) < 0.02 * kelvin
    assert float(m["u"].abs().max()) < 1e-4
    assert math.isfinite(req) and req > 0.7 * radius
    d.close()


def test_contact_angle_follows_the_wetting_parameter():
    """A hemisphere of R = 18 (width 5) on the bottom wall of 64 x 64 x 40
    (solid planes z = 0 and 39), all rates 1, 10 000 steps (the angles do not
    change between 10 000 and 40 000 steps).  Angle from a sphere fit to the
    mid-density surface (tests/_wetting.py).  Neutral wetting keeps 90
    degrees; phi > 1 makes the wall hydrophilic, each larger phi a smaller
    angle; delta_rho > 0 hydrophobic, each larger delta_rho a larger angle
    (measured 90.3; 72.8, 56.8, 40.6 for phi = 1.1, 1.2, 1.3; 100.4, 115.5,
    132.4 for delta_rho = 0.2, 0.5, 0.8).  The liquid volume stays put (no
    evaporation: every angle belongs to the same drop)."""
    import sys
    sys.path.insert(0, os.path.dirname(__file__))
    from _wetting import contact_angle
    nx, ny, nz, R = 64, 64, 40, 18.0
    mask = I.wall_mask(nx, ny, nz, planes=(0, nz - 1))
    solid = mask.astype(bool)
    angles = {}
    for mode, value in [(0, 0.0), (1, 1.1), (1, 1.2), (1, 1.3), (2, 0.2), (2, 0.5), (2, 0.8)]:
        p, rl, rv = paper_params(0.8, wetting_mode=mode, wetting_value=value)
        rho0 = I.sessile_droplet(nx, ny, nz, R, rl, rv, wall_z=0.5).astype(np.float32)
        d = Domain(nx, ny, nz, "f32", solid_mask=mask)
        d.set_params(p)
        d.set_state(torch.from_numpy(rho0))
        d.step(10000)
        assert d.sync_status() == 0
        rho = d.moments()["rho"].double().cpu().numpy()
        vol0 = float(((rho0 - rv) / (rl - rv))[~solid].sum())
        vol = float(((rho - rv) / (rl - rv))[~solid].sum())
        assert vol == pytest.approx(vol0, rel=0.02)
        angles[(mode, value)] = contact_angle(rho, rl, rv, solid)
        d.close()
    assert angles[(0, 0.0)] == pytest.approx(90.0, abs=2.0)
    phi = [angles[(1, v)] for v in (1.1, 1.2, 1.3)]
    drho = [angles[(2, v)] for v in (0.2, 0.5, 0.8)]
    assert 88.0 > phi[0] > phi[1] > phi[2]
    assert 92.0 < drho[0] < drho[1] < drho[2]
