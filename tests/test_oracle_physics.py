"""Physical results the oracle must reproduce (Sec. III): the Laplace law of a
stationary droplet, the neutral contact angle on a wall, and the shape of a
droplet carried by a uniform flow.

The 3-D runs of the paper are far too large for the FP64 oracle, so each
check uses the same D3Q27 model on a quasi-2-D domain one node thick
(periodic in that direction): every field is uniform along it, a sphere
becomes a cylinder and the Laplace law reads Delta p = sigma / R.  Paper
EOS (a = 9/392, b = 2/21, R = 1), T = 0.7 T_c, kappa = 0.02, all rates 1,
initial tanh interfaces of width 5 (Eqs. 34-35).
"""
import json
import math
import os

import numpy as np
import pytest
import torch

from oracle import step as S
from oracle import thermo as T
from paper_2504_03819_gb300 import inputs as I

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))
A392, B = 9.0 / 392.0, 2.0 / 21.0


def setup(**kw):
    eos = T.at_reduced_temperature(A392, B, 1.0, 0.7)
    rl, rv = T.maxwell(eos)
    p = S.Params(a=A392, b=B, R=1.0, T=eos.T, kappa=0.02, rho_l=rl, rho_v=rv, **kw)
    return eos, p, rl, rv


def cylinder(n, radius, rl, rv):
    """Cylinder along z in an n x n x 1 domain, centred in x-y."""
    return I.droplet(n, n, 1, radius, rl, rv, centre=((n - 1) / 2.0, (n - 1) / 2.0, 0.0))


def test_laplace_law_cylinder():
    """Sec. III B: at equilibrium the pressure jump across the interface of a
    drop of radius R is sigma / R (cylinder) with sigma the flat-interface
    value of Sec. III A (0.204, printed), and both bulk phases sit at one
    chemical potential.  The equimolar radius R = 8.1 with an interface about
    3 nodes wide leaves a curvature correction of a few percent, so the
    product Delta p R is held to 7 % (measured 0.2137, +4.7 %); the bulk
    chemical potentials of the two phases agree to 5 % of their common
    Kelvin shift from coexistence (measured 1.7 %)."""
    eos, p, rl, rv = setup()
    n = 32
    solid = torch.zeros(1, n, n, dtype=torch.bool)
    f = S.initial_populations(torch.from_numpy(cylinder(n, 8.0, rl, rv)), None, solid, p)
    f = S.run(f, solid, p, 500)
    m = S.macroscopic(f, solid, p)
    r = m["rho"][0]
    rin, rout = float(r[n // 2, n // 2]), float(r[0, 0])
    area = float(((r - rout) / (rin - rout)).sum())
    req = math.sqrt(area / math.pi)
    sigma = GOLD["surface_tension_flat_0p7Tc"]["sigma"]
    dp = eos.p0(rin) - eos.p0(rout)
    assert dp * req == pytest.approx(sigma, rel=0.07)
    # one chemical potential: both bulk values moved by the same Kelvin shift
    # (to 5 %; the centre and corner nodes still carry interface tails)
    shift = eos.mu0(rin) - eos.mu0(rl)
    assert abs(eos.mu0(rin) - eos.mu0(rout)) < 0.05 * abs(shift)
    # and the drop is at rest: the residual (spurious) flow is small
    assert float(m["u"].abs().max()) < 1e-4
    # both phases moved off the flat coexistence densities the way the Kelvin
    # effect does: the pressure jump raises both densities
    assert rin > rl and rout > rv


def contact_angle_2d(rho, mid, wall=0.5, zmin=2):
    """Circle fit to the mid-density contour of a drop on the wall plane
    z = wall (rows z >= zmin, points interpolated along x); the angle inside
    the liquid."""
    pts = []
    nz, nx = rho.shape
    for z in range(zmin, nz - 2):
        row = rho[z]
        for x in range(nx - 1):
            if (row[x] - mid) * (row[x + 1] - mid) < 0:
                pts.append((x + (mid - row[x]) / (row[x + 1] - row[x]), float(z)))
    P = np.array(pts)
    A = np.c_[2 * P, np.ones(len(P))]
    cx, cz, c = np.linalg.lstsq(A, (P ** 2).sum(1), rcond=None)[0]
    rad = math.sqrt(c + cx * cx + cz * cz)
    return math.degrees(math.acos(max(-1.0, min(1.0, -(cz - wall) / rad))))


def test_neutral_wetting_contact_angle():
    """Sec. III C: with the surface density set to the fluid-weighted average
    (Eq. 37, no contact-line modification) and the surface chemical potential
    of Eq. 36, a drop keeps neutral wetting, 90 degrees (the paper prints
    89.9 for its 3-D drop).  A half-cylinder on the bottom wall of a
    40 x 1 x 20 domain (solid planes z = 0 and 19), angle from a circle fit
    to the mid-density contour."""
    eos, p, rl, rv = setup(wetting_mode=0)
    nx, nz = 40, 20
    mask = I.wall_mask(nx, 1, nz, planes=(0, nz - 1))
    solid = torch.from_numpy(mask.astype(bool))
    rho0 = I.sessile_droplet(nx, 1, nz, 8.0, rl, rv, wall_z=0.5)
    f = S.initial_populations(torch.from_numpy(rho0), None, solid, p)
    f = S.run(f, solid, p, 500)
    m = S.macroscopic(f, solid, p)
    theta = contact_angle_2d(m["rho"][:, 0, :].numpy(), 0.5 * (rl + rv))
    assert theta == pytest.approx(GOLD["contact_angles"]["neutral"], abs=1.5)
    assert float(m["mass"]) == pytest.approx(float(rho0[~mask.astype(bool)].sum()), rel=1e-12)


def _wetting_angle(mode, value, nsteps=400):
    eos, p, rl, rv = setup(wetting_mode=mode, wetting_value=value)
    nx, nz = 40, 20
    mask = I.wall_mask(nx, 1, nz, planes=(0, nz - 1))
    solid = torch.from_numpy(mask.astype(bool))
    rho0 = I.sessile_droplet(nx, 1, nz, 8.0, rl, rv, wall_z=0.5)
    f = S.run(S.initial_populations(torch.from_numpy(rho0), None, solid, p), solid, p, nsteps)
    m = S.macroscopic(f, solid, p)
    assert float(m["mass"]) == pytest.approx(float(rho0[~mask.astype(bool)].sum()), rel=1e-12)
    return contact_angle_2d(m["rho"][:, 0, :].numpy(), 0.5 * (rl + rv))


def test_wetting_parameter_sets_the_contact_angle():
    """Sec. III C, Eq. 38: inside the contact-line band the surface density
    becomes phi * rho_ave (phi > 1) or rho_ave - delta_rho (delta_rho > 0),
    limited to the band.  A denser surface attracts the liquid, so the phi
    branch makes the wall hydrophilic (angle below 90 degrees, falling as phi
    grows); a lighter one repels it, so the delta-rho branch makes it
    hydrophobic (above 90 degrees, rising with delta_rho).  The paper's 3-D
    drops give 33.5 degrees at phi = 1.6 and 153.4 at delta_rho = 1.8; the
    quasi-2-D half-cylinder of the neutral-angle test (40 x 1 x 20, 400 steps,
    where the angle has settled) is held to the direction and the ordering:
    measured 67.9 and about 52 degrees for phi = 1.2 and 1.4, 105 and 120
    degrees for delta_rho = 0.5 and 1.0.  Applying phi as 1/phi, adding
    delta_rho, or exchanging the two branches fails the ordering."""
    phi12, phi14 = _wetting_angle(1, 1.2), _wetting_angle(1, 1.4)
    d05, d10 = _wetting_angle(2, 0.5), _wetting_angle(2, 1.0)
    assert phi14 < phi12 < 85.0
    assert 95.0 < d05 < d10
    assert phi14 + 5.0 < phi12 and d05 + 5.0 < d10


def test_translated_cylinder_keeps_its_shape(monkeypatch):
    """Sec. III B: with the third- and fourth-order corrections the model is
    Galilean invariant, so a drop carried by a uniform flow keeps its shape
    (models without them deform it).  An equilibrated cylinder is given a
    uniform velocity U = 0.1 and run for one period of the box (320 steps);
    the droplet position drifts a little (momentum is conserved only to the
    lattice force balance), so shapes are compared about their own centroid:
    the density field re-centred by a Fourier shift matches the stationary
    one to 8 % of the density contrast and the drop stays round to 3 %
    (measured 5.7 % and 2 %).  The same run without the corrections (Q = 0,
    hence no fourth-order term either) goes non-finite."""
    err, asp = _translate(1.0, monkeypatch)
    assert err < 0.08
    assert asp == pytest.approx(1.0, abs=0.03)
    err0, _ = _translate(0.0, monkeypatch)
    assert not err0 < 3 * 0.08


def _translate(q_scale, monkeypatch):
    eos, p, rl, rv = setup()
    n = 32
    solid = torch.zeros(1, n, n, dtype=torch.bool)
    f = S.initial_populations(torch.from_numpy(cylinder(n, 8.0, rl, rv)), None, solid, p)
    rest = S.macroscopic(S.run(f, solid, p, 300), solid, p)["rho"][0]
    u0 = torch.zeros(3, 1, n, n, dtype=torch.float64)
    u0[0] = 0.1
    f = S.initial_populations(rest.view(1, n, n), u0, solid, p)
    orig = S.fields

    def scaled(ff, ss, pp):
        d = orig(ff, ss, pp)
        d["Q"] = d["Q"] * q_scale
        return d

    monkeypatch.setattr(S, "fields", scaled)
    moved = S.macroscopic(S.run(f, solid, p, 320), solid, p)["rho"][0]
    monkeypatch.setattr(S, "fields", orig)
    if not torch.isfinite(moved).all():
        return math.inf, math.inf

    def centroid(r, axis):
        ang = 2 * math.pi * torch.arange(n, dtype=torch.float64) / n
        w = (r - rv).sum(dim=1 - axis)
        return math.atan2(float((w * torch.sin(ang)).sum()), float((w * torch.cos(ang)).sum())) / (2 * math.pi) * n

    dx = centroid(moved, 1) - centroid(rest, 1)
    dy = centroid(moved, 0) - centroid(rest, 0)
    kx = torch.fft.fftfreq(n, dtype=torch.float64).view(1, n)
    ky = torch.fft.fftfreq(n, dtype=torch.float64).view(n, 1)
    back = torch.fft.ifft2(torch.fft.fft2(moved) * torch.exp(2j * math.pi * (kx * dx + ky * dy))).real
    err = float((back - rest).abs().max()) / (rl - rv)

    def aspect(r):
        w = (r - rv).clamp_min(0)
        cx, cy = centroid(r, 1), centroid(r, 0)
        x = torch.arange(n, dtype=torch.float64)
        ddx = torch.remainder(x - cx + n / 2, n) - n / 2
        ddy = torch.remainder(x - cy + n / 2, n) - n / 2
        ixx = float((w * ddx.view(1, n) ** 2).sum())
        iyy = float((w * ddy.view(n, 1) ** 2).sum())
        return ixx / iyy

    return err, aspect(moved)


@pytest.mark.parametrize("mode", ["nu", "omega1"])
def test_shear_wave_decays_at_the_model_viscosity(mode):
    """Sec. II B: omega_1 relaxes the shear moments, and the nu-mode sets it per
    node by 1/omega_1 = rho nu / p_m + 1/2, i.e. a kinematic viscosity
    nu = (p_m / rho)(1/omega_1 - 1/2) (the generalized equilibrium carries p_m,
    not rho c_s^2, in its second moments).  A transverse wave u_x = U sin(k z)
    in a uniform liquid (no force, no Q: the flow has no x dependence) must
    decay as exp(-nu k^2 t), the Navier-Stokes closed form.  In this liquid
    p_m / rho = 0.044, far from c_s^2 = 1/3, so the check tells the two apart.
    Measured on 1 x 1 x 32 nodes between steps 40 and 340 (after the start-up
    transient of the equilibrium initial state): -0.9 % (nu-mode) and +0.06 %
    (omega_1 = 1.25) from the closed form; held to 2 %."""
    eos, p, rl, rv = setup()
    nz, U = 32, 1e-3
    solid = torch.zeros(nz, 1, 1, dtype=torch.bool)
    rho0 = torch.full((nz, 1, 1), rl, dtype=torch.float64)
    pm = float((1.0 + S.mu0(rho0, p)[0, 0, 0]) / 3.0)
    if mode == "nu":
        p.nu = 0.04
        nu = p.nu
    else:
        om = [1.0] * 11
        om[1] = 1.25
        p.omega = om
        nu = pm / rl * (1.0 / 1.25 - 0.5)
    k = 2.0 * math.pi / nz
    z = torch.arange(nz, dtype=torch.float64)
    u0 = torch.zeros(3, nz, 1, 1, dtype=torch.float64)
    u0[0, :, 0, 0] = U * torch.sin(k * z)
    f = S.initial_populations(rho0, u0, solid, p)

    def amplitude(ff):
        ux = S.macroscopic(ff, solid, p)["u"][0, :, 0, 0]
        return float(2.0 / nz * (ux * torch.sin(k * z)).sum())

    f = S.run(f, solid, p, 40)
    a1 = amplitude(f)
    f = S.run(f, solid, p, 300)
    a2 = amplitude(f)
    rate = math.log(a1 / a2) / 300.0
    assert rate == pytest.approx(nu * k * k, rel=0.02)


def test_sound_wave_frequency_follows_the_eos_and_capillarity():
    """Sec. II: the force F = (1/3 - rho) grad mu with the pressure p_m of the
    generalized equilibrium leaves -rho grad mu in the momentum equation, so a
    small density wave rho_l (1 + eps cos kz) in the liquid oscillates at
    omega^2 = k^2 rho (mu0'(rho) + kappa lambda_k), with lambda_k = 2(1 - cos k)
    the eigenvalue of minus the lattice Laplacian (Eq. 2) and mu0' of the vdW
    EOS (Eq. 32).  On the lattice k becomes sin k, the eigenvalue of the
    model's gradient stencil for this mode (O(k^2) dispersion).  At 0.7 T_c,
    kappa = 0.02 on 1 x 1 x 32 nodes the period is 61.8 steps; the capillary
    term moves omega by 1 %, and a pressure of rho / 3 instead would move it
    by 11 %.  The period from interpolated zero crossings of the mode
    amplitude over six periods is held to 0.3 % (measured +0.12 %; +0.03 % on
    64 nodes, where the k form is off by -0.13 % against -0.52 % on 32)."""
    eos, p, rl, rv = setup()
    nz, eps = 32, 1e-5
    solid = torch.zeros(nz, 1, 1, dtype=torch.bool)
    k = 2.0 * math.pi / nz
    z = torch.arange(nz, dtype=torch.float64)
    rho0 = (rl * (1.0 + eps * torch.cos(k * z))).view(nz, 1, 1)
    h = 1e-6
    dmu0 = (eos.mu0(rl + h) - eos.mu0(rl - h)) / (2.0 * h)
    omega = math.sin(k) * math.sqrt(rl * (dmu0 + p.kappa * 2.0 * (1.0 - math.cos(k))))
    f = S.initial_populations(rho0, None, solid, p)
    amp = []
    for _ in range(400):
        r = S.macroscopic(f, solid, p)["rho"][:, 0, 0]
        amp.append(float(((r - r.mean()) * torch.cos(k * z)).sum()))
        f = S.step(f, solid, p)
    cross = [i - 1 + amp[i - 1] / (amp[i - 1] - amp[i]) for i in range(1, len(amp))
             if (amp[i - 1] > 0.0) != (amp[i] > 0.0)]
    period = 2.0 * (cross[-1] - cross[0]) / (len(cross) - 1)
    assert len(cross) >= 12
    assert 2.0 * math.pi / period == pytest.approx(omega, rel=0.003)


def _vapour_between_walls(omega3, nsteps):
    """max |u| every 20 steps of uniform vapour at 0.7 T_c (nu = 0.15)
    between halfway bounce-back walls (8 x 8 x 8, solid planes z = 0, 7),
    seeded with N(0, 1e-3^2) density noise."""
    om = [1.0] * 11
    om[3] = omega3
    eos, p, rl, rv = setup(nu=0.15, omega=om)
    n = 8
    solid = torch.from_numpy(I.wall_mask(n, n, n, planes=(0, n - 1)).astype(bool))
    rho = I.add_noise(np.full((n, n, n), rv), 1e-3, seed=3)
    f = S.initial_populations(torch.from_numpy(rho), None, solid, p)
    out = []
    for _ in range(nsteps // 20):
        f = S.run(f, solid, p, 20)
        out.append(float(S.macroscopic(f, solid, p)["u"].abs().max()))
    return out


def test_vapour_at_a_wall_needs_a_lower_third_order_rate():
    """Sec. III C runs its drops at 0.7 T_c and nu = 0.15 between halfway
    bounce-back walls with every rate but omega_1 equal to 1 (Sec. II B).
    There the vapour (rho_v = 0.448) carries p_m = (1 + mu)/3 ~ 1/3, 0.74
    rho: far from rho c_s^2, with a negative rest population.  Uniform vapour
    between two walls, with only density noise, grows a mode in the first
    fluid layer (wall-tangential wavenumber pi) by more than two orders of
    magnitude in 60 steps.  Without the walls the same vapour relaxes; with
    the force and the Q terms switched off it still grows, so the mode needs
    neither the force nor Eq. 27, only the equilibrium and the bounce-back.
    omega_3 (the symmetric third-order moments, Eq. 23) in [0.3, 0.6] damps
    it; omega_4, omega_5 and the rates of the other orders do not.  The
    static equilibrium, hence the contact angle, does not depend on the
    rates; the paper's wall runs are made with omega_3 = 0.5."""
    grows = _vapour_between_walls(1.0, 80)
    assert grows[-1] > 100.0 * grows[0]
    decays = _vapour_between_walls(0.5, 200)
    assert decays[-1] < 0.1 * decays[0]
    assert all(np.isfinite(decays))
