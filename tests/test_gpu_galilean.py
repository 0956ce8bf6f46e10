"""The moving-droplet workload's own output: shape drift against the
translated stationary droplet, FP32 and FP16 storage.

A Galilean-invariant model (Sec. II B: the collision in the frame moving
with u; the third- and fourth-order corrections of Eqs. 27-28) carries a
drop with the flow without deforming it, so the moving field equals the
stationary run's field shifted by the drop's displacement.

The workload as stated (256^3 periodic, R = 32, width 2, U = (0.05, 0.02,
0), a = 9/49, b = 2/21, kappa = 0.01 at 0.85 T_c, omega_1 = 1.6) cannot
show it: its equilibrium interface is 1.16 nodes wide and the lattice holds
the drop in place while the vapour flows past (the second test).  The
check therefore runs the workload's geometry and velocity with the paper's
own drop setup (a = 9/392, kappa = 0.02, 0.7 T_c, nu = 0.15, width 5:
interface 3.1 nodes), 20 000 steps, beside a stationary run (U = 0) of the
same storage.  Measured, FP32 (FP16):
* the drop travels along U (displacement y / x = 0.399 (0.391) against
  0.4; z below 0.01 node) but trails the flow and slows down: 85 of the
  100 nodes of U t by step 2000, 449 (456) of 1000 by step 20 000.  The
  lattice sum of F = (1/3 - rho) grad mu vanishes only at equilibrium, so a
  moving interface loses momentum (as in the moving-wall run);
* shape: the moving field moved back by its measured displacement (Fourier
  shift) differs from the stationary one by 0.21-0.36 % of the density
  contrast (rms over the domain; the maximum, 14-33 %, sits at the
  interface where a fraction of a node of misplacement shows), and the
  liquid's principal radii of gyration agree to 1.2 % (aspect 1.010 (1.012)
  at step 2000, 1.002 at step 20 000; the stationary drop 1.0000);
* FP16 storage travels 1.4 % further than FP32 and keeps the same shape
  figures.
Analysis only (torch on the device); every step runs in the library.
"""
import math

import numpy as np
import pytest
import torch

from paper_2504_03819_gb300 import Domain, Params
from paper_2504_03819_gb300 import inputs as I

pytestmark = pytest.mark.gpu

N, RADIUS, U = 256, 32.0, (0.05, 0.02, 0.0)
CHECK = (2000, 5000, 10000, 20000)


def _params(eos):
    om = [1.0] * 11
    if eos == "stated":  # a = 9/49, kappa = 0.01, 0.85 T_c, omega_1 = 1.6
        om[1] = 1.6
        p = Params.vdw(9.0 / 49.0, 2.0 / 21.0, 1.0, 0.85, 0.01, omega=om)
    else:  # the paper's drop runs: a = 9/392, kappa = 0.02, 0.7 T_c, nu = 0.15
        p = Params.vdw(9.0 / 392.0, 2.0 / 21.0, 1.0, 0.7, 0.02, omega=om, nu=0.15)
    p.rho_shift = 2.0 * p.rho_l * p.rho_v / (p.rho_l + p.rho_v)
    return p


def _domain(storage, p, u, width):
    d = Domain(N, N, N, storage)
    d.set_params(p)
    rho0 = I.droplet(N, N, N, RADIUS, p.rho_l, p.rho_v, width=width).astype(np.float32)
    u0 = I.uniform_velocity(N, N, N, u).astype(np.float32)
    d.set_state(torch.from_numpy(rho0), torch.from_numpy(u0))
    return d


def _centroid(rho, rv):
    """Circular mean position per axis (x, y, z) of rho - rho_v."""
    w = rho - rv
    ang = 2.0 * math.pi * torch.arange(N, dtype=torch.float64, device=rho.device) / N
    out = []
    for dim in (2, 1, 0):  # x, y, z of a (z, y, x) field
        prof = w.sum(dim=tuple(k for k in range(3) if k != dim))
        th = math.atan2(float((prof * torch.sin(ang)).sum()), float((prof * torch.cos(ang)).sum()))
        out.append((th % (2.0 * math.pi)) * N / (2.0 * math.pi))
    return out


def _wrap(v):
    return (v + N / 2.0) % N - N / 2.0


def _shape_error(moving, still, disp, contrast):
    """max and rms of |moving(x + disp) - still(x)| / contrast (Fourier shift)."""
    k = torch.fft.fftfreq(N, dtype=torch.float64, device=moving.device)
    ph = (k.view(1, 1, N) * disp[0] + k.view(1, N, 1) * disp[1] + k.view(N, 1, 1) * disp[2])
    back = torch.fft.ifftn(torch.fft.fftn(moving) * torch.exp(2j * math.pi * ph)).real
    diff = (back - still).abs() / contrast
    return float(diff.max()), float(diff.pow(2).mean().sqrt())


def _aspect(rho, rv):
    """sqrt(largest / smallest eigenvalue) of the liquid's gyration tensor."""
    w = (rho - rv).clamp_min(0.0)
    c = _centroid(rho, rv)
    ar = torch.arange(N, dtype=torch.float64, device=rho.device)
    d = [_wrap(ar - c[0]).view(1, 1, N), _wrap(ar - c[1]).view(1, N, 1), _wrap(ar - c[2]).view(N, 1, 1)]
    tot = float(w.sum())
    g = np.zeros((3, 3))
    for a in range(3):
        for b in range(a, 3):
            g[a, b] = g[b, a] = float((w * d[a] * d[b]).sum()) / tot
    ev = np.linalg.eigvalsh(g)
    return math.sqrt(ev[-1] / ev[0])


def _liquid_centroid(rho, level):
    """Circular mean position per axis (x, y, z) of the nodes above level."""
    idx = torch.nonzero(rho > level).double()
    out = []
    for dim in (2, 1, 0):
        a = 2.0 * math.pi * idx[:, dim] / N
        th = math.atan2(float(torch.sin(a).mean()), float(torch.cos(a).mean()))
        out.append((th % (2.0 * math.pi)) * N / (2.0 * math.pi))
    return out


def _run(storage):
    p = _params("paper")
    rl, rv = p.rho_l, p.rho_v
    mov, still = _domain(storage, p, U, 5.0), _domain(storage, p, (0.0, 0.0, 0.0), 5.0)
    rho = lambda d: d.moments()["rho"].double()  # noqa: E731
    c_prev = [a - b for a, b in zip(_centroid(rho(mov), rv), _centroid(rho(still), rv))]
    disp = [0.0, 0.0, 0.0]
    out = {}
    t = 0
    while t < CHECK[-1]:
        mov.step(1000)
        still.step(1000)
        t += 1000
        assert mov.sync_status() == 0 and still.sync_status() == 0
        rm, rs = rho(mov), rho(still)
        assert bool(torch.isfinite(rm).all()) and bool(torch.isfinite(rs).all())
        c = [a - b for a, b in zip(_centroid(rm, rv), _centroid(rs, rv))]
        disp = [s + _wrap(a - b) for s, a, b in zip(disp, c, c_prev)]
        c_prev = c
        if t in CHECK:
            emax, erms = _shape_error(rm, rs, disp, rl - rv)
            out[t] = dict(disp=list(disp), lag=[1.0 - disp[a] / (U[a] * t) if U[a] else None for a in range(3)],
                          err_max=emax, err_rms=erms, aspect=_aspect(rm, rv), aspect_still=_aspect(rs, rv))
            print(storage, t, out[t], flush=True)
    final = rho(mov)
    mov.close()
    still.close()
    return out, final, rl - rv


_TRAVEL = {}


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_moving_droplet_keeps_the_shape_of_the_translated_stationary_one(storage):
    """Held at every checkpoint: rms shape error below 0.6 % of the
    contrast, maximum below 40 %, aspect below 1.02; the displacement along
    U (y / x within 3 % of 0.4, z below 0.05 node) and at least 40 % of U t
    at step 20 000; FP16 and FP32 travel within 3 % of each other."""
    out, _, _ = _run(storage)
    for t, r in out.items():
        assert r["err_rms"] < 0.006, (t, r)
        assert r["err_max"] < 0.4, (t, r)
        assert r["aspect"] < 1.02, (t, r)
        assert r["disp"][1] / r["disp"][0] == pytest.approx(U[1] / U[0], rel=0.03), (t, r)
        assert abs(r["disp"][2]) < 0.05, (t, r)
    last = out[CHECK[-1]]
    assert last["disp"][0] > 0.4 * U[0] * CHECK[-1]
    _TRAVEL[storage] = last["disp"][0]
    if len(_TRAVEL) == 2:
        assert _TRAVEL["f16"] == pytest.approx(_TRAVEL["f32"], rel=0.03)


def test_the_stated_workload_pins_its_drop():
    """The stated set (a = 9/49, kappa = 0.01 at 0.85 T_c) has an equilibrium
    interface (rho_l - rho_v) / max|d rho/dz| = 1.16 nodes wide (the paper's
    a = 9/392, kappa = 0.02 give 4.6 at 0.85 T_c and 3.1 at 0.7 T_c), and an
    interface that thin is held by the lattice: the liquid stops within a few
    hundred steps while the vapour keeps the imposed velocity.  Measured at
    256^3 (R = 32, width 2, U = (0.05, 0.02, 0)): the liquid's mean u_x falls
    from 0.05 to 0.007 by step 250 and to about 0.001 after, the vapour's
    stays at 0.049, and the liquid node set does not change after step 500
    (centroid of the liquid nodes moved 0.008 nodes by step 3000, 0.001
    between steps 500 and 1000).  Held after 1000 steps: liquid mean |u_x| <
    0.005, vapour mean u_x > 0.045, liquid centroid moved less than 0.1 node
    since step 500 (U_x alone would carry it 25)."""
    p = _params("stated")
    rl, rv = p.rho_l, p.rho_v
    d = _domain("f32", p, U, 2.0)
    d.step(500)
    mid = 0.5 * (rl + rv)
    c0 = _liquid_centroid(d.moments()["rho"].double(), mid)
    d.step(500)
    assert d.sync_status() == 0
    m = d.moments()
    rho, u = m["rho"].double(), m["u"].double()
    liq = rho > mid
    c1 = _liquid_centroid(rho, mid)
    d.close()
    assert abs(float(u[0][liq].mean())) < 0.005
    assert float(u[0][~liq].mean()) > 0.045
    assert max(abs(_wrap(a - b)) for a, b in zip(c1, c0)) < 0.1
