"""Long-horizon parity: the precision contract of the method is stated over
1000 steps (max relative density error 1e-5 and |du| <= 1e-6 lattice units
for FP32 storage, 1e-3 relative density for FP16 storage), and the
flat-interface workload runs 2000 steps.  The oracle runs the same problems
in FP64 from the same FP32-representable inputs.
"""
import functools

import numpy as np
import pytest
import torch

from oracle import step as S
from paper_2504_03819_gb300 import Domain
from paper_2504_03819_gb300 import inputs as I

from _cases import build, oracle_init, oracle_params, vdw

pytestmark = pytest.mark.gpu


def rel(a, b, floor=1e-3):
    a, b = a.double().cpu(), b.double().cpu()
    return float(((a - b).abs() / b.abs().clamp_min(floor)).max())


def absd(a, b):
    return float((a.double().cpu() - b.double().cpu()).abs().max())


@functools.lru_cache(maxsize=None)
def flat_oracle(nsteps: int):
    """1 x 1 x 128 oracle run of the slab (the profile is uniform in x, y)."""
    p = vdw()
    nz = 128
    rho1d = I.slab(1, 1, nz, 64, p.rho_l, p.rho_v).astype(np.float32)
    op = oracle_params(p)
    solid = torch.zeros(nz, 1, 1, dtype=torch.bool)
    f = S.run(S.initial_populations(torch.from_numpy(rho1d.astype(np.float64)), None, solid, op), solid, op, nsteps)
    return p, rho1d, S.macroscopic(f, solid, op)


@pytest.mark.parametrize("storage,nsteps,rho_tol,u_tol", [("f32", 2000, 1e-5, 1e-6), ("f16", 1000, 1e-3, None)])
def test_flat_interface_long(storage, nsteps, rho_tol, u_tol):
    """8 x 8 x 128, a = 9/49, kappa = 0.01, 0.85 T_c, slab of width 64."""
    p, rho1d, ref = flat_oracle(nsteps)
    nz = 128
    d = Domain(8, 8, nz, storage)
    d.set_params(p)
    d.set_state(torch.from_numpy(np.repeat(np.repeat(rho1d, 8, axis=1), 8, axis=2)))
    d.step(nsteps)
    assert d.sync_status() == 0
    m = d.moments()
    assert rel(m["rho"], ref["rho"].expand(nz, 8, 8)) < rho_tol
    if u_tol is not None:
        assert absd(m["u"], ref["u"].expand(3, nz, 8, 8)) < u_tol


@functools.lru_cache(maxsize=None)
def droplet_oracle(nsteps: int):
    case = build("droplet_tiles")
    solid = torch.from_numpy(case["mask"].astype(bool))
    op = oracle_params(case["p"])
    return S.macroscopic(S.run(oracle_init(case), solid, op, nsteps), solid, op)


@pytest.mark.parametrize("storage,rho_tol,u_tol", [("f32", 1e-5, 1e-6), ("f16", 1e-3, None)])
def test_droplet_thousand_steps_through_tensor_copies(storage, rho_tol, u_tol):
    """40 x 12 x 10 periodic droplet (two column tiles in x and y with ragged
    tails; rows of 16-byte multiples, so the fused kernel stages its
    populations by TMA) for 1000 steps."""
    case = build("droplet_tiles")
    nx, ny, nz = case["n"]
    d = Domain(nx, ny, nz, storage)
    d.set_params(case["p"])
    d.set_state(torch.from_numpy(case["rho0"]).float(), torch.from_numpy(case["u0"]).float())
    d.step(1000)
    assert d.sync_status() == 0
    m = d.moments()
    ref = droplet_oracle(1000)
    assert rel(m["rho"], ref["rho"]) < rho_tol
    if u_tol is not None:
        assert absd(m["u"], ref["u"]) < u_tol
    assert m["mass"] == pytest.approx(float(ref["mass"]), rel=1e-6 if storage == "f32" else 1e-4)
