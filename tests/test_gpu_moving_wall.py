"""Moving walls on the GPU (lbm_set_wall_velocity) against the FP64 oracle:
the exact Couette profile, one step and fifty steps with seeded wall
velocities in every direction, and the adjoint of a step.  Tolerances as in
test_gpu_parity.py and test_gpu_adjoint.py.
"""
import numpy as np
import pytest
import torch

from oracle import adjoint as OA
from oracle import step as S
from paper_2504_03819_gb300 import Domain
from paper_2504_03819_gb300 import binding as Bd
from paper_2504_03819_gb300 import inputs as I

from _cases import build, oracle_init, oracle_params, perturbed, vdw

pytestmark = pytest.mark.gpu
DT = torch.float64


def seeded_wall_u(case, seed, scale=0.02):
    nx, ny, nz = case["n"]
    g = np.random.default_rng(seed)
    u = (scale * g.standard_normal((3, nz, ny, nx))).astype(np.float32)
    u[:, ~case["mask"].astype(bool)] = 0.0
    return torch.from_numpy(u)


def gpu(case, wall_u):
    nx, ny, nz = case["n"]
    d = Domain(nx, ny, nz, "f32", solid_mask=case["mask"])
    d.set_params(case["p"])
    d.set_wall_velocity(wall_u)
    return d


def oracle_p(case, wall_u):
    op = oracle_params(case["p"])
    op.wall_u = wall_u.double()
    return op


def test_couette_channel_profile():
    """8 x 8 x 12, walls z = 0 (at rest) and z = 11 (U = 0.01 along x),
    uniform density: the exact linear profile between the halfway planes."""
    p = vdw()
    nx, ny, nz, U = 8, 8, 12, 0.01
    mask = I.wall_mask(nx, ny, nz, planes=(0, nz - 1))
    wu = np.zeros((3, nz, ny, nx), np.float32)
    wu[0, nz - 1] = U
    d = Domain(nx, ny, nz, "f32", solid_mask=mask)
    d.set_params(p)
    d.set_wall_velocity(torch.from_numpy(wu))
    d.set_state(torch.full((nz, ny, nx), 2.0))
    d.step(1500)
    assert d.sync_status() == 0
    ux = d.moments()["u"][0, 1:nz - 1].double().cpu()
    exact = U * (torch.arange(1, nz - 1, dtype=DT) - 0.5) / (nz - 2)
    assert float((ux - exact.view(-1, 1, 1)).abs().max()) < 1e-4 * U


@pytest.mark.parametrize("name", ["wall_tiles", "wall_phi", "wall_delta_nu"])
def test_one_step_with_moving_walls(name):
    case = build(name)
    wu = seeded_wall_u(case, seed=3)
    fr = perturbed(case, oracle_init(case), seed=23)
    d = gpu(case, wu)
    d.set_populations(fr.float())
    d.step(1)
    assert d.sync_status() == 0
    got = d.get_populations().cpu()
    ref = S.step(fr, torch.from_numpy(case["mask"].astype(bool)), oracle_p(case, wu))
    assert float((got.double() - ref).abs().max()) / float(ref.abs().max()) < 2e-6


def test_fifty_steps_with_moving_walls():
    case = build("wall_tiles")
    wu = torch.zeros(3, *case["mask"].shape)
    wu[0][torch.from_numpy(case["mask"].astype(bool))] = 0.02
    wu[1][torch.from_numpy(case["mask"].astype(bool))] = -0.01
    d = gpu(case, wu)
    d.set_state(torch.from_numpy(case["rho0"]).float(), torch.from_numpy(case["u0"]).float())
    d.step(50)
    assert d.sync_status() == 0
    m = d.moments()
    solid = torch.from_numpy(case["mask"].astype(bool))
    op = oracle_p(case, wu)
    ref = S.macroscopic(S.run(oracle_init(case), solid, op, 50), solid, op)
    fl = ~solid
    r = ref["rho"][fl]
    assert float(((m["rho"].double().cpu()[fl] - r).abs() / r.abs()).max()) < 1e-5
    assert float((m["u"].double().cpu() - ref["u"]).abs().max()) < 1e-6
    assert m["mass"] == pytest.approx(float(ref["mass"]), rel=1e-6)


@pytest.mark.parametrize("name", ["wall_tiles", "wall_delta_nu"])
def test_adjoint_step_with_moving_walls(name):
    case = build(name)
    wu = seeded_wall_u(case, seed=4)
    fr = perturbed(case, oracle_init(case), seed=33)
    nx, ny, nz = case["n"]
    g = torch.Generator().manual_seed(9)
    fluid = torch.from_numpy(~case["mask"].astype(bool)).to(DT)
    lam = (torch.randn(27, nz, ny, nx, generator=g, dtype=DT) * fluid).float().double()
    d = gpu(case, wu)
    d.set_populations(fr.float())
    raw = d.get_state().clone()
    grad = torch.zeros(Bd.NGRAD, dtype=DT, device="cuda")
    lt = d.adjoint_step(raw, lam.float().cuda(), grad)
    solid = torch.from_numpy(case["mask"].astype(bool))
    ref_lt, gk, go, gw = OA.step_vjp(fr, solid, oracle_p(case, wu), lam)
    scale = float(ref_lt.abs().max())
    assert float((lt.double().cpu() - ref_lt).abs().max()) / scale < 1e-4
    ref_g = torch.cat([gk.view(1), go.view(11), gw.view(1)])
    assert float((grad.cpu() - ref_g).abs().max()) / float(ref_g.abs().max()) < 1e-4
