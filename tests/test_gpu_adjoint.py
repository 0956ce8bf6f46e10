"""GPU discrete adjoint against the FP64 oracle's reverse mode (whose own
gradients are pinned by central differences in test_oracle_adjoint.py).

The adjoint is linear in lambda; FP32 evaluation of the transposed step is
expected within ~1e-6 of the largest component per step.  The bounds below
are 1e-4 relative for one step (FP32 of a linear map with magnitudes up to
~10) and the method's gradient contract, 1e-3 relative, for multi-step
gradients.
"""
import copy

import numpy as np
import pytest
import torch

from oracle import adjoint as OA
from oracle import step as S
from paper_2504_03819_gb300 import Domain
from paper_2504_03819_gb300 import binding as Bd
from paper_2504_03819_gb300.adjoint import LBMRollout, rollout_gradient, theta_of
from paper_2504_03819_gb300 import inputs as I

from _cases import CASES, build, oracle_init, oracle_params, perturbed

pytestmark = pytest.mark.gpu
DT = torch.float64


def gpu(case):
    nx, ny, nz = case["n"]
    d = Domain(nx, ny, nz, "f32", solid_mask=case["mask"] if case["mask"].any() else None)
    d.set_params(case["p"])
    return d


def relmax(a, b):
    a, b = a.double().cpu(), b.double().cpu()
    return float((a - b).abs().max()) / max(float(b.abs().max()), 1e-30)


def oracle_theta_grads(case, f, lam):
    """lambda_t and [kappa, omega.., wetting] cotangents of one oracle step."""
    solid = torch.from_numpy(case["mask"].astype(bool))
    lt, gk, go, gw = OA.step_vjp(f, solid, oracle_params(case["p"]), lam)
    return lt, torch.cat([gk.view(1), go.view(11), gw.view(1)])


@pytest.mark.parametrize("name", list(CASES))
def test_one_adjoint_step(name):
    case = build(name)
    fr = perturbed(case, oracle_init(case), seed=31)
    nx, ny, nz = case["n"]
    g = torch.Generator().manual_seed(7)
    fluid = torch.from_numpy(~case["mask"].astype(bool)).to(DT)
    lam = torch.randn(27, nz, ny, nx, generator=g, dtype=DT) * fluid
    lam = lam.float().double()
    d = gpu(case)
    d.set_populations(fr.float())
    raw = d.get_state().clone()
    grad = torch.zeros(Bd.NGRAD, dtype=DT, device="cuda")
    lt = d.adjoint_step(raw, lam.float().cuda(), grad)
    ref_lt, ref_g = oracle_theta_grads(case, fr, lam)
    assert relmax(lt, ref_lt) < 1e-4
    gg = grad.cpu()
    scale = float(ref_g.abs().max())
    # omega_0 has no effect (k100* = F/2): exactly zero in both
    assert abs(float(ref_g[1])) < 1e-9 * scale
    assert float((gg - ref_g).abs().max()) / scale < 1e-4, (gg, ref_g)


@pytest.mark.parametrize("kind,name", [(Bd.OBJ_ENERGY, "droplet_periodic"), (Bd.OBJ_ENERGY, "wall_phi"),
                                       (Bd.OBJ_CENTROID_X, "droplet_periodic"),
                                       (Bd.OBJ_CONTACT_RADIUS, "wall_phi"), (Bd.OBJ_CONTACT_RADIUS, "wall_delta_nu")])
def test_objective_value_and_seed(kind, name):
    case = build(name)
    fr = perturbed(case, oracle_init(case), seed=41)
    d = gpu(case)
    d.set_populations(fr.float())
    grad = torch.zeros(Bd.NGRAD, dtype=DT, device="cuda")
    J, lam = d.objective(kind, wall_z=0, grad=grad)
    solid = torch.from_numpy(case["mask"].astype(bool))
    op = copy.copy(oracle_params(case["p"]))
    kappa = torch.tensor(float(op.kappa), dtype=DT, requires_grad=True)
    wv = torch.tensor(float(op.wetting_value), dtype=DT, requires_grad=True)
    op.kappa, op.wetting_value = kappa, wv
    onames = {Bd.OBJ_ENERGY: "energy", Bd.OBJ_CENTROID_X: "centroid_x", Bd.OBJ_CONTACT_RADIUS: "contact_radius"}
    f = fr.clone().requires_grad_(True)
    Jr = OA.objective(onames[kind], f, solid, op, wall_z=0)
    gr, gk, gw = torch.autograd.grad(Jr, (f, kappa, wv), allow_unused=True)
    assert float(J[0]) == pytest.approx(float(Jr.detach()), rel=2e-6, abs=1e-12)
    assert relmax(lam, gr) < 1e-4
    gk = 0.0 if gk is None else float(gk)
    gw = 0.0 if gw is None else float(gw)
    gg = grad.cpu()
    assert float(gg[0]) == pytest.approx(gk, rel=1e-4, abs=1e-9)
    if case["p"].wetting_mode != 0:
        assert float(gg[12]) == pytest.approx(gw, rel=1e-4, abs=1e-9)


@pytest.mark.parametrize("name", ["wall_phi", "wall_delta_nu", "droplet_periodic"])
def test_initialisation_adjoint(name):
    case = build(name)
    nx, ny, nz = case["n"]
    g = torch.Generator().manual_seed(3)
    fluid = torch.from_numpy(~case["mask"].astype(bool)).to(DT)
    lam0 = (torch.randn(27, nz, ny, nx, generator=g, dtype=DT) * fluid).float().double()
    d = gpu(case)
    grad = torch.zeros(Bd.NGRAD, dtype=DT, device="cuda")
    g_rho0 = d.adjoint_init(torch.from_numpy(case["rho0"]).float(), torch.from_numpy(case["u0"]).float(),
                            lam0.float(), grad)
    solid = torch.from_numpy(case["mask"].astype(bool))
    q = copy.copy(oracle_params(case["p"]))
    kappa = torch.tensor(float(q.kappa), dtype=DT, requires_grad=True)
    wv = torch.tensor(float(q.wetting_value), dtype=DT, requires_grad=True)
    q.kappa, q.wetting_value = kappa, wv
    r0 = torch.from_numpy(case["rho0"]).clone().requires_grad_(True)
    f0 = S.initial_populations(r0, torch.from_numpy(case["u0"]), solid, q)
    gr, gk, gw = torch.autograd.grad((f0 * lam0).sum(), (r0, kappa, wv), allow_unused=True)
    gr = torch.where(solid, torch.zeros_like(gr), gr)
    assert relmax(g_rho0, gr) < 1e-4
    gg = grad.cpu()
    assert float(gg[0]) == pytest.approx(float(gk), rel=1e-4, abs=1e-6 * float(gr.abs().max()))
    if gw is not None and case["p"].wetting_mode != 0:
        assert float(gg[12]) == pytest.approx(float(gw), rel=1e-4, abs=1e-6 * float(gr.abs().max()))


def sessile_case(n=8, mode=1, value=1.3):
    from _cases import vdw, f32
    p = vdw(wetting_mode=mode, wetting_value=value)
    p.omega = [1.0, 1.3] + [1.0] * 9
    mask = I.wall_mask(n, n, n, planes=(0, n - 1))
    rho0 = f32(I.add_noise(I.sessile_droplet(n, n, n, 3.0, p.rho_l, p.rho_v), 1e-3, seed=12345))
    return p, mask, rho0


@pytest.mark.parametrize("objective", [Bd.OBJ_CONTACT_RADIUS, Bd.OBJ_ENERGY])
def test_rollout_gradient_matches_fp64_adjoint(objective):
    """Gradient of the contact-line radius / kinetic energy after 6 steps on
    an 8^3 wall case (checkpoints every 2 steps) against the oracle's FP64
    reverse mode: kappa, omega_1, wetting value and the initial density."""
    p, mask, rho0 = sessile_case()
    n = 8
    d = Domain(n, n, n, "f32", solid_mask=mask)
    d.set_params(p)
    J, grad, g_rho0 = rollout_gradient(d, torch.from_numpy(rho0).float(), None, 6, 2, objective, wall_z=0)
    solid = torch.from_numpy(mask.astype(bool))
    onames = {Bd.OBJ_ENERGY: "energy", Bd.OBJ_CONTACT_RADIUS: "contact_radius"}
    ref = OA.gradients(torch.from_numpy(rho0), None, solid, oracle_params(p), 6, onames[objective])
    assert J == pytest.approx(ref["J"], rel=1e-5)
    gg = grad.cpu()
    for i, key in ((0, "kappa"), (12, "wetting_value")):
        assert float(gg[i]) == pytest.approx(ref[key], rel=1e-3, abs=1e-6 * abs(ref[key]) + 1e-12), key
    assert float(gg[2]) == pytest.approx(float(ref["omega"][1]), rel=1e-3)
    assert relmax(g_rho0, ref["rho0"]) < 1e-3


def test_wall_workload_copy_gradient_matches_fp64_adjoint():
    """Scaled copy of the differentiable droplet-on-a-wall workload (64^3, R =
    16, K = 100): 16^3 with solid planes z = 0 and 15, a hemisphere of R = 4
    with N(0, 1e-3) noise from default_rng(12345) on the initial density,
    phi-wetting 1.2 and all rates 1, at 0.85 T_c with the paper's EOS
    coefficient and kappa (a = 9/392, kappa = 0.02: with a = 9/49, kappa =
    0.01 this workload goes non-finite).  Contact-line radius after 40 steps
    with checkpoints every 10 steps (four segments, each recomputed from its
    checkpoint): dJ/d kappa, omega_1, phi and the initial density against the
    oracle's FP64 reverse mode, to the gradient contract 1e-3."""
    from _cases import A392, vdw, f32
    n, T, K = 16, 40, 10
    p = vdw(a=A392, t=0.85, kappa=0.02, wetting_mode=1, wetting_value=1.2)
    mask = I.wall_mask(n, n, n, planes=(0, n - 1))
    rho0 = f32(I.add_noise(I.sessile_droplet(n, n, n, 4.0, p.rho_l, p.rho_v), 1e-3, seed=12345))
    d = Domain(n, n, n, "f32", solid_mask=mask)
    d.set_params(p)
    J, grad, g_rho0 = rollout_gradient(d, torch.from_numpy(rho0).float(), None, T, K, Bd.OBJ_CONTACT_RADIUS,
                                       wall_z=0)
    solid = torch.from_numpy(mask.astype(bool))
    ref = OA.gradients(torch.from_numpy(rho0), None, solid, oracle_params(p), T, "contact_radius")
    assert J == pytest.approx(ref["J"], rel=1e-5)
    gg = grad.cpu()
    assert float(gg[0]) == pytest.approx(ref["kappa"], rel=1e-3)
    assert float(gg[2]) == pytest.approx(float(ref["omega"][1]), rel=1e-3)
    assert float(gg[12]) == pytest.approx(ref["wetting_value"], rel=1e-3)
    assert relmax(g_rho0, ref["rho0"]) < 1e-3


def test_autograd_function_backward():
    p, mask, rho0 = sessile_case(mode=2, value=0.6)
    n = 8
    d = Domain(n, n, n, "f32", solid_mask=mask)
    r0 = torch.from_numpy(rho0).clone().requires_grad_(True)
    theta = theta_of(p).requires_grad_(True)
    J = LBMRollout.apply(r0, theta, d, p, None, 4, 2, Bd.OBJ_CONTACT_RADIUS, 0)
    J.backward()
    solid = torch.from_numpy(mask.astype(bool))
    ref = OA.gradients(torch.from_numpy(rho0), None, solid, oracle_params(p), 4, "contact_radius")
    assert float(J) == pytest.approx(ref["J"], rel=1e-5)
    assert float(theta.grad[12]) == pytest.approx(ref["wetting_value"], rel=1e-3)
    assert relmax(r0.grad, ref["rho0"]) < 1e-3


def test_adjoint_step_bitwise_deterministic():
    """Two domains built independently (their own boundary lists) give the
    same lambda(t) and parameter gradient bit for bit: every reduction of the
    adjoint runs in a fixed order."""
    case = build("wall_tiles")
    fr = perturbed(case, oracle_init(case), seed=51)
    nx, ny, nz = case["n"]
    g = torch.Generator().manual_seed(8)
    lam = (torch.randn(27, nz, ny, nx, generator=g, dtype=DT)
           * torch.from_numpy(~case["mask"].astype(bool)).to(DT)).float().cuda()
    out = []
    for _ in range(2):
        d = gpu(case)
        d.set_populations(fr.float())
        raw = d.get_state().clone()
        grad = torch.zeros(Bd.NGRAD, dtype=DT, device="cuda")
        lt = d.adjoint_step(raw, lam, grad)
        out.append((lt.clone(), grad.clone()))
        d.close()
    assert torch.equal(out[0][0], out[1][0])
    assert torch.equal(out[0][1], out[1][1])


@pytest.mark.parametrize("name", ["droplet_tiles", "wall_tiles"])
def test_one_adjoint_step_fp16_storage(name):
    """The adjoint with FP16 population storage: the oracle's reverse mode at
    the populations the FP16 state holds (read back through
    lbm_get_populations), so both sides linearise the same state."""
    case = build(name)
    fr = perturbed(case, oracle_init(case), seed=61)
    nx, ny, nz = case["n"]
    d = Domain(nx, ny, nz, "f16", solid_mask=case["mask"] if case["mask"].any() else None)
    d.set_params(case["p"])
    d.set_populations(fr.float())
    held = d.get_populations().double().cpu()
    g = torch.Generator().manual_seed(12)
    fluid = torch.from_numpy(~case["mask"].astype(bool)).to(DT)
    lam = (torch.randn(27, nz, ny, nx, generator=g, dtype=DT) * fluid).float().double()
    raw = d.get_state().clone()
    grad = torch.zeros(Bd.NGRAD, dtype=DT, device="cuda")
    lt = d.adjoint_step(raw, lam.float().cuda(), grad)
    ref_lt, ref_g = oracle_theta_grads(case, held, lam)
    assert relmax(lt, ref_lt) < 1e-4
    scale = float(ref_g.abs().max())
    assert float((grad.cpu() - ref_g).abs().max()) / scale < 1e-4
