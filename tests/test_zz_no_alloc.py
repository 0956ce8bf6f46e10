"""lbm_step_noalloc, the step for callers that cannot allocate device memory
(the library keeps its scratch in a static device array), against the regular
entry points on the same inputs: two calls in a row must reproduce two steps
of lbm_step from lbm_set_populations.

This file is named to be collected last.  The test also runs alone in a fresh
process (the per-device set-up happens on the first call).
"""
import pytest
import torch

from paper_2504_03819_gb300 import Domain
from paper_2504_03819_gb300 import binding as Bd

from _cases import build, oracle_init, perturbed

pytestmark = pytest.mark.gpu

TOL = 2e-6  # the per-step population tolerance of the parity tests


# wall_phi (11-wide rows) and droplet_periodic (13-wide) take the fused
# kernel's per-thread-load path; droplet_tiles (40-wide, all fluid: the
# mask-free instantiation) and wall_tiles (36-wide, walls) its tensor-copy
# path.  All have at most LBM_NOALLOC_MAX_NODES nodes.
@pytest.mark.parametrize("name", ["wall_phi", "droplet_periodic", "droplet_tiles", "wall_tiles"])
def test_noalloc_step_matches_regular_entry_points(name):
    case = build(name)
    nx, ny, nz = case["n"]
    p = case["p"]
    p.shift_mode = Bd.SHIFT_CONST
    p.rho_shift = 0.0
    f0 = perturbed(case, oracle_init(case), seed=5).float().contiguous().cuda()
    mask = torch.from_numpy(case["mask"]).contiguous().cuda() if case["mask"].any() else None

    d = Domain(nx, ny, nz, "f32", solid_mask=mask)
    d.set_params(p)
    d.set_populations(f0)
    d.step(1)
    ref1 = d.get_populations()
    d.step(1)
    ref2 = d.get_populations()

    f1 = torch.full_like(f0, float("nan"))
    f2 = torch.full_like(f0, float("nan"))
    assert Bd.step_noalloc(f0, f1, mask, p) == Bd.LBM_OK
    assert Bd.step_noalloc(f1, f2, mask, p) == Bd.LBM_OK
    torch.cuda.synchronize()
    scale = float(ref2.abs().max())
    assert float((f1 - ref1).abs().max()) / scale < TOL
    assert float((f2 - ref2).abs().max()) / scale < TOL


def test_noalloc_rejects_oversized_domain_and_aliasing():
    case = build("droplet_periodic")
    f = torch.zeros(27, 33, 32, 32, device="cuda")          # 33792 nodes > 32768
    g = torch.zeros_like(f)
    assert Bd.step_noalloc(f, g, None, case["p"]) == Bd.LBM_ERR_SIZE
    h = torch.zeros(27, 4, 4, 4, device="cuda")
    assert Bd.step_noalloc(h, h, None, case["p"]) == Bd.LBM_ERR_ARG


def test_noalloc_reports_a_non_finite_state():
    """The step's status word is read back: a NaN population in f_in gives
    LBM_ERR_NONFINITE, and the next clean call returns LBM_OK again."""
    case = build("droplet_tiles")
    p = case["p"]
    p.shift_mode = Bd.SHIFT_CONST
    p.rho_shift = 0.0
    f0 = oracle_init(case).float().contiguous().cuda()
    bad = f0.clone()
    bad[:, 3, 4, 5] = float("nan")
    out = torch.empty_like(f0)
    assert Bd.step_noalloc(bad, out, None, p) == Bd.LBM_ERR_NONFINITE
    assert Bd.step_noalloc(f0, out, None, p) == Bd.LBM_OK
