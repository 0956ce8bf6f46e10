"""lbm_step(n) replays captured CUDA graphs of 16 steps; the populations must
be bitwise those of n single steps, from either buffer, with walls, after a
parameter change (which discards the graphs) and for FP16 storage.  The
adjoint segment sweep is captured the same way and must match its direct
launches bit for bit."""
import pytest
import torch

from paper_2504_03819_gb300 import Domain
from paper_2504_03819_gb300 import binding as Bd
from paper_2504_03819_gb300.adjoint import rollout_gradient

from _cases import build

pytestmark = pytest.mark.gpu


def start(case, storage="f32"):
    nx, ny, nz = case["n"]
    d = Domain(nx, ny, nz, storage, solid_mask=case["mask"] if case["mask"].any() else None)
    d.set_params(case["p"])
    d.set_state(torch.from_numpy(case["rho0"]).float(), torch.from_numpy(case["u0"]).float())
    return d


@pytest.mark.parametrize("name,storage", [("droplet_tiles", "f32"), ("wall_tiles", "f32"), ("droplet_odd", "f32"),
                                          ("droplet_tiles", "f16")])
def test_graph_steps_match_single_steps(name, storage):
    case = build(name)
    a, b = start(case, storage), start(case, storage)
    a.step(1)                      # odd starting buffer for the graphs
    a.step(35)                     # two graphs + three single steps
    for _ in range(36):
        b.step(1)
    assert a.sync_status() == b.sync_status() == 0
    assert torch.equal(a.get_populations(), b.get_populations())
    # a parameter change discards the captured graphs
    p = case["p"]
    om = list(p.omega)
    om[1] = 1.3
    p.omega = om
    a.set_params(p)
    b.set_params(p)
    a.step(32)
    for _ in range(32):
        b.step(1)
    assert torch.equal(a.get_populations(), b.get_populations())
    assert a.launch_count() == b.launch_count()


@pytest.mark.parametrize("name,storage", [("wall_tiles", "f32"), ("droplet_tiles", "f16")])
def test_graph_adjoint_segments_match_direct_launches(name, storage):
    """lbm_adjoint_segment replays one captured graph per (segment length,
    buffers): a 10-step rollout with checkpoints every 4 steps (segments of
    4, 4 and 2) gives bitwise the gradient of the same sweep launched kernel
    by kernel (profiling on disables the graphs), twice in a row (the second
    sweep replays the cached graphs)."""
    case = build(name)
    rho0 = torch.from_numpy(case["rho0"]).float()
    u0 = torch.from_numpy(case["u0"]).float()
    out = []
    for prof in (True, False, False):
        d = start(case, storage)
        d.profile(prof)
        J, grad, g_rho0 = rollout_gradient(d, rho0, u0, 10, 4, Bd.OBJ_ENERGY)
        assert d.sync_status() == 0
        out.append((J, grad.clone(), g_rho0.clone()))
        if not prof:
            J2, grad2, g2 = rollout_gradient(d, rho0, u0, 10, 4, Bd.OBJ_ENERGY)
            assert J2 == J and torch.equal(grad2, grad) and torch.equal(g2, g_rho0)
        d.close()
    for o in out[1:]:
        assert o[0] == out[0][0]
        assert torch.equal(o[1], out[0][1])
        assert torch.equal(o[2], out[0][2])
