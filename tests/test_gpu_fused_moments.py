"""The fused step also produces the next state's moments (rho, j and mu0 of
Eq. 11 and Eq. 32): every block of a thread-block cluster sums the
populations of the planes the cluster has finished pushing, and an edge pass
completes the first and last rows of each cluster and the first and last
planes of each block's z range.  These moments must be the bits a fresh
moments pass computes from the same state, node for node, or the
trajectories drift apart.

Each test runs a trajectory whose steps use the fused kernel's moments and
the same trajectory with the moments recomputed from the state before every
step (lbm_set_raw_state of the state just read marks them stale), and
compares the final raw states bit for bit.  The domains cover a cluster that
spans the y range (no edge rows), clusters with edge rows, z ranges with
edge planes, a z range that is the whole domain (its end planes wrap onto
each other), walls, both shift modes and FP16 storage; the full-size
domains are the bench's launch configuration.
"""
import numpy as np
import pytest
import torch

from paper_2504_03819_gb300 import Domain
from paper_2504_03819_gb300 import inputs as I

from _cases import build, vdw

pytestmark = pytest.mark.gpu


def trajectories(make, nsteps):
    """Final raw states of `nsteps` steps with the fused moments (graphs and
    single steps) and with a fresh moments pass before every step."""
    a = make()
    a.step(nsteps)
    assert a.sync_status() == 0
    fused = a.get_state().clone()
    a.profile(True)
    a.step(3)
    counts = {k: v[1] for k, v in a.profile_read().items()}
    a.profile(False)
    a.close()
    b = make()
    for _ in range(nsteps):
        b.set_raw_state(b.get_state().clone())
        b.step(1)
    assert b.sync_status() == 0
    fresh = b.get_state().clone()
    b.close()
    return fused, fresh, counts


def from_case(name, storage, fused=True):
    case = build(name)

    def make():
        nx, ny, nz = case["n"]
        d = Domain(nx, ny, nz, storage, solid_mask=case["mask"] if case["mask"].any() else None)
        d.fuse_moments(fused)
        d.set_params(case["p"])
        d.set_state(torch.from_numpy(case["rho0"]).float(), torch.from_numpy(case["u0"]).float())
        return d
    return make


def droplet(n, storage, radius, u=(0.03, -0.02, 0.01), omega1=1.0, walls=(), fused=True):
    nx, ny, nz = n
    om = [1.0] * 11
    om[1] = omega1
    kw = dict(wetting_mode=1, wetting_value=1.2) if walls else {}
    p = vdw(omega=om, **kw)
    mask = I.wall_mask(nx, ny, nz, planes=walls) if walls else None
    if walls:
        rho0 = I.sessile_droplet(nx, ny, nz, radius, p.rho_l, p.rho_v, wall_z=walls[0] + 0.5, width=2.0)
        u0 = I.uniform_velocity(nx, ny, nz)
    else:
        rho0 = I.droplet(nx, ny, nz, radius, p.rho_l, p.rho_v, width=2.0)
        u0 = I.uniform_velocity(nx, ny, nz, u)

    def make():
        d = Domain(nx, ny, nz, storage, solid_mask=mask)
        d.fuse_moments(fused)
        d.set_params(p)
        d.set_state(torch.from_numpy(rho0.astype(np.float32)), torch.from_numpy(u0.astype(np.float32)))
        return d
    return make


@pytest.mark.parametrize("name,storage", [
    ("droplet_tiles", "f32"),       # cluster spans y; z ranges of 4 planes with edge planes
    ("droplet_tiles", "f16"),
    ("wall_tiles", "f32"),          # walls, a one-plane last z range
    ("wall_tiles_delta", "f16"),    # walls, delta-rho wetting, general rates, FP16
    ("tiles_rates_const", "f32"),   # constant shift, general rates
])
def test_fused_moments_equal_a_fresh_moments_pass(name, storage):
    fused, fresh, counts = trajectories(from_case(name, storage), 20)
    assert torch.equal(fused, fresh)
    # the steps took the fused path: no separate moments pass after the first
    assert counts["collide"] == 3 and counts["moments"] == 0 and counts["moments_edge"] == 3


@pytest.mark.parametrize("n,storage", [
    ((64, 64, 16), "f32"),   # clusters of 2 x 8 blocks: edge rows every 32 rows; edge planes
    ((64, 64, 16), "f16"),
    ((32, 16, 4), "f32"),    # one z range covers the domain: its end planes wrap onto each other
])
def test_fused_moments_edge_rows_and_wrapping_z(n, storage):
    fused, fresh, _ = trajectories(droplet(n, storage, radius=min(n) / 3.0 + 1.0), 18)
    assert torch.equal(fused, fresh)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_fused_moments_full_size_moving_droplet(storage):
    """The bench's workload and launch shape: 256^3, R = 32, omega_1 = 1.6."""
    fused, fresh, counts = trajectories(droplet((256, 256, 256), storage, 32.0, u=(0.05, 0.02, 0.0), omega1=1.6),
                                        16)
    assert torch.equal(fused, fresh)
    assert counts["moments"] == 0


def test_fused_moments_full_size_wall():
    fused, fresh, _ = trajectories(droplet((256, 256, 128), "f32", 40.0, walls=(0, 127)), 16)
    assert torch.equal(fused, fresh)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_steps_are_bitwise_reproducible(storage):
    """Three runs of the same 16 steps on 128^3 (several hundred blocks per
    wave, the tensor-copy path) give the same raw state bit for bit.  A
    missing proxy fence between the tile buffer's ordinary reads and the next
    tensor copy into it once changed a few nodes per step at random."""
    make = droplet((128, 128, 128), storage, 16.0, u=(0.05, 0.02, 0.0), omega1=1.6, fused=False)
    states = []
    for _ in range(3):
        d = make()
        d.step(16)
        assert d.sync_status() == 0
        states.append(d.get_state().clone())
        d.close()
    assert torch.equal(states[0], states[1]) and torch.equal(states[0], states[2])
