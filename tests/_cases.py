"""Shared workload definitions for the GPU parity tests.

Each case gives the domain, solid mask, model parameters and seeded initial
fields from paper_2504_03819_gb300.inputs, plus converters that hand the same
(FP32-representable) inputs to the CUDA library and to the FP64 oracle.
"""
from __future__ import annotations

import numpy as np
import torch

from oracle import step as S
from oracle import thermo as T
from paper_2504_03819_gb300 import inputs as I
from paper_2504_03819_gb300.binding import Params

A49, A392, B = 9.0 / 49.0, 9.0 / 392.0, 2.0 / 21.0


def vdw(a=A49, t=0.85, kappa=0.01, **kw) -> Params:
    """Parameters at T = t T_c with the coexistence densities of the oracle's
    Maxwell construction (so no input of the oracle comes from the library)."""
    eos = T.at_reduced_temperature(a, B, 1.0, t)
    rl, rv = T.maxwell(eos)
    return Params(a=a, b=B, R=1.0, T=eos.T, kappa=kappa, rho_l=rl, rho_v=rv, **kw)


def oracle_params(p: Params) -> S.Params:
    return S.Params(a=p.a, b=p.b, R=p.R, T=p.T, kappa=p.kappa, omega=list(p.omega), nu=p.nu,
                    q4=bool(p.q4_correction), wetting_mode=p.wetting_mode, wetting_value=p.wetting_value,
                    rho_l=p.rho_l, rho_v=p.rho_v)


def f32(x) -> np.ndarray:
    """Round to FP32 (what the device receives) and return as float64."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


CASES = {
    # periodic droplet, ragged sizes (not multiples of 32 / 256)
    "droplet_periodic": dict(n=(13, 10, 14), walls=(), radius=4.0, u=(0.02, -0.01, 0.015), p={}),
    # walls at z = 0 and z = nz-1, hydrophilic wetting, sessile droplet
    "wall_phi": dict(n=(11, 9, 12), walls=(0, 11), radius=4.0, sessile=True, u=(0.0, 0.0, 0.0),
                     p=dict(wetting_mode=1, wetting_value=1.3)),
    # hydrophobic wetting, viscosity mode, shear rate != 1
    "wall_delta_nu": dict(n=(10, 12, 11), walls=(0, 10), radius=4.0, sessile=True, u=(0.01, 0.0, 0.0),
                          p=dict(wetting_mode=2, wetting_value=0.9, nu=0.15)),
    # neutral wetting, general rates, no fourth-order correction
    "wall_neutral_rates_noq4": dict(n=(9, 9, 10), walls=(0,), radius=3.5, sessile=True, u=(0.0, 0.01, 0.0),
                                    p=dict(q4_correction=0,
                                           omega=[1.0, 1.6, 1.2, 0.9, 1.1, 1.3, 0.8, 1.4, 1.05, 0.95, 1.5])),
    # odd node count (FP16 moments take the one-node-per-thread path), one
    # partial tile, uniform flow along a diagonal
    "droplet_odd": dict(n=(9, 9, 9), walls=(), radius=3.0, u=(0.01, 0.01, 0.01), p={}),
    # rows of 16-byte multiples (tensor-copy staging of the population
    # tiles): two tiles in x and y with ragged tails, periodic (FP16 too)
    "droplet_tiles": dict(n=(40, 12, 10), walls=(), radius=4.0, u=(0.02, 0.01, -0.01), p={}),
    # the same staging with walls and hydrophilic wetting (FP32 rows only)
    "wall_tiles": dict(n=(36, 10, 9), walls=(0, 8), radius=3.5, sessile=True, u=(0.01, 0.0, 0.0),
                       p=dict(wetting_mode=1, wetting_value=1.2)),
    # general rates on the tensor-copy path (rows of 16-byte multiples in
    # FP32 and FP16): two tiles in x with a ragged tail, three in y
    "tiles_rates": dict(n=(40, 10, 9), walls=(), radius=3.5, u=(0.02, -0.01, 0.01),
                        p=dict(omega=[1.0, 1.6, 1.2, 0.9, 1.1, 1.3, 0.8, 1.4, 1.05, 0.95, 1.5])),
    # the same with populations stored minus the constant shift w_i rho_0
    "tiles_rates_const": dict(n=(40, 10, 9), walls=(), radius=3.5, u=(0.02, -0.01, 0.01), const_shift=True,
                              p=dict(omega=[1.0, 1.6, 1.2, 0.9, 1.1, 1.3, 0.8, 1.4, 1.05, 0.95, 1.5])),
    # walls, hydrophobic (delta-rho) wetting and general rates on the
    # tensor-copy path in FP32 and FP16 (40-wide rows)
    "wall_tiles_delta": dict(n=(40, 8, 10), walls=(0, 9), radius=3.5, sessile=True, u=(0.01, 0.0, 0.0),
                             p=dict(wetting_mode=2, wetting_value=0.7,
                                    omega=[1.0, 1.3, 1.1, 0.95, 1.05, 1.2, 0.9, 1.1, 1.0, 0.9, 1.2])),
    # paper EOS, 0.7 T_c, kappa = 0.02, degenerate 1 x 1 x n flat interface
    "flat_paper_1d": dict(n=(1, 1, 48), walls=(), slab=24, u=(0.0, 0.0, 0.0),
                          p=dict(a=A392, t=0.7, kappa=0.02, nu=0.15)),
}


def build(name: str):
    c = CASES[name]
    nx, ny, nz = c["n"]
    pk = dict(c["p"])
    a, t, kappa = pk.pop("a", A49), pk.pop("t", 0.85), pk.pop("kappa", 0.01)
    p = vdw(a, t, kappa, **pk)
    mask = I.wall_mask(nx, ny, nz, planes=c["walls"])
    if "slab" in c:
        rho0 = I.slab(nx, ny, nz, c["slab"], p.rho_l, p.rho_v)
    elif c.get("sessile"):
        rho0 = I.sessile_droplet(nx, ny, nz, c["radius"], p.rho_l, p.rho_v, wall_z=c["walls"][0] + 0.5)
    else:
        rho0 = I.droplet(nx, ny, nz, c["radius"], p.rho_l, p.rho_v)
    u0 = I.uniform_velocity(nx, ny, nz, c["u"])
    if c.get("const_shift"):
        p.shift_mode = 0
        p.rho_shift = 2 * p.rho_l * p.rho_v / (p.rho_l + p.rho_v)
    return dict(n=(nx, ny, nz), p=p, mask=mask, rho0=f32(rho0), u0=f32(u0))


def oracle_init(case) -> torch.Tensor:
    solid = torch.from_numpy(case["mask"].astype(bool))
    return S.initial_populations(torch.from_numpy(case["rho0"]), torch.from_numpy(case["u0"]), solid,
                                 oracle_params(case["p"]))


def perturbed(case, f: torch.Tensor, seed: int, scale: float = 0.002) -> torch.Tensor:
    """f plus a seeded non-equilibrium perturbation, rounded to FP32, zero on
    solid nodes."""
    nx, ny, nz = case["n"]
    pert = torch.from_numpy(I.random_populations(nx, ny, nz, seed, scale=scale))
    solid = torch.from_numpy(case["mask"].astype(bool))
    g = torch.where(solid, torch.zeros_like(f), f + pert * f.abs().clamp_min(0.01))
    return torch.from_numpy(g.numpy().astype(np.float32).astype(np.float64))
