"""Seeded synthetic inputs shaped like the paper's test cases (Sec. III).

This module holds no arithmetic of the lattice Boltzmann method itself: it only
builds initial density/velocity fields and solid masks from closed-form
profiles, as NumPy float64 arrays laid out (nz, ny, nx) / (3, nz, ny, nx).
Both the CUDA path and the CPU oracle take their inputs from here.

Profiles
  * tanh interface of width W (Eq. 34):
        rho = (rho_l + rho_v)/2 - (rho_l - rho_v)/2 tanh(2 (r0 - r) / W)
    with r0 the distance to the droplet centre (Eq. 35) for a droplet and the
    distance to the slab mid-plane for a flat slab.  W = 5 as in Sec. III B.
  * solid walls: whole z-planes of the solid mask.
"""
from __future__ import annotations

import numpy as np

W_INTERFACE = 5.0


def _grid(nx: int, ny: int, nz: int):
    z, y, x = np.meshgrid(np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
                          np.arange(nx, dtype=np.float64), indexing="ij")
    return x, y, z


def droplet(nx: int, ny: int, nz: int, radius: float, rho_l: float, rho_v: float,
            centre=None, width: float = W_INTERFACE) -> np.ndarray:
    """Liquid sphere of the given radius in vapour (Eqs. 34-35).

    centre defaults to the domain centre ((n-1)/2 on each axis).
    """
    if centre is None:
        centre = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
    x, y, z = _grid(nx, ny, nz)
    r0 = np.sqrt((x - centre[0]) ** 2 + (y - centre[1]) ** 2 + (z - centre[2]) ** 2)
    return 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * np.tanh(2.0 * (r0 - radius) / width)


def slab(nx: int, ny: int, nz: int, thickness: float, rho_l: float, rho_v: float,
         width: float = W_INTERFACE) -> np.ndarray:
    """Liquid slab of the given thickness centred in z, vapour elsewhere (flat
    interfaces normal to z, Sec. III A).  The slab occupies
    z in [nz/2 - thickness/2, nz/2 + thickness/2)."""
    x, y, z = _grid(nx, ny, nz)
    zc = nz / 2.0 - 0.5
    r0 = np.abs(z - zc)
    return 0.5 * (rho_l + rho_v) - 0.5 * (rho_l - rho_v) * np.tanh(2.0 * (r0 - thickness / 2.0) / width)


def wall_mask(nx: int, ny: int, nz: int, planes=(0,)) -> np.ndarray:
    """uint8 solid mask (1 = solid) with the given z-planes solid."""
    m = np.zeros((nz, ny, nx), dtype=np.uint8)
    for zp in planes:
        m[zp] = 1
    return m


def sessile_droplet(nx: int, ny: int, nz: int, radius: float, rho_l: float, rho_v: float,
                    wall_z: float = 0.5, width: float = W_INTERFACE) -> np.ndarray:
    """Sphere of the given radius centred on the wall plane z = wall_z at the
    x-y centre (a hemisphere above a wall at z = 0, Sec. III C)."""
    return droplet(nx, ny, nz, radius, rho_l, rho_v,
                   centre=((nx - 1) / 2.0, (ny - 1) / 2.0, wall_z), width=width)


def uniform_velocity(nx: int, ny: int, nz: int, u=(0.0, 0.0, 0.0)) -> np.ndarray:
    out = np.zeros((3, nz, ny, nx), dtype=np.float64)
    for a in range(3):
        out[a] = u[a]
    return out


def add_noise(rho: np.ndarray, sigma: float, seed: int = 12345) -> np.ndarray:
    """rho + N(0, sigma^2) drawn from numpy.random.default_rng(seed)."""
    rng = np.random.default_rng(seed)
    return rho + sigma * rng.standard_normal(rho.shape)


def random_populations(nx: int, ny: int, nz: int, seed: int, scale: float = 0.05,
                       base: np.ndarray | None = None, dtype=np.float64) -> np.ndarray:
    """Seeded random perturbation field of shape (27, nz, ny, nx), optionally
    added to a base population field (for non-equilibrium test states).
    dtype=np.float32 draws FP32 normals directly (full-size fields)."""
    rng = np.random.default_rng(seed)
    pert = rng.standard_normal((27, nz, ny, nx), dtype=dtype)
    pert *= dtype(scale) if dtype is np.float32 else scale
    return pert if base is None else base + pert
