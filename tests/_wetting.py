"""Measurements on droplet density fields (host-side analysis for the tests;
no method arithmetic): the contact angle of a drop on a wall from a sphere
fit to its mid-density surface, and the equimolar radius of a free drop.

Contact angle (the paper does not say how it measures it): the points where
rho crosses (rho_l + rho_v)/2 between neighbouring fluid nodes along x, y
and z, linearly interpolated, excluding the first fluid layer above the
wall; an algebraic least-squares sphere |p - c|^2 = R^2 through them; the
wall plane z = z_wall (halfway between the solid layer and the first fluid
layer); the angle inside the liquid from the cap geometry,
cos(theta) = (z_wall - c_z) / R.  A second measure (cap_angle) takes the
drop's height and base radius, tan(theta/2) = h / r_base; on a true
spherical cap the two agree to a few degrees, so a larger gap between them
shows a drop whose shape near the wall departs from a cap.
"""
from __future__ import annotations

import math

import numpy as np


def crossing_points(rho: np.ndarray, mid: float, solid: np.ndarray | None = None, zmin: float = 2.0) -> np.ndarray:
    """(x, y, z) points where rho (nz, ny, nx) crosses `mid` between
    neighbouring nodes along each axis (no wrap), both nodes fluid, z >= zmin."""
    pts = []
    fluid = np.ones_like(rho, dtype=bool) if solid is None else ~solid.astype(bool)
    nz, ny, nx = rho.shape
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    for axis in range(3):
        a = [slice(None)] * 3
        b = [slice(None)] * 3
        a[axis] = slice(0, -1)
        b[axis] = slice(1, None)
        ra, rb = rho[tuple(a)], rho[tuple(b)]
        ok = fluid[tuple(a)] & fluid[tuple(b)] & ((ra - mid) * (rb - mid) < 0)
        t = (mid - ra[ok]) / (rb[ok] - ra[ok])
        coords = [c[tuple(a)][ok].astype(np.float64) for c in (x, y, z)]
        coords[2 - axis] = coords[2 - axis] + t
        pts.append(np.stack(coords, axis=1))
    P = np.concatenate(pts)
    return P[P[:, 2] >= zmin]


def sphere_fit(P: np.ndarray):
    """Centre (3,) and radius of the least-squares sphere through points P."""
    A = np.c_[2.0 * P, np.ones(len(P))]
    sol = np.linalg.lstsq(A, (P ** 2).sum(1), rcond=None)[0]
    c = sol[:3]
    return c, math.sqrt(sol[3] + float(c @ c))


def contact_angle(rho: np.ndarray, rho_l: float, rho_v: float, solid: np.ndarray | None = None,
                  z_wall: float = 0.5, zmin: float = 2.0) -> float:
    """Contact angle (degrees, inside the liquid) of a drop sitting on the
    wall plane z = z_wall."""
    P = crossing_points(rho, 0.5 * (rho_l + rho_v), solid, zmin)
    c, R = sphere_fit(P)
    return math.degrees(math.acos(max(-1.0, min(1.0, (z_wall - c[2]) / R))))


def cap_angle(rho: np.ndarray, rho_l: float, rho_v: float, z_wall: float = 0.5) -> float:
    """Contact angle (degrees) from the cap geometry tan(theta/2) = h / r_base:
    h is the height above the wall plane where the mid-density surface
    crosses the vertical line through the x-y centre of the domain (linear
    interpolation between nodes), r_base the radius of a disc with the
    liquid fraction (rho - rho_v)/(rho_l - rho_v), clipped to [0, 1], of the
    first fluid layer (z = 1) as its area."""
    nz, ny, nx = rho.shape
    mid = 0.5 * (rho_l + rho_v)
    col = rho[:, ny // 2, nx // 2]
    h = float("nan")
    for z in range(1, nz - 2):
        if col[z] >= mid > col[z + 1]:
            h = z + (col[z] - mid) / (col[z] - col[z + 1]) - z_wall
            break
    area = float(((rho[1] - rho_v) / (rho_l - rho_v)).clip(0.0, 1.0).sum())
    return math.degrees(2.0 * math.atan2(h, math.sqrt(area / math.pi)))


def equimolar_radius(rho: np.ndarray, rho_in: float, rho_out: float) -> float:
    """Radius of the sphere holding the drop's excess mass at density
    rho_in in vapour of density rho_out."""
    vol = float(((rho - rho_out) / (rho_in - rho_out)).sum())
    return (3.0 * vol / (4.0 * math.pi)) ** (1.0 / 3.0)
