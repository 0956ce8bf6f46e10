"""FP64 discrete adjoint of the oracle time step (CPU).

Test infrastructure only (see ``oracle/__init__.py``).

The paper has no adjoint; the gradient of a scalar objective J(f(T)) after T
steps of the step of ``oracle.step`` is defined here as the exact
reverse-mode derivative of that discrete map (autograd of the FP64 code).  It
is pinned by central finite differences in tests/test_oracle_adjoint.py.

Objectives (on the final state):
  kinetic energy     1/2 sum_fluid rho |u|^2
  centroid_x         sum x (rho - rho_v) / sum (rho - rho_v) over fluid nodes
  contact_radius     sqrt(A / pi), A = sum over the first fluid layer above
                     the wall plane z = wall_z of (rho - rho_v)/(rho_l - rho_v)
Parameters differentiated: kappa, the 11 relaxation rates, the wetting value
(phi or delta_rho) and the initial density field rho0.
"""
from __future__ import annotations

import copy
import math

import torch

from . import step as S

DT = torch.float64


def objective(name: str, f: torch.Tensor, solid: torch.Tensor, p: S.Params, wall_z: int = 0) -> torch.Tensor:
    m = S.macroscopic(f, solid, p)
    fluid = ~solid
    rho = m["rho"]
    if name == "energy":
        return m["energy"]
    if name == "centroid_x":
        nz, ny, nx = rho.shape
        x = torch.arange(nx, dtype=DT).view(1, 1, nx).expand(nz, ny, nx)
        wgt = torch.where(fluid, rho - p.rho_v, torch.zeros_like(rho))
        return (x * wgt).sum() / wgt.sum()
    if name == "contact_radius":
        layer = torch.where(fluid[wall_z + 1], rho[wall_z + 1] - p.rho_v, torch.zeros_like(rho[0]))
        area = layer.sum() / (p.rho_l - p.rho_v)
        return torch.sqrt(area / math.pi)
    raise ValueError(name)


def forward_objective(rho0: torch.Tensor, u0, solid: torch.Tensor, p: S.Params, nsteps: int,
                      name: str, wall_z: int = 0) -> torch.Tensor:
    f = S.initial_populations(rho0, u0, solid, p)
    f = S.run(f, solid, p, nsteps)
    return objective(name, f, solid, p, wall_z)


def gradients(rho0, u0, solid, p: S.Params, nsteps: int, name: str, wall_z: int = 0) -> dict:
    """dJ/d{kappa, omega[0..10], wetting_value, rho0} by reverse mode."""
    q = copy.copy(p)
    kappa = torch.tensor(float(p.kappa), dtype=DT, requires_grad=True)
    omega = torch.tensor([float(v) for v in p.omega], dtype=DT, requires_grad=True)
    wv = torch.tensor(float(p.wetting_value), dtype=DT, requires_grad=True)
    r0 = rho0.detach().clone().requires_grad_(True)
    q.kappa, q.omega, q.wetting_value = kappa, omega, wv
    J = forward_objective(r0, u0, solid, q, nsteps, name, wall_z)
    gk, go, gw, gr = torch.autograd.grad(J, (kappa, omega, wv, r0), allow_unused=True)
    z = lambda g, like: torch.zeros_like(like) if g is None else g
    return dict(J=float(J.detach()), kappa=float(z(gk, kappa)), omega=z(go, omega).detach(),
                wetting_value=float(z(gw, wv)), rho0=z(gr, r0).detach())


def step_vjp(f: torch.Tensor, solid: torch.Tensor, p: S.Params, lam_next: torch.Tensor):
    """lambda_t = (d f(t+1) / d f(t))^T lambda_{t+1} for one step, plus the
    parameter cotangents (kappa, omega, wetting value) of the same step."""
    q = copy.copy(p)
    kappa = torch.tensor(float(p.kappa), dtype=DT, requires_grad=True)
    omega = torch.tensor([float(v) for v in p.omega], dtype=DT, requires_grad=True)
    wv = torch.tensor(float(p.wetting_value), dtype=DT, requires_grad=True)
    q.kappa, q.omega, q.wetting_value = kappa, omega, wv
    ft = f.detach().clone().requires_grad_(True)
    out = S.step(ft, solid, q)
    g = torch.autograd.grad(out, (ft, kappa, omega, wv), grad_outputs=lam_next, allow_unused=True)
    z = lambda v, like: torch.zeros_like(like) if v is None else v.detach()
    return z(g[0], ft), z(g[1], kappa), z(g[2], omega), z(g[3], wv)
