"""Gradients of an objective of the state after T steps, by the discrete
adjoint of the CUDA step with checkpointing.

The forward pass keeps the raw state every K steps; the backward pass walks
the segments from the last to the first, recomputes the K states of a
segment from its checkpoint, and runs lbm_adjoint_step backwards through
them; lbm_adjoint_init finally carries the adjoint to the initial density.
Every step of both passes runs in the library's kernels; this module only
orders the calls and holds the checkpoints (device tensors).
"""
from __future__ import annotations

import torch

from .binding import NGRAD, Domain, Params


def _set_theta(p: Params, theta) -> Params:
    q = Params(**{k: getattr(p, k) for k in p.__dataclass_fields__})
    th = [float(v) for v in theta]
    q.kappa = th[0]
    q.omega = th[1:12]
    q.wetting_value = th[12]
    return q


def theta_of(p: Params) -> torch.Tensor:
    """[kappa, omega_0..omega_10, wetting_value] as float64."""
    return torch.tensor([p.kappa] + list(p.omega) + [p.wetting_value], dtype=torch.float64)


def forward_checkpoints(dom: Domain, rho0, u0, nsteps: int, K: int) -> dict:
    dom.set_state(rho0, u0)
    ckpts = {0: dom.get_state().clone()}
    s = 0
    while s < nsteps:
        k = min(K, nsteps - s)
        dom.step(k)
        s += k
        if s < nsteps:
            ckpts[s] = dom.get_state(sync=False).clone()
    return ckpts


def backward_from(dom: Domain, ckpts: dict, nsteps: int, lam, grad, rho0, u0):
    """Adjoint sweep from dJ/df(T) = lam back to dJ/drho0: one
    lbm_adjoint_segment per checkpoint segment, last to first."""
    seg = max(b - a for a, b in zip(sorted(ckpts), sorted(ckpts)[1:] + [nsteps]))
    pool = torch.empty(seg * dom.adjoint_pool_bytes(), dtype=torch.uint8, device=dom.device)
    lam_a, lam_b = lam.clone(), torch.empty_like(lam)
    t_end = nsteps
    for s0 in sorted(ckpts, reverse=True):
        dom.adjoint_segment(ckpts[s0], t_end - s0, pool, lam_a, lam_b, grad)
        t_end = s0
    return dom.adjoint_init(rho0, u0, lam_a, grad)


def rollout_gradient(dom: Domain, rho0, u0, nsteps: int, K: int, objective: int, wall_z: int = 0):
    """J(f(T)) and its gradients: (J, dJ/dtheta (NGRAD float64), dJ/drho0)."""
    ckpts = forward_checkpoints(dom, rho0, u0, nsteps, K)
    grad = torch.zeros(NGRAD, dtype=torch.float64, device=dom.device)
    J, lam = dom.objective(objective, wall_z, grad)
    g_rho0 = backward_from(dom, ckpts, nsteps, lam, grad, rho0, u0)
    return float(J[0]), grad, g_rho0


class LBMRollout(torch.autograd.Function):
    """J = objective(f(T)) as a differentiable function of rho0 and theta =
    [kappa, omega_0..omega_10, wetting_value] (float64, CPU or CUDA).

    forward(rho0, theta, dom, params, u0, nsteps, K, objective, wall_z)
    """

    @staticmethod
    def forward(ctx, rho0, theta, dom, params, u0, nsteps, K, objective, wall_z):
        dom.set_params(_set_theta(params, theta.detach().cpu()))
        r0 = rho0.detach().to(device=dom.device, dtype=torch.float32).contiguous()
        ckpts = forward_checkpoints(dom, r0, u0, nsteps, K)
        g_direct = torch.zeros(NGRAD, dtype=torch.float64, device=dom.device)
        J, lam = dom.objective(objective, wall_z, g_direct)
        ctx.dom, ctx.ckpts, ctx.lam, ctx.r0, ctx.u0, ctx.nsteps = dom, ckpts, lam, r0, u0, nsteps
        ctx.g_direct = g_direct
        ctx.theta_device, ctx.rho0_dtype, ctx.rho0_device = theta.device, rho0.dtype, rho0.device
        return J[0].to(theta.device)

    @staticmethod
    def backward(ctx, gJ):
        grad = ctx.g_direct.clone()
        g_rho0 = backward_from(ctx.dom, ctx.ckpts, ctx.nsteps, ctx.lam, grad, ctx.r0, ctx.u0)
        gJ = gJ.to(torch.float64)
        g_theta = (grad * gJ.to(grad.device)).to(ctx.theta_device)
        g_r = (g_rho0.to(torch.float64) * gJ.to(g_rho0.device)).to(device=ctx.rho0_device, dtype=ctx.rho0_dtype)
        return g_r, g_theta, None, None, None, None, None, None, None
