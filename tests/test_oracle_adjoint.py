"""Pins for oracle/adjoint.py: the reverse-mode gradient of the FP64 step
against central finite differences of the same FP64 forward map, and the
adjoint identity <J v, w> = <v, J^T w> for one step.
"""
import copy

import numpy as np
import pytest
import torch

from oracle import adjoint as A
from oracle import step as S
from oracle import thermo as T
from paper_2504_03819_gb300 import inputs as I

DT = torch.float64
B = 2.0 / 21.0


def setup(mode=1, value=1.3, n=8):
    eos = T.at_reduced_temperature(9.0 / 49.0, B, 1.0, 0.85)
    rl, rv = T.maxwell(eos)
    p = S.Params(a=9.0 / 49.0, b=B, R=1.0, T=eos.T, kappa=0.01, omega=[1.0, 1.3] + [1.0] * 9,
                 wetting_mode=mode, wetting_value=value, rho_l=rl, rho_v=rv)
    solid = torch.tensor(I.wall_mask(n, n, n, planes=(0, n - 1)).astype(bool))
    rho0 = torch.tensor(I.add_noise(I.sessile_droplet(n, n, n, 3.0, rl, rv), 1e-3, seed=12345))
    return p, solid, rho0


def fd(fun, x0, h):
    return (fun(x0 + h) - fun(x0 - h)) / (2 * h)


@pytest.mark.parametrize("name", ["contact_radius", "energy"])
def test_parameter_gradients_match_central_differences(name):
    p, solid, rho0 = setup()
    nsteps = 3
    g = A.gradients(rho0, None, solid, p, nsteps, name)

    def J_with(**kw):
        q = copy.copy(p)
        for k, v in kw.items():
            setattr(q, k, v)
        return float(A.forward_objective(rho0, None, solid, q, nsteps, name))

    h = 1e-4
    gk = fd(lambda v: J_with(kappa=v), p.kappa, h * 0.01)
    assert g["kappa"] == pytest.approx(gk, rel=1e-5, abs=1e-9)
    gw = fd(lambda v: J_with(wetting_value=v), p.wetting_value, h)
    assert g["wetting_value"] == pytest.approx(gw, rel=1e-5, abs=1e-9)
    assert abs(gw) > 1e-8 or name == "energy"

    def om(v):
        o = list(p.omega)
        o[1] = v
        return J_with(omega=o)

    go1 = fd(om, p.omega[1], h)
    assert float(g["omega"][1]) == pytest.approx(go1, rel=1e-5, abs=1e-9)
    # omega_0 drops out of the step (k100* = F/2): its gradient is zero
    assert abs(float(g["omega"][0])) < 1e-12
    # initial density at three nodes near the contact line
    for (z, y, x) in [(1, 4, 6), (2, 3, 3), (1, 1, 4)]:
        def jr(v, z=z, y=y, x=x):
            r = rho0.clone()
            r[z, y, x] = v
            return float(A.forward_objective(r, None, solid, p, nsteps, name))
        gr = fd(jr, float(rho0[z, y, x]), h)
        assert float(g["rho0"][z, y, x]) == pytest.approx(gr, rel=1e-4, abs=1e-9)


def test_one_step_adjoint_identity():
    """<J v, w> = <v, J^T w> with J = d f(t+1)/d f(t) (JVP by central
    differences of the FP64 step, VJP by the adjoint)."""
    p, solid, rho0 = setup(mode=2, value=0.6, n=6)
    f = S.initial_populations(rho0, None, solid, p)
    g = torch.Generator().manual_seed(1)
    fluid = (~solid).to(DT)
    v = torch.randn(f.shape, generator=g, dtype=DT) * fluid
    w = torch.randn(f.shape, generator=g, dtype=DT) * fluid
    h = 1e-6
    jv = (S.step(f + h * v, solid, p) - S.step(f - h * v, solid, p)) / (2 * h)
    jtw, _, _, _ = A.step_vjp(f, solid, p, w)
    lhs = float((jv * w).sum())
    rhs = float((v * jtw).sum())
    assert lhs == pytest.approx(rhs, rel=1e-7)
