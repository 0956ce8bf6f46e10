"""FP16 population storage modelled in the FP64 oracle (test infrastructure):
after every step each population is replaced by round16(f - s) + s, with s
the rest-equilibrium shift the library stores populations with,
w_q rho_b + c_b E_q keyed by the node's rho_b = rho and c_b = p_m - rho/3 of
the state it was collided from (E_q of Eq. 16 at u = 0: -19/9, 2/9, 1/18,
1/72 by speed class).  The distance of that run from the exact FP64 run is
the error the storage rounding alone produces: the floor an FP16-storage
implementation cannot go below, whatever its arithmetic.
"""
from __future__ import annotations

import functools

import torch

from oracle import lattice as L
from oracle import step as S

from _cases import build, oracle_init, oracle_params


def _shift_classes():
    c = L.velocities()
    e = {0: -19.0 / 9.0, 1: 2.0 / 9.0, 2: 1.0 / 18.0, 3: 1.0 / 72.0}
    E = torch.tensor([e[int((c[q] ** 2).sum())] for q in range(27)], dtype=torch.float64)
    return L.weights().double().view(27, 1, 1, 1), E.view(27, 1, 1, 1)


def rounded_run(f0: torch.Tensor, solid: torch.Tensor, op: S.Params, nsteps: int) -> torch.Tensor:
    """The oracle's nsteps steps from f0 with every stored population rounded
    as FP16 storage rounds it (the initial state included)."""
    w, E = _shift_classes()

    def basis(f):
        m = S.macroscopic(f, solid, op)
        return m["rho"], (1.0 + m["mu"] - m["rho"]) / 3.0

    def stored(f, rb, cb):
        s = w * rb + cb * E
        return torch.where(solid, f, (f - s).half().double() + s)

    fr = stored(f0, *basis(f0))
    for _ in range(nsteps):
        b = basis(fr)
        fr = stored(S.step(fr, solid, op), *b)
    return fr


@functools.lru_cache(maxsize=None)
def storage_rounding_error(name: str, nsteps: int) -> float:
    """Max relative fluid density difference between the FP64 oracle with
    FP16 storage rounding and the exact FP64 oracle after nsteps steps."""
    case = build(name)
    solid = torch.from_numpy(case["mask"].astype(bool))
    op = oracle_params(case["p"])
    f0 = oracle_init(case)
    fr = rounded_run(f0, solid, op, nsteps)
    fx = f0
    for _ in range(nsteps):
        fx = S.step(fx, solid, op)
    r, x = S.macroscopic(fr, solid, op)["rho"], S.macroscopic(fx, solid, op)["rho"]
    fl = ~solid
    return float(((r - x).abs() / x.abs().clamp_min(1e-3))[fl].max())
