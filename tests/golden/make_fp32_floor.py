"""Write fp32_floor.json: for each parity case, how far the FP64 oracle
itself moves after 50 steps when every population is perturbed by FP32-sized
relative noise (6e-8, about 2^-24, drawn N(0, 1) from torch.Generator seeds
0, 1, 2) after every step: the max over the seeds of the max relative fluid
density departure from the clean run.  An FP32 implementation rounds at
least that much per step, so its 50-step error cannot be expected below
this floor.  Calls only the oracle and the input generator.

    python tests/golden/make_fp32_floor.py
"""
import json
import os
import sys

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

from oracle import step as S  # noqa: E402

from _cases import CASES, build, oracle_init, oracle_params  # noqa: E402

STEPS = 50
EPS = 6e-8
SEEDS = (0, 1, 2)


def floor(name: str) -> float:
    case = build(name)
    solid = torch.from_numpy(case["mask"].astype(bool))
    op = oracle_params(case["p"])
    f0 = oracle_init(case)
    ref = S.macroscopic(S.run(f0, solid, op, STEPS), solid, op)["rho"]
    fl = ~solid
    worst = 0.0
    for seed in SEEDS:
        g = torch.Generator().manual_seed(seed)
        f = f0.clone()
        for _ in range(STEPS):
            f = S.step(f, solid, op)
            f = f * (1 + EPS * torch.randn(f.shape, generator=g, dtype=torch.float64))
        r = S.macroscopic(f, solid, op)["rho"]
        worst = max(worst, float(((r - ref).abs() / ref.abs())[fl].max()))
    return worst


if __name__ == "__main__":
    out = {"_about": __doc__.split("\n\n")[0].replace("\n", " "), "steps": STEPS, "eps": EPS}
    for name in CASES:
        out[name] = floor(name)
        print(name, out[name], flush=True)
    json.dump(out, open(os.path.join(HERE, "fp32_floor.json"), "w"), indent=1)
