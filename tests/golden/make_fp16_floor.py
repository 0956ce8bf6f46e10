"""Write fp16_floor.json: for each listed parity case, the relative density
error that FP16 population storage alone produces after 50 steps, measured
as the distance between the FP64 oracle with the storage rounding modelled
(tests/_fp16.py) and the exact FP64 oracle; and the same after 1000 steps for
the listed workload copies of long_cases.py, against the exact oracle's
fields that make_long_parity.py stored (on their z-planes).  Calls only the
oracle, the input generator and that rounding model.

    python tests/golden/make_fp16_floor.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

import numpy as np  # noqa: E402
import torch  # noqa: E402

from _fp16 import rounded_run, storage_rounding_error  # noqa: E402
from make_long_parity import setup  # noqa: E402
from oracle import step as S  # noqa: E402

CASES = ["tiles_rates"]
STEPS = 50
LONG = ["moving64"]


def long_floor(name: str) -> float:
    """Max relative fluid density difference, on the stored z-planes, between
    the oracle with FP16 storage rounding and the exact oracle after the
    workload copy's 1000 steps."""
    c, p, rho0, u0, mask = setup(name)
    solid = torch.from_numpy(mask.astype(bool))
    ref = np.load(os.path.join(HERE, f"long_{name}.npz"))
    f0 = S.initial_populations(torch.from_numpy(rho0), torch.from_numpy(u0), solid, p)
    rho = S.macroscopic(rounded_run(f0, solid, p, int(ref["steps"])), solid, p)["rho"].numpy()
    planes = ref["planes"] if "planes" in ref.files else np.arange(mask.shape[0])
    fl = ~mask.astype(bool)[planes]
    x = ref["rho"].astype(np.float64)[fl]
    return float((np.abs(rho[planes][fl] - x) / np.maximum(np.abs(x), 1e-3)).max())


if __name__ == "__main__":
    if os.environ.get("ORACLE_THREADS"):
        torch.set_num_threads(int(os.environ["ORACLE_THREADS"]))
    path = os.path.join(HERE, "fp16_floor.json")
    out = json.load(open(path)) if os.path.exists(path) else {}
    out["_about"] = __doc__.split("\n\n")[0].replace("\n", " ")
    out["steps"] = STEPS
    for name in sys.argv[1:] or CASES + LONG:
        if name in LONG:
            out.setdefault("long", {"steps": 1000})[name] = long_floor(name)
            print(name, out["long"][name], flush=True)
        else:
            out[name] = storage_rounding_error(name, STEPS)
            print(name, out[name], flush=True)
    json.dump(out, open(path, "w"), indent=1)
