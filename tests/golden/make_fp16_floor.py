"""Write fp16_floor.json: for each listed parity case, the relative density
error that FP16 population storage alone produces after 50 steps, measured
as the distance between the FP64 oracle with the storage rounding modelled
(tests/_fp16.py) and the exact FP64 oracle.  Calls only the oracle, the
input generator and that rounding model.

    python tests/golden/make_fp16_floor.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

from _fp16 import storage_rounding_error  # noqa: E402

CASES = ["tiles_rates"]
STEPS = 50

if __name__ == "__main__":
    out = {"_about": __doc__.split("\n\n")[0].replace("\n", " "), "steps": STEPS}
    for name in CASES:
        out[name] = storage_rounding_error(name, STEPS)
        print(name, out[name], flush=True)
    json.dump(out, open(os.path.join(HERE, "fp16_floor.json"), "w"), indent=1)
