"""Write the FP64 oracle's state after 1000 steps of each scaled workload copy
in long_cases.py to long_<name>.npz (density and velocity fields rounded to
FP32 -- their rounding, 6e-8 relative, is far below the tolerances they are
compared at -- and the FP64 fluid mass; the 64-node copies keep the fields on
the z-planes their case lists).

Calls only oracle/ and the seeded input generator; the initial fields are
rounded to FP32 first, as the CUDA library receives them.

    python tests/golden/make_long_parity.py [name ...]
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402
import torch  # noqa: E402

from long_cases import LONG_CASES, STEPS, eos_of  # noqa: E402
from oracle import step as S  # noqa: E402
from oracle import thermo as T  # noqa: E402
from paper_2504_03819_gb300 import inputs as I  # noqa: E402


def inputs(c, rl, rv):
    nx, ny, nz = c["n"]
    if c["walls"]:
        rho0 = I.sessile_droplet(nx, ny, nz, c["radius"], rl, rv, wall_z=c["walls"][0] + 0.5, width=c["width"])
    else:
        rho0 = I.droplet(nx, ny, nz, c["radius"], rl, rv, width=c["width"])
    u0 = I.uniform_velocity(nx, ny, nz, c["u"])
    mask = I.wall_mask(nx, ny, nz, planes=c["walls"])
    f32 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)  # noqa: E731
    return f32(rho0), f32(u0), mask


def setup(name):
    """Oracle parameters, FP32-representable initial fields and the solid
    mask of a workload copy."""
    c = LONG_CASES[name]
    EOS = eos_of(c)
    eos = T.at_reduced_temperature(EOS["a"], EOS["b"], EOS["R"], EOS["t_over_tc"])
    rl, rv = T.maxwell(eos)
    om = [1.0] * 11
    om[1] = c["omega1"]
    p = S.Params(a=EOS["a"], b=EOS["b"], R=EOS["R"], T=eos.T, kappa=EOS["kappa"], omega=om,
                 wetting_mode=c["wetting_mode"], wetting_value=c["wetting_value"], rho_l=rl, rho_v=rv)
    rho0, u0, mask = inputs(c, rl, rv)
    return c, p, rho0, u0, mask


def run(name):
    c, p, rho0, u0, mask = setup(name)
    solid = torch.from_numpy(mask.astype(bool))
    t0 = time.time()
    f = S.initial_populations(torch.from_numpy(rho0), torch.from_numpy(u0), solid, p)
    f = S.run(f, solid, p, STEPS)
    m = S.macroscopic(f, solid, p)
    assert bool(torch.isfinite(m["rho"]).all()), f"{name}: oracle went non-finite"
    rho, u = m["rho"].numpy(), m["u"].numpy()
    extra = {}
    if "planes" in c:  # large copies: keep every fourth z-plane
        planes = np.asarray(c["planes"], dtype=np.int64)
        rho, u = rho[planes], u[:, planes]
        extra["planes"] = planes
    np.savez_compressed(os.path.join(HERE, f"long_{name}.npz"), rho=rho.astype(np.float32),
                        u=u.astype(np.float32), mass=np.float64(m["mass"]), steps=STEPS, **extra)
    print(f"{name}: {time.time() - t0:.0f} s, max|u| {float(m['u'].abs().max()):.4g}, "
          f"rho in [{float(m['rho'][~solid].min()):.4f}, {float(m['rho'][~solid].max()):.4f}]", flush=True)


if __name__ == "__main__":
    if os.environ.get("ORACLE_THREADS"):
        torch.set_num_threads(int(os.environ["ORACLE_THREADS"]))
    for name in sys.argv[1:] or list(LONG_CASES):
        run(name)
