"""Scaled copies of the paper-shaped workloads for the 1000-step parity runs.

Plain data shared by the script that writes the FP64 oracle's results
(make_long_parity.py, which calls only oracle/ and the input generator) and
by the GPU test that compares the CUDA library with them.  Each copy keeps
the workload's model parameters and shrinks the domain so the oracle finishes
1000 steps in minutes:

  droplet24   stationary droplet (64^3, R = 8 workload): 24^3 periodic, R = 8,
              interface width 5, u = 0
  moving24    moving droplet (256^3, R = 32, U = (0.05, 0.02, 0), omega_1 =
              1.6 workload): 24^3 periodic, R = 6, width 2 (width 5 diverges
              with this EOS), same U and rates
  wall32p     droplet on a wall (256 x 256 x 128, R = 40, phi-wetting
              workload): 32 x 32 x 20 with solid planes z = 0 and z = 19,
              hemisphere R = 8 on the wall plane z = 0.5, width 5, phi = 1.2,
              with the paper's EOS coefficient and kappa (a = 9/392, kappa =
              0.02) at 0.8 T_c.  With a = 9/49, kappa = 0.01 a drop on a wall
              is too ill-conditioned for a 1000-step comparison (the FP64
              oracle itself moves by 1e-3 under 1e-6 noise per step) and goes
              non-finite within 40 000 steps.

The same three at the sizes of the workloads' own parity-run copies:

  droplet64   stationary droplet: 64^3 periodic, R = 8, width 5, u = 0
  moving64    moving droplet: 64^3 periodic, R = 8 (the 256^3 drop scaled by
              1/4), width 2, U = (0.05, 0.02, 0), omega_1 = 1.6
  wall64p     droplet on a wall: 64 x 64 x 32 with solid planes z = 0 and
              z = 31, hemisphere R = 10, width 5, phi = 1.2, paper EOS
              coefficient and kappa at 0.8 T_c (as wall32p)

Their results are stored on every fourth z-plane ("planes"), with the fluid
mass of the whole domain, to keep the files small.

Unless a case sets its own: van der Waals a = 9/49, b = 2/21, R = 1 at T =
0.85 T_c, kappa = 0.01.
"""

STEPS = 1000

LONG_CASES = {
    "droplet24": dict(n=(24, 24, 24), radius=8.0, width=5.0, u=(0.0, 0.0, 0.0), walls=(),
                      omega1=1.0, wetting_mode=0, wetting_value=0.0),
    "moving24": dict(n=(24, 24, 24), radius=6.0, width=2.0, u=(0.05, 0.02, 0.0), walls=(),
                     omega1=1.6, wetting_mode=0, wetting_value=0.0),
    "wall32p": dict(n=(32, 32, 20), radius=8.0, width=5.0, u=(0.0, 0.0, 0.0), walls=(0, 19),
                    omega1=1.0, wetting_mode=1, wetting_value=1.2,
                    eos=dict(a=9.0 / 392.0, b=2.0 / 21.0, R=1.0, t_over_tc=0.8, kappa=0.02)),
    "droplet64": dict(n=(64, 64, 64), radius=8.0, width=5.0, u=(0.0, 0.0, 0.0), walls=(),
                      omega1=1.0, wetting_mode=0, wetting_value=0.0, planes=tuple(range(3, 64, 4))),
    "moving64": dict(n=(64, 64, 64), radius=8.0, width=2.0, u=(0.05, 0.02, 0.0), walls=(),
                     omega1=1.6, wetting_mode=0, wetting_value=0.0, planes=tuple(range(3, 64, 4))),
    "wall64p": dict(n=(64, 64, 32), radius=10.0, width=5.0, u=(0.0, 0.0, 0.0), walls=(0, 31),
                    omega1=1.0, wetting_mode=1, wetting_value=1.2, planes=tuple(range(1, 32, 4)),
                    eos=dict(a=9.0 / 392.0, b=2.0 / 21.0, R=1.0, t_over_tc=0.8, kappa=0.02)),
}
EOS = dict(a=9.0 / 49.0, b=2.0 / 21.0, R=1.0, t_over_tc=0.85, kappa=0.01)


def eos_of(case: dict) -> dict:
    return case.get("eos", EOS)
