"""The multi-rank path of bench.py on CPU (gloo, world size 2, 127.0.0.1).

A run on N GPUs is N independent replicas: ranks meet only in the barriers
around the timed region and in the max over ranks of the elapsed time, and
the reported value is all ranks' lattice updates over that maximum.  These
tests run those pieces as two gloo processes, and the reference arm of
bench.py under torch.distributed.run, where rank 0 alone works and prints.
"""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    ms = 10.0 + 5.0 * rank            # rank 1 is the slowest replica
    ms_max = bench.max_over_ranks(ms, w)
    nodes, steps = 1000, 4
    value = w * nodes * steps / (ms_max * 1e-3) / 1e6
    bench.barrier(w)
    out.put((rank, ms_max, value))
    dist.destroy_process_group()


def test_two_gloo_ranks_barrier_and_max_over_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    # both ranks see the slowest rank's time, and the value counts both
    # replicas' updates over it
    assert [g[1] for g in got] == [15.0, 15.0]
    assert got[0][2] == got[1][2] == pytest.approx(2 * 1000 * 4 / 15e-3 / 1e6)


def test_reference_arm_under_torchrun_prints_once():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()), "bench.py", "--impl", "reference",
           "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(l) for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["cpu_baseline"]["kind"] == "oracle"
