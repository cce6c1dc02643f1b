"""Host logic of bench.py's multi-process path on CPU ranks (gloo, world size 2):
the process group set-up, the barrier, the max over ranks of the timings, the
whole-job throughput of independent replicas, and the reference arm running on
rank 0 alone."""

import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, os, sys, argparse
sys.path.insert(0, os.environ["BENCH_ROOT"])
import bench
rank, world, local = bench.dist_setup()
bench.dist_init(world, local, backend="gloo")
bench.barrier(world)
ms = bench.max_over_ranks(10.0 + 5.0 * rank, world)
v = bench.job_throughput(1e9, world, ms)
ref = bench.run_reference(argparse.Namespace(workload="qft-m26-c64", steps=1, warmup=0), rank, world) if rank else None
bench.barrier(world)
print(json.dumps({"rank": rank, "world": world, "ms": ms, "value": v, "ref": ref}))
import torch.distributed as dist
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), BENCH_ROOT=ROOT)
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for d in outs:
        assert d["world"] == 2
        assert d["ms"] == 15.0  # the slowest rank's time on every rank
        assert abs(d["value"] - 2 * 1e9 / 15e-3) < 1e-3 * d["value"]
    assert outs[1]["ref"] is None  # the reference arm does no work off rank 0


def test_single_rank_defaults():
    sys.path.insert(0, ROOT)
    import bench
    env = {k: os.environ.pop(k) for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK") if k in os.environ}
    try:
        assert bench.dist_setup() == (0, 1, 0)
        assert bench.max_over_ranks(3.5, 1) == 3.5
        assert bench.job_throughput(2e9, 1, 4.0) == 2e9 / 4e-3
    finally:
        os.environ.update(env)


def test_clock_sampler_summary():
    """The clocks record of a bench line: median SM clock over the samples
    taken inside the timed region only, the maximum clock, and every throttle
    reason that was Active in any of them."""
    sys.path.insert(0, ROOT)
    import bench
    cs = bench.ClockSampler(0)
    cs.lines = [
        "1200, 2070, 300.0, 0x0, Not Active, Active, Not Active, Not Active",  # before the region
        "2070, 2070, 1100.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "2055, 2070, 1350.0, 0x4, Not Active, Not Active, Not Active, Active",
        "2070, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
    ]
    cs.start = 1
    s = cs.summary()
    assert s["samples"] == 3
    assert s["sm_mhz"] == 2070.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]  # the hw_thermal line before the region is not counted
    empty = bench.ClockSampler(0)
    assert empty.summary()["reasons"] == ["unavailable"]
