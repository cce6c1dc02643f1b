"""One state split over CPU ranks (gloo; Section 3.1, Section 3.3 Figure 8):
each rank holds 2^(M - n_global) amplitudes, runs the local gate steps that
the library planned for it (here with the oracle, on the host) and the
redistributions as chunk swaps over torch.distributed.  The assembled state
and the fidelity from the all-reduced partial sums must equal the oracle's
whole-state run: world size 2 and 4, the quantum FFT and the brickwork with
Toffolis at M = 14."""

import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, os.environ["QS_ROOT"])
import numpy as np
import torch
import torch.distributed as dist
from oracle import Oracle
from workloads import generators as W
from paper_quant_ph_9804039_gb300.shard import ShardPlan, exchange_chunks

rank, world = int(os.environ["RANK"]), int(os.environ["WORLD_SIZE"])
dist.init_process_group("gloo", rank=rank, world_size=world)
M, which = int(os.environ["QS_M"]), os.environ["QS_CIRCUIT"]
ng = world.bit_length() - 1
L = M - ng
orc = Oracle()
c = W.circuit_c2_qft(M, sigma=1e-4) if which == "qft" else W.circuit_c4_brickwork_toffoli(M, layers=8)
x = W.random_state(M, seed=2).astype(np.complex128)
res = {}
shards = {}
for name in ("ideal", "noisy"):
    sp = ShardPlan(M, ng, rank, c[name])
    shard = x[rank << L:(rank + 1) << L].copy()
    t = torch.from_numpy(shard)
    for kind, arg in sp.steps:
        if kind == "local":
            orc.apply_circuit(shard, arg)
        else:
            exchange_chunks(t, rank, L, arg)
    shards[name] = shard
    res[name] = {"exchanges": sp.n_exchanges, "moved": sp.moved}
# F and norm from the all-reduced partial sums
s = np.zeros(3)
s[0] = float(np.vdot(shards["noisy"], shards["noisy"]).real)
ov = np.vdot(shards["ideal"], shards["noisy"])
s[1], s[2] = ov.real, ov.imag
st = torch.from_numpy(s)
dist.all_reduce(st)
res["F"] = float(st[1] ** 2 + st[2] ** 2)
res["norm"] = float(st[0])
# assemble on rank 0
for name in ("ideal", "noisy"):
    t = torch.view_as_real(torch.from_numpy(shards[name])).contiguous()
    if rank == 0:
        parts = [t] + [torch.empty_like(t) for _ in range(world - 1)]
        for r in range(1, world):
            dist.recv(parts[r], r)
        full = torch.view_as_complex(torch.cat(parts)).numpy()
        ref = orc.run(M, c[name], x)
        res[name]["err"] = float(np.abs(full - ref).max())
        if name == "noisy":
            Fo, no = orc.fidelity(orc.run(M, c["ideal"], x), ref)
            res["F_err"] = abs(res["F"] - Fo)
            res["norm_err"] = abs(res["norm"] - no)
    else:
        dist.send(t, 0)
print(json.dumps(res))
dist.destroy_process_group()
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [2, 4])
@pytest.mark.parametrize("circuit", ["qft", "brickwork"])
def test_sharded_state_on_gloo_ranks(world, circuit):
    port = _free_port()
    procs = []
    for r in range(world):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), QS_ROOT=ROOT, QS_M="14", QS_CIRCUIT=circuit, CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=300)
        assert p.returncode == 0, e[-3000:]
        outs.append(json.loads(o.strip().splitlines()[-1]))
    r0 = outs[0]
    for name in ("ideal", "noisy"):
        assert r0[name]["err"] <= 1e-12, (name, r0[name])
        assert r0[name]["exchanges"] >= 1  # the circuit targets the top qubits
        assert all(o[name]["exchanges"] == r0[name]["exchanges"] for o in outs)  # the same schedule on every rank
    assert r0["F_err"] <= 1e-12 and r0["norm_err"] <= 1e-12
    assert all(abs(o["F"] - r0["F"]) < 1e-15 for o in outs)


def test_chunk_schedule_pairs_every_rank_once_per_round():
    """Round d of a redistribution pairs rank r with the rank whose pair bits
    differ by d: a perfect matching, the same on both sides."""
    sys.path.insert(0, ROOT)
    from paper_quant_ph_9804039_gb300.shard import chunk_schedule
    L, gbits, world = 10, [0, 2], 8
    sched = {r: chunk_schedule(r, L, gbits) for r in range(world)}
    for d in range(3):
        partner = {r: sched[r][d][1] for r in range(world)}
        for r in range(world):
            assert partner[partner[r]] == r and partner[r] != r
            # the partner's chunk index is this rank's own index, and vice versa
            own = sum(((r >> j) & 1) << i for i, j in enumerate(gbits))
            assert sched[partner[r]][d][0] == own


def test_shard_plan_counts_on_host():
    """The plan is host logic (no device work): exchanges only when a
    non-diagonal gate targets a rank bit; a circuit on local qubits needs none."""
    sys.path.insert(0, ROOT)
    from paper_quant_ph_9804039_gb300.shard import ShardPlan
    from workloads import generators as W
    M = 12
    local = W._pack([W.gate_record(W.mat_h(), q) for q in range(M - 2)] +
                    [W.gate_record(W.mat_phase(0.3), M - 1, (0,))])  # diagonal on a rank bit
    sp = ShardPlan(M, 2, 3, local)
    assert sp.n_exchanges == 0 and all(k == "local" for k, _ in sp.steps)
    top = W._pack([W.gate_record(W.mat_h(), M - 1)])
    sp = ShardPlan(M, 2, 0, top)
    assert sp.n_exchanges == 2  # bring it in, then restore the order
    assert abs(sp.moved - 1.0) < 1e-12  # half a shard each time
