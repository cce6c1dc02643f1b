"""A state split over 4 shards on one GPU: each shard runs its rank's local
steps with the library's kernels (plans of L = M - 2 qubits), and the
redistributions are the same chunk swaps the ranks would send with NCCL,
done here as device copies between the shards.  The assembled state matches
the oracle's whole-state run (complex64 tolerances), and F from the summed
partial overlaps matches the oracle's F."""

import os

import numpy as np
import pytest

import paper_quant_ph_9804039_gb300 as qs
from paper_quant_ph_9804039_gb300.shard import ShardedCircuit, chunk_schedule, overlap
from workloads import generators as W

pytestmark = pytest.mark.gpu

NT = max(1, os.cpu_count() or 1)


def _run_emulated(M, ng, recs, x, mode):
    import torch
    P, L = 1 << ng, M - ng
    circs = [ShardedCircuit(M, ng, r, recs, mode=mode) for r in range(P)]
    states = [qs.State(L).set(x[r << L:(r + 1) << L]) for r in range(P)]
    segs = []
    for c in circs:
        s, ex = [[]], []
        for (kind, arg), plan in zip(c.plan.steps, c.local):
            if kind == "local":
                s[-1].append(plan)
            else:
                ex.append(arg)
                s.append([])
        segs.append((s, ex))
    nex = len(segs[0][1])
    assert all(len(e) == nex for _, e in segs)
    for i in range(nex + 1):
        for r in range(P):
            for plan in segs[r][0][i]:
                if plan is not None:
                    plan.execute(states[r])
        if i < nex:
            torch.cuda.synchronize()
            gbits = segs[0][1][i]
            C = 1 << (L - len(gbits))
            old = [s.tensor.clone() for s in states]
            for r in range(P):
                own = sum(((r >> j) & 1) << k for k, j in enumerate(gbits))
                for b, partner, off, n in chunk_schedule(r, L, gbits):
                    states[r].tensor[off:off + n].copy_(old[partner][own * C:own * C + C])
            torch.cuda.synchronize()
    return states, circs


@pytest.mark.parametrize("circuit", ["qft", "brickwork"])
@pytest.mark.parametrize("mode", ["tiled", "fused", "unfused"])
def test_four_shards_on_one_gpu(orc, circuit, mode):
    M, ng = 18, 2
    c = W.circuit_c2_qft(M, sigma=1e-4) if circuit == "qft" else W.circuit_c4_brickwork_toffoli(M, layers=8)
    x = W.random_state(M, seed=2)
    si, ci = _run_emulated(M, ng, c["ideal"], x, mode)
    sn, cn = _run_emulated(M, ng, c["noisy"], x, mode)
    assert ci[0].plan.n_exchanges >= 2
    x128 = x.astype(np.complex128)
    for states, name in ((si, "ideal"), (sn, "noisy")):
        got = np.concatenate([s.get() for s in states]).astype(np.complex128)
        ref = orc.run(M, c[name], x128, nthreads=NT)
        assert np.abs(got - ref).max() <= 1e-5 and np.linalg.norm(got - ref) <= 1e-5, name
    tot = sum(overlap(a, b) for a, b in zip(si, sn))
    F, nrm = tot[1] ** 2 + tot[2] ** 2, tot[0]
    Fo, nrmo = orc.fidelity(orc.run(M, c["ideal"], x128, nthreads=NT), orc.run(M, c["noisy"], x128, nthreads=NT))
    assert abs(F - Fo) <= 1e-6 and abs(nrm - nrmo) <= 1e-6
