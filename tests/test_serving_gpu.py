"""The continuous-batching request loop (qsim_server_*) on the GPU.

A request's kernels, launch shapes and reduction order do not depend on what
else runs, so its fidelity and norm must be the same (bit for bit) alone and
in a mix of concurrent requests; against the oracle they agree to 1e-6.
"""

import os
import time

import numpy as np
import pytest

import paper_quant_ph_9804039_gb300 as qs
from workloads import generators as W

pytestmark = pytest.mark.gpu
NT = max(1, os.cpu_count() or 1)


def _items(n, seed, m_lo=10, m_hi=18, len_lo=40, len_hi=200):
    reqs = W.serving_requests(n, m_lo, m_hi, len_lo, len_hi, seed=seed)
    return [(r, W.request_circuit(r)) for r in reqs]


def _run(server, items):
    ids = {}
    for r, c in items:
        ids[server.submit(r["M"], c["ideal"], c["noisy"])] = r["id"]
    out = {}
    deadline = time.time() + 300
    while len(out) < len(items) and time.time() < deadline:
        for res in server.poll(256, wait_ms=1000):
            out[ids[res["id"]]] = res
    assert len(out) == len(items)
    return out


def test_alone_equals_mix():
    items = _items(24, seed=21)
    s1 = qs.Server(hbm_budget=1 << 30, max_slots=1)
    alone = {}
    for it in items:
        alone.update(_run(s1, [it]))
    s1.close()
    s8 = qs.Server(hbm_budget=1 << 30, max_slots=8)
    mix = _run(s8, items)
    st = s8.stats()
    s8.close()
    assert st["max_active"] > 1 and st["n_completed"] == len(items)
    for rid, a in alone.items():
        b = mix[rid]
        assert a["status"] == 0 and b["status"] == 0
        assert a["F"] == b["F"] and a["norm"] == b["norm"], rid


def test_results_match_oracle(orc):
    items = _items(6, seed=22, m_lo=8, m_hi=14)
    srv = qs.Server(hbm_budget=1 << 30, max_slots=4)
    out = _run(srv, items)
    srv.close()
    for r, c in items:
        ri = orc.run(r["M"], c["ideal"], nthreads=NT)
        rn = orc.run(r["M"], c["noisy"], nthreads=NT)
        Fo, no = orc.fidelity(ri, rn)
        assert abs(out[r["id"]]["F"] - Fo) <= 1e-6 and abs(out[r["id"]]["norm"] - no) <= 1e-6


def test_budget_admission():
    """With room for only a few requests at once, memory held never exceeds the
    budget, everything completes, and a request that can never fit is
    rejected with QSIM_ENOMEM."""
    items = _items(16, seed=23, m_lo=16, m_hi=18)
    budget = 3 * 2 * 8 * (1 << 18)
    srv = qs.Server(hbm_budget=budget, max_slots=8)
    out = _run(srv, items)
    st = srv.stats()
    assert st["peak_bytes"] <= budget and all(v["status"] == 0 for v in out.values())
    big = _items(1, seed=24, m_lo=22, m_hi=22)[0]
    rid = srv.submit(22, big[1]["ideal"], big[1]["noisy"])
    res = []
    while not res:
        res = srv.poll(1, wait_ms=1000)
    assert res[0]["id"] == rid and res[0]["status"] == qs.QSIM_ENOMEM
    srv.close()


def test_bad_request_rejected_at_submit():
    srv = qs.Server(hbm_budget=1 << 26, max_slots=2)
    g = W._pack([W.gate_record(W.mat_x(), 7)])
    with pytest.raises(qs.QsimError) as e:
        srv.submit(5, g, g)
    assert e.value.code == qs.QSIM_EINVAL
    srv.close()


def test_poisson_stream_latencies():
    items = _items(60, seed=25, m_lo=12, m_hi=20, len_lo=50, len_hi=300)
    srv = qs.Server(hbm_budget=8 << 30, max_slots=8)
    ids = {}
    rng = np.random.default_rng(3)
    for r, c in items:
        time.sleep(float(rng.exponential(0.0005)))
        ids[srv.submit(r["M"], c["ideal"], c["noisy"])] = r["id"]
    out = []
    while len(out) < len(items):
        out += srv.poll(256, wait_ms=1000)
    srv.close()
    lat = np.array([o["t_done"] - o["t_submit"] for o in out])
    assert np.all(lat > 0) and np.all([o["t_start"] >= o["t_submit"] for o in out])
    assert np.percentile(lat, 99) >= np.percentile(lat, 50) > 0
