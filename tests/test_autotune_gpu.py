"""Measured autotuning: the rates of AUTO's time model are measured on the
device once and replayed from the JSON tuning cache (in memory, then from the
file in a fresh process); AUTO's choice is recorded in the plan description;
a trajectory plan's timed configuration is replayed from the file."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

import paper_quant_ph_9804039_gb300 as qs
from workloads import generators as W

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture
def cache_file(tmp_path):
    path = tmp_path / "tune.json"
    qs.set_tune_cache(path)
    yield path
    qs.set_tune_cache(qs.DEFAULT_TUNE_CACHE)


def test_rates_measured_then_replayed(cache_file):
    r1 = qs.tune_rates("c64", specialize=False)
    assert r1["source"].startswith("measured now"), r1
    for k in ("pass_bw", "perm_bw"):
        assert 5e11 < r1[k] < 2e13, (k, r1[k])
    assert all(5e11 < v < 2e13 for v in r1["fused_direct"] + r1["fused_staged"]), r1
    assert r1["fma_rate"] > 1e12
    r2 = qs.tune_rates("c64", specialize=False)
    assert r2["source"].startswith("replayed") and r2["pass_bw"] == r1["pass_bw"]
    data = json.loads(cache_file.read_text())
    assert any(k.startswith("rates|") and k.endswith("|c64|general") for k in data), list(data)
    qs.set_tune_cache(cache_file)  # drops the memory copy: the file is read back
    r3 = qs.tune_rates("c64", specialize=False)
    assert r3["source"].startswith("replayed")
    assert abs(r3["pass_bw"] / r1["pass_bw"] - 1) < 1e-6


def test_auto_choice_recorded(cache_file):
    M = 20
    q = qs.Plan(M, W.circuit_c2_qft(M, sigma=1e-4)["noisy"], mode="auto")
    line = next(ln for ln in q.describe().splitlines() if ln.startswith("auto:"))
    for cand in ("tiled b=12", "tiled b=11", "fused k=5", "fused k=4", "fused k=3", "chosen"):
        assert cand in line, line
    assert q.stats()["mode"] == qs.MODE_TILED, line
    b = qs.Plan(M, W.circuit_c4_brickwork_toffoli(M, layers=24)["noisy"], mode="auto")
    line = next(ln for ln in b.describe().splitlines() if ln.startswith("auto:"))
    assert b.stats()["mode"] == qs.MODE_FUSED, line
    assert b.stats()["fuse_k"] in (3, 4, 5)


_CHILD = r"""
import sys
sys.path.insert(0, {root!r})
import paper_quant_ph_9804039_gb300 as qs
from workloads import generators as W
qs.set_tune_cache({path!r})
b = W.circuit_brickwork(10, 4)
print(qs.TrajPlan(10, b["ideal"], b["axes"], max_T=64, use_graph=False).describe())
"""


def test_trajectory_choice_replayed_in_a_new_process(cache_file):
    code = _CHILD.format(root=ROOT, path=str(cache_file))
    first = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert first.returncode == 0, first.stderr[-2000:]
    assert "replayed" not in first.stdout and "chosen:" in first.stdout
    assert any(k.startswith("traj|") for k in json.loads(cache_file.read_text()))
    second = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert second.returncode == 0, second.stderr[-2000:]
    assert "configuration replayed from the tuning cache" in second.stdout, second.stdout
    chosen = [ln for ln in first.stdout.splitlines() if ln.startswith("chosen:")]
    assert chosen and chosen[0] in second.stdout
