"""Error trajectories (one persistent launch) against the CPU oracle.

F per trajectory is checked to dF = 1e-6 (complex64 amplitudes, FP64 gate and
fidelity arithmetic).  The mean then agrees to dF.  When every F moves by at
most dF the deviations from the mean move by at most 2 dF, so (Cauchy-Schwarz)
the unbiased variance moves by at most 4 std(F) dF sqrt(T/(T-1)) +
4 dF^2 T/(T-1): the variance tolerance used here.
"""

import math
import os

import numpy as np
import pytest

import paper_quant_ph_9804039_gb300 as qs
from workloads import generators as W

pytestmark = pytest.mark.gpu
NT = max(1, os.cpu_count() or 1)
DF = 1e-6


def _var_tol(var, T):
    r = T / (T - 1) if T > 1 else 1.0
    return 4.0 * math.sqrt(max(var, 0.0)) * DF * math.sqrt(r) + 4.0 * DF * DF * r


@pytest.mark.parametrize("M,layers,T", [(1, 3, 5), (6, 4, 17), (10, 6, 64), (13, 5, 40)])
def test_trajectories_match_oracle(orc, M, layers, T):
    b = W.circuit_brickwork(M, layers, toffoli_every=2 if M >= 3 else 0)
    eps = W.trajectory_eps(len(b["ideal"]), T, 5e-3)
    F, mean, var = qs.run_trajectories(M, b["ideal"], b["axes"], eps)
    Fo, mo, vo = orc.trajectories(M, b["ideal"], b["axes"], eps, nthreads=NT)
    assert np.abs(F - Fo).max() <= DF
    assert abs(mean - mo) <= DF and abs(var - vo) <= _var_tol(vo, len(F))


def test_single_error_closed_form():
    """One X with an x-axis error on |0...0>: F = cos^2(eps/2)."""
    M = 3
    recs = W._pack([W.gate_record(W.mat_x(), 1)])
    axes = np.array([[1.0, 0.0, 0.0]])
    e = np.array([[1e-3], [0.3], [2.0]])
    F, _, _ = qs.run_trajectories(M, recs, axes, e)
    assert np.allclose(F, np.cos(e[:, 0] / 2) ** 2, atol=1e-7, rtol=0)


def test_zero_error_and_empty_circuit():
    b = W.circuit_brickwork(9, 4)
    F, mean, var = qs.run_trajectories(9, b["ideal"], b["axes"], np.zeros((7, len(b["ideal"]))))
    assert np.abs(F - 1.0).max() <= 1e-6 and var <= 1e-12
    F, mean, var = qs.run_trajectories(4, W._pack([]), np.zeros((0, 3)), np.zeros((3, 0)))
    assert np.array_equal(F, np.ones(3)) and mean == 1.0 and var == 0.0


def test_graph_replay_is_deterministic(orc):
    M = 12
    b = W.circuit_brickwork(M, 6)
    eps = W.trajectory_eps(len(b["ideal"]), 300, 5e-3)
    pg = qs.TrajPlan(M, b["ideal"], b["axes"], max_T=300, use_graph=True)
    pd = qs.TrajPlan(M, b["ideal"], b["axes"], max_T=300, use_graph=False)
    F1, m1, v1 = pg.run(eps)
    F2, m2, v2 = pg.run(eps)
    F3, m3, v3 = pd.run(eps)
    assert np.array_equal(F1, F2) and np.array_equal(F1, F3)
    F4, _, _ = pg.run(eps[:100])  # a smaller batch through the same plan
    assert np.array_equal(F4, F1[:100])
    Fo, _, _ = orc.trajectories(M, b["ideal"], b["axes"], eps[:20], nthreads=NT)
    assert np.abs(F1[:20] - Fo).max() <= 1e-6


def test_batched_brickwork_m16_t4096(orc):
    """The batched workload: M=16, 4096 trajectories of a 20-layer brickwork
    (Haar SU(2) on every qubit, CNOTs on alternating pairs), over-rotation
    sigma=5e-3 from per-trajectory seeds; mean and variance of F against the
    oracle over all 4096 trajectories."""
    M, T = 16, 4096
    b = W.circuit_brickwork(M, 20)
    eps = W.trajectory_eps(len(b["ideal"]), T, 5e-3)
    plan = qs.TrajPlan(M, b["ideal"], b["axes"], max_T=T)
    F, mean, var = plan.run(eps)
    Fo, mo, vo = orc.trajectories(M, b["ideal"], b["axes"], eps, nthreads=NT)
    assert np.abs(F - Fo).max() <= DF
    assert abs(mean - mo) <= DF and abs(var - vo) <= _var_tol(vo, len(F))
    assert 0.5 < mean < 1.0 and plan.info()["n_passes"] >= 1


def _diag_circuit(M, rng):
    """Hadamards, controlled phases and Rz gates with z-axis errors (diagonal
    erroneous gates: inside the tile and on outside qubits), plus Haar gates."""
    recs, axes = [], []
    for layer in range(4):
        for q in range(M):
            recs.append(W.gate_record(W.mat_h() if layer % 2 == 0 else W.mat_haar_su2(rng), q))
            axes.append(list(W.su2_axis(W.record_matrix(recs[-1]))[1]) if layer % 2 else [1.0, 0.0, 0.0])
        for _ in range(2 * M):
            t = int(rng.integers(M))
            c = int(rng.choice([v for v in range(M) if v != t]))
            if rng.random() < 0.5:
                recs.append(W.gate_record(W.mat_phase(float(rng.uniform(-3, 3))), t, (c,)))
            else:
                recs.append(W.gate_record(W.mat_rz(float(rng.uniform(-3, 3))), t))
            axes.append([0.0, 0.0, 1.0])
    return W._pack(recs), np.array(axes, dtype=np.float64)


@pytest.mark.parametrize("kernel", ["smem", "register"])
@pytest.mark.parametrize("M,layers,T,case", [(11, 5, 40, "brick"), (13, 6, 64, "brick"), (16, 4, 50, "brick"),
                                              (12, 0, 30, "diag"), (14, 0, 30, "diag")])
def test_trajectory_kernels_match_oracle(orc, kernel, M, layers, T, case):
    """Both trajectory kernels (shared-memory tile passes; register rounds
    generated for the circuit) against the oracle, trajectory by trajectory."""
    rng = np.random.default_rng(800 + M)
    if case == "brick":
        b = W.circuit_brickwork(M, layers, toffoli_every=2)
        gates, axes = b["ideal"], b["axes"]
    else:
        gates, axes = _diag_circuit(M, rng)
    eps = W.trajectory_eps(len(gates), T, 5e-3)
    plan = qs.TrajPlan(M, gates, axes, max_T=T, kernel=kernel)
    d = plan.describe()
    assert ("chosen: register-round kernel" in d) == (kernel == "register"), d
    F, mean, var = plan.run(eps)
    Fo, mo, vo = orc.trajectories(M, gates, axes, eps, nthreads=NT)
    assert np.abs(F - Fo).max() <= DF
    assert abs(mean - mo) <= DF and abs(var - vo) <= _var_tol(vo, len(F))
