"""Decoherence after every operation (qsim_run_decoherence; Section 3.4,
EQ 3, EQ 8 reading in the oracle): the GPU run against the oracle on the same
gates and draws, complex64 and complex128.  The jump decisions compare a
draw with a probability computed from the state, so the draws are kept at
least 1e-4 away from the oracle's probabilities (on the same side, which
leaves every decision and later probability unchanged); then the decisions
must agree exactly and the states within the precision's tolerance."""

import os

import numpy as np
import pytest

import paper_quant_ph_9804039_gb300 as qs
from workloads import generators as W

pytestmark = pytest.mark.gpu

NT = max(1, os.cpu_count() or 1)


def _case(M, n, gamma, seed, x=None):
    """n random gates (Haar SU(2) times a phase, Rz, X; 0..2 controls when M
    allows), dephasing angles and jump draws."""
    rng = np.random.default_rng(seed)
    recs = []
    for _ in range(n):
        t = int(rng.integers(M))
        nc = int(rng.integers(0, min(2, M - 1) + 1))
        ctl = [int(v) for v in rng.choice([q for q in range(M) if q != t], size=nc, replace=False)] if nc else []
        kind = int(rng.integers(3))
        U = (W.mat_haar_su2(rng) * np.exp(1j * rng.uniform(0, 6.3)) if kind == 0 else
             W.mat_rz(float(rng.uniform(0, 6.3))) if kind == 1 else W.mat_x())
        recs.append(W.gate_record(U, t, ctl))
    recs = W._pack(recs)
    delta = rng.normal(0.0, 0.05, len(recs))
    r = rng.random(len(recs))
    return recs, delta, r


def _oracle(orc, M, recs, delta, r, gamma, x):
    psi = x.astype(np.complex128).copy()
    jumps, p = orc.decoherence(psi, recs, delta, r, gamma, nthreads=NT)
    return psi, jumps, p


def _away(r, p, margin=1e-4):
    r = r.copy()
    close = np.abs(r - p) < margin
    r[close] = np.where(r[close] < p[close], p[close] - 2 * margin, p[close] + 2 * margin)
    return np.clip(r, 0.0, np.nextafter(1.0, 0.0))


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("M,n,gamma", [(1, 20, 0.3), (2, 30, 0.2), (7, 80, 0.05), (12, 120, 0.02), (18, 60, 0.01)])
def test_decoherence_against_oracle(orc, prec, M, n, gamma):
    recs, delta, r = _case(M, n, gamma, 40 + M)
    dt = np.complex64 if prec == "c64" else np.complex128
    x = W.random_state(M, seed=3, dtype=dt)
    ref, jref, pref = _oracle(orc, M, recs, delta, r, gamma, x)
    r = _away(r, pref)
    ref, jref, pref = _oracle(orc, M, recs, delta, r, gamma, x)
    st = qs.State(M, prec).set(x)
    jumps, p = qs.run_decoherence(st, recs, delta, r, gamma)
    assert np.array_equal(jumps, jref)
    got = st.get().astype(np.complex128)
    if prec == "c128":
        assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)
        assert np.abs(p - pref).max() <= 1e-12
    else:
        assert np.abs(got - ref).max() <= 1e-5 and np.linalg.norm(got - ref) <= 1e-5
        assert np.abs(p - pref).max() <= 1e-6
    assert jref.sum() >= 1 or M > 12  # the small cases take jumps


def test_decoherence_without_noise_is_the_circuit(orc):
    """gamma = 0 and delta = 0: the plain circuit."""
    M = 14
    recs, _, r = _case(M, 100, 0.0, 7)
    x = W.random_state(M, seed=3)
    st = qs.State(M).set(x)
    jumps, p = qs.run_decoherence(st, recs, np.zeros(len(recs)), r, 0.0)
    assert jumps.sum() == 0 and np.all(p == 0)
    ref = orc.run(M, recs, x.astype(np.complex128), nthreads=NT)
    got = st.get().astype(np.complex128)
    assert np.abs(got - ref).max() <= 1e-5 and np.linalg.norm(got - ref) <= 1e-5


def test_decoherence_controls_on_previous_target(orc):
    """Gates controlled by the previous operation's target (the quadruple
    path with the control inside the quadruple), and repeated targets (the
    pair path)."""
    M = 10
    rng = np.random.default_rng(3)
    recs = []
    for k in range(40):
        t = int(rng.integers(M))
        if k % 3 == 0 and recs:
            prev_t = int(recs[-1]["target"])
            if prev_t != t:
                recs.append(W.gate_record(W.mat_haar_su2(rng), t, (prev_t,)))
                continue
        recs.append(W.gate_record(W.mat_haar_su2(rng), t))
        if k % 5 == 0:
            recs.append(W.gate_record(W.mat_haar_su2(rng), t))  # same target twice
    recs = W._pack(recs)
    delta = rng.normal(0, 0.1, len(recs))
    r = rng.random(len(recs))
    x = W.random_state(M, seed=5, dtype=np.complex128)
    _, _, pref = _oracle(orc, M, recs, delta, r, 0.1, x)
    r = _away(r, pref)
    ref, jref, pref = _oracle(orc, M, recs, delta, r, 0.1, x)
    st = qs.State(M, "c128").set(x)
    jumps, p = qs.run_decoherence(st, recs, delta, r, 0.1)
    assert np.array_equal(jumps, jref)
    assert np.linalg.norm(st.get() - ref) <= 1e-12
