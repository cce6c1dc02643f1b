"""The three-state model on the GPU (qsim_qutrit_apply / qsim_qutrit_overlap;
Section 2.0, Sections 3.0-3.1) against the oracle's three-level
transformations: random laser pulses with level controls, complex64 and
complex128; an exact level permutation; the DFT3 uniform state; the sums."""

import numpy as np
import pytest

import paper_quant_ph_9804039_gb300 as qs
from workloads import generators as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("M", [1, 2, 4, 7, 11])
def test_pulses_against_oracle(orc, prec, M):
    c = W.circuit_qutrit(M, 60, seed_circuit=M)
    dt = np.complex64 if prec == "c64" else np.complex128
    x = W.random_state3(M, seed=M, dtype=dt)
    st = qs.QutritState(M, prec).set(x).apply(c["noisy"])
    got = st.get().astype(np.complex128)
    ref = orc.qutrit_apply(x.astype(np.complex128), c["noisy"])
    if prec == "c128":
        assert np.linalg.norm(got - ref) <= 1e-12
    else:
        assert np.abs(got - ref).max() <= 1e-5 and np.linalg.norm(got - ref) <= 1e-5


def test_level_permutation_is_exact(orc):
    M = 8
    shift = np.roll(np.eye(3), 1, axis=0)
    recs = W.pack3([W.gate3_record(shift, t, (c,), (v,)) for t, c, v in ((0, 3, 1), (5, 0, 2), (7, 2, 0))])
    x = W.random_state3(M, seed=4)
    got = qs.QutritState(M).set(x).apply(recs).get()
    ref = orc.qutrit_apply(x.astype(np.complex128), recs).astype(np.complex64)
    assert np.array_equal(got, ref)


def test_dft3_uniform_and_overlap(orc):
    M = 12
    st = qs.QutritState(M).apply(W.pack3([W.gate3_record(W.mat_dft3(), q) for q in range(M)]))
    assert np.allclose(st.get(), 3.0 ** (-M / 2), atol=1e-7)
    c = W.circuit_qutrit(M, 80, sigma=1e-2)
    x = W.random_state3(M, seed=1)
    a = qs.QutritState(M).set(x).apply(c["ideal"])
    b = qs.QutritState(M).set(x).apply(c["noisy"])
    n, re, im = qs.qutrit_overlap(a, b)
    ra = orc.qutrit_apply(x.astype(np.complex128), c["ideal"])
    rb = orc.qutrit_apply(x.astype(np.complex128), c["noisy"])
    ov = np.vdot(ra, rb)
    assert abs(n - np.vdot(rb, rb).real) <= 1e-6
    assert abs((re * re + im * im) - abs(ov) ** 2) <= 1e-6
    assert abs(re * re + im * im - 1.0) > 1e-6  # the errors show


def test_mult3_size():
    """3^16 states (the size of the paper's three-state benchmark): norm kept
    over 200 pulses in complex64, and equal to the complex128 run."""
    M = 16
    c = W.circuit_qutrit(M, 200, seed_circuit=16)
    a = qs.QutritState(M, "c64").apply(c["noisy"])
    b = qs.QutritState(M, "c128").apply(c["noisy"])
    n, _, _ = qs.qutrit_overlap(None, a)
    assert abs(n - 1.0) <= 1e-5
    d = a.get().astype(np.complex128) - b.get()
    assert np.abs(d).max() <= 1e-5 and np.linalg.norm(d) <= 1e-5
