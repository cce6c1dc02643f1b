"""Pins of the CPU oracle to facts fixed outside it.

Each pin takes an ``Oracle`` (``oracle.Oracle``) and raises AssertionError
when the oracle disagrees with the paper or the mathematics.  The same pins
run against the real oracle (``test_oracle_pins.py``) and against mutated
builds of it (``test_oracle_mutants.py``), where at least one must fail.
"""

from __future__ import annotations

import math
import os
from functools import reduce

import numpy as np

from workloads import generators as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


def dense_gate(M: int, U: np.ndarray, target: int, controls=()) -> np.ndarray:
    """The full 2^M x 2^M matrix of a controlled single-target gate, built by
    Kronecker products (Section 1.3): I + P1(controls) (x) (U - I)(target).
    The first Kronecker factor is the most significant qubit."""
    I2 = np.eye(2, dtype=np.complex128)
    P1 = np.diag([0.0, 1.0]).astype(np.complex128)
    factors = []
    for q in range(M - 1, -1, -1):
        if q == target:
            factors.append(np.asarray(U, dtype=np.complex128) - I2)
        elif q in controls:
            factors.append(P1)
        else:
            factors.append(I2)
    return np.eye(1 << M, dtype=np.complex128) + reduce(np.kron, factors)


def _rand_gate(rng, M, unitary=True):
    if unitary:
        U = W.mat_haar_su2(rng) * np.exp(1j * rng.uniform(0, 2 * np.pi))
    else:
        U = rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))
    t = int(rng.integers(M))
    nc = int(rng.integers(0, min(2, M - 1) + 1))
    others = [q for q in range(M) if q != t]
    ctl = [int(v) for v in rng.choice(others, size=nc, replace=False)] if nc else []
    return U, t, ctl


def _rand_state(rng, M):
    x = rng.standard_normal(1 << M) + 1j * rng.standard_normal(1 << M)
    return x / np.linalg.norm(x)


# ------------------------------------------------------------------- pins ---
def pin_fig1_superposition(orc):
    """Figure 1: |0> is (1, 0) with probabilities (1, 0); a Hadamard makes the
    superposition (1/sqrt2, 1/sqrt2) with probabilities (1/2, 1/2)."""
    rows = _read_table("fig1_qubit_vectors.txt")
    want = {c: np.zeros(2, dtype=np.complex128) for c in "ab"}
    prob = {c: np.zeros(2) for c in "ab"}
    for case, bit, re, im, p in rows:
        want[case][int(bit)] = complex(float(re), float(im))
        prob[case][int(bit)] = float(p)
    psi = orc.zero_state(1)
    assert np.array_equal(psi, want["a"])
    assert np.array_equal(orc.probabilities(psi), prob["a"])
    orc.apply_gate(psi, W.mat_h(), 0)
    assert np.allclose(psi, want["b"], atol=1e-15, rtol=0)
    assert np.allclose(orc.probabilities(psi), prob["b"], atol=1e-15, rtol=0)


def pin_table1_cnot(orc):
    """Table 1 / Figure 2: the CNOT (control A = qubit 1, resultant B = qubit 0)
    maps basis states by the truth table and swaps a2 and a3 exactly."""
    for A, B, A2, B2 in (map(int, r) for r in _read_table("table1_cnot_truth.txt")):
        psi = np.zeros(4, dtype=np.complex128)
        psi[2 * A + B] = 1.0
        orc.apply_gate(psi, W.mat_x(), 0, (1,))
        want = np.zeros(4, dtype=np.complex128)
        want[2 * A2 + B2] = 1.0
        assert np.array_equal(psi, want)
    Mx = np.array([[float(v) for v in r] for r in _read_table("fig2_cnot_matrix.txt")])
    rng = np.random.default_rng(11)
    a = rng.standard_normal(4) + 1j * rng.standard_normal(4)
    psi = a.copy()
    orc.apply_gate(psi, W.mat_x(), 0, (1,))
    assert np.array_equal(psi, Mx @ a)
    assert np.array_equal(psi, a[[0, 1, 3, 2]])


def pin_brute_force(orc):
    """Section 1.3: every gate equals the 2^M x 2^M matrix product (M <= 6),
    for random (also non-unitary) 2x2 blocks and random controls."""
    rng = np.random.default_rng(5)
    for M in range(1, 7):
        for trial in range(6):
            psi = _rand_state(rng, M)
            ref = psi.copy()
            for _ in range(12):
                U, t, ctl = _rand_gate(rng, M, unitary=bool(trial % 2))
                ref = dense_gate(M, U, t, ctl) @ ref
                orc.apply_gate(psi, U, t, ctl)
            assert np.allclose(psi, ref, atol=1e-11 * max(1.0, np.abs(ref).max()), rtol=0), (M, trial)


def pin_toffoli_permutation(orc):
    """Section 2.0's three-bit controlled-NOT is an exact permutation: it swaps
    the pairs whose two control bits are one, and nothing else."""
    rng = np.random.default_rng(6)
    M = 5
    a = rng.standard_normal(1 << M) + 1j * rng.standard_normal(1 << M)
    psi = a.copy()
    orc.apply_gate(psi, W.mat_x(), 1, (4, 2))
    perm = np.array([i ^ 2 if (i & 16) and (i & 4) else i for i in range(1 << M)])
    assert np.array_equal(psi, a[perm])


def pin_norm_preserved(orc):
    """A unitary gate keeps the sum of probabilities at one (Section 1.2)."""
    rng = np.random.default_rng(7)
    M = 10
    psi = _rand_state(rng, M)
    for _ in range(60):
        U, t, ctl = _rand_gate(rng, M, unitary=True)
        orc.apply_gate(psi, U, t, ctl)
    assert abs(orc.norm(psi) - 1.0) < 1e-13
    assert abs(orc.probabilities(psi).sum() - 1.0) < 1e-13


def pin_uniform_superposition(orc):
    """Section 1.2: a Hadamard on every qubit of |0...0> puts all 2^M values in
    equal superposition, amplitude 2^{-M/2} each."""
    for M in (1, 2, 5, 9, 12):
        psi = orc.zero_state(M)
        for q in range(M):
            orc.apply_gate(psi, W.mat_h(), q)
        assert np.allclose(psi, 2.0 ** (-M / 2), atol=1e-15, rtol=0)


def pin_inverse_returns_input(orc):
    """A circuit followed by its inverse (reversed, conjugate-transposed gates)
    returns the input state."""
    c = W.circuit_c1_random(M=8, n_gates=120)
    rng = np.random.default_rng(8)
    x = _rand_state(rng, 8)
    psi = x.copy()
    orc.apply_circuit(psi, c["noisy"])
    assert not np.allclose(psi, x, atol=1e-3)
    orc.apply_circuit(psi, W.inverse_circuit(c["noisy"]))
    assert np.allclose(psi, x, atol=1e-12, rtol=0)


def pin_qft_closed_form(orc):
    """The error-free QFT circuit (Section 2.2's quantum FFT) with its
    bit-reversal swaps maps x to sqrt(N) * ifft(x)."""
    for M in (1, 2, 3, 6, 10):
        c = W.circuit_c2_qft(M, sigma=0.0)
        x = W.random_state(M, seed=2, dtype=np.complex128)
        psi = x.copy()
        orc.apply_circuit(psi, c["ideal"])
        ref = np.fft.ifft(x) * math.sqrt(1 << M)
        assert np.allclose(psi, ref, atol=1e-13, rtol=0), M


def pin_single_error(orc):
    """One X gate with a rotation error eps about x on |0...0>: the noisy state
    is cos(eps/2)|e_t> - i sin(eps/2)|0>, so F = cos^2(eps/2) exactly."""
    M = 3
    for eps in (1e-3, 0.3, 2.0):
        recs = W._pack([W.gate_record(W.mat_x(), 1)])
        axes = np.array([[1.0, 0.0, 0.0]])
        F, mean, var = orc.trajectories(M, recs, axes, np.array([[eps]]))
        assert abs(F[0] - math.cos(eps / 2) ** 2) < 1e-15
        noisy = orc.run(M, W.with_errors(recs, axes, np.array([eps])))
        ideal = orc.run(M, recs)
        F2, nrm = orc.fidelity(ideal, noisy)
        assert abs(F2 - math.cos(eps / 2) ** 2) < 1e-15 and abs(nrm - 1.0) < 1e-15


def pin_error_gate_closed_forms(orc):
    """Angle deviation (Sections 1.4, 2.0): Rz(t) with an error about z is
    Rz(t + eps), Ry likewise; X with an error about x is X.Rx(eps) =
    cos(eps/2) X - i sin(eps/2) I; a zero axis leaves the gate unchanged."""
    for t, e in ((0.3, 0.01), (4.0, -0.2)):
        assert np.allclose(orc.error_gate(W.mat_rz(t), (0, 0, 1), e), W.mat_rz(t + e), atol=1e-15)
        assert np.allclose(orc.error_gate(W.mat_ry(t), (0, 1, 0), e), W.mat_ry(t + e), atol=1e-15)
        assert np.allclose(orc.error_gate(W.mat_rx(t), (1, 0, 0), e), W.mat_rx(t + e), atol=1e-15)
        want = math.cos(e / 2) * W.mat_x() - 1j * math.sin(e / 2) * np.eye(2)
        assert np.allclose(orc.error_gate(W.mat_x(), (1, 0, 0), e), want, atol=1e-15)
    U = W.mat_haar_su2(np.random.default_rng(3))
    assert np.array_equal(orc.error_gate(U, (0, 0, 0), 0.5), U)
    # the error follows the gate's own rotation: U . R_n(eps), not R_n(eps) . U
    e = 0.25
    assert np.allclose(orc.error_gate(W.mat_h(), (1, 0, 0), e), W.mat_h() @ W.mat_rx(e), atol=1e-15)
    assert np.allclose(orc.error_gate(W.mat_x(), (0, 1, 0), e), W.mat_x() @ W.mat_ry(e), atol=1e-15)
    assert not np.allclose(W.mat_h() @ W.mat_rx(e), W.mat_rx(e) @ W.mat_h(), atol=1e-3)


def pin_su2_over_rotation(orc):
    """A Haar SU(2) U = exp(-i t/2 n.sigma) with an error about its own axis is
    exp(-i (t + eps)/2 n.sigma)."""
    rng = np.random.default_rng(4)
    for _ in range(5):
        U = W.mat_haar_su2(rng)
        t, n = W.su2_axis(U)
        assert np.allclose(W.mat_rot_axis(n, t), U, atol=1e-14)
        e = float(rng.normal(0, 0.1))
        assert np.allclose(orc.error_gate(U, n, e), W.mat_rot_axis(n, t + e), atol=1e-14)


def pin_sigma_zero_fidelity_one(orc):
    """With no injected error the noisy run equals the ideal one: F = 1, norm 1."""
    c = W.circuit_c1_random(M=9, n_gates=150, sigma=0.0)
    ideal = orc.run(9, c["ideal"])
    noisy = orc.run(9, c["noisy"])
    F, nrm = orc.fidelity(ideal, noisy)
    assert abs(F - 1.0) < 1e-13 and abs(nrm - 1.0) < 1e-13
    b = W.circuit_brickwork(8, 4)
    eps = np.zeros((3, len(b["ideal"])))
    Fs, mean, var = orc.trajectories(8, b["ideal"], b["axes"], eps)
    assert np.all(np.abs(Fs - 1.0) < 1e-13) and var < 1e-26


def pin_reductions_library(orc):
    """norm, overlap, fidelity and probabilities agree with numpy's own
    vdot / abs on random vectors."""
    rng = np.random.default_rng(9)
    a = rng.standard_normal(1000) + 1j * rng.standard_normal(1000)
    b = rng.standard_normal(1000) + 1j * rng.standard_normal(1000)
    assert abs(orc.overlap(a, b) - np.vdot(a, b)) < 1e-10
    F, nrm = orc.fidelity(a, b)
    assert abs(F - abs(np.vdot(a, b)) ** 2) < 1e-8 * abs(np.vdot(a, b)) ** 2
    assert abs(nrm - np.vdot(b, b).real) < 1e-10
    assert np.allclose(orc.probabilities(a), np.abs(a) ** 2, rtol=1e-15, atol=0)


def pin_trajectory_statistics(orc):
    """Mean and unbiased variance of the per-trajectory fidelities, and each
    trajectory's F equals a single noisy run with that trajectory's errors."""
    M = 6
    b = W.circuit_brickwork(M, 3)
    eps = W.trajectory_eps(len(b["ideal"]), 5, 0.05)
    F, mean, var = orc.trajectories(M, b["ideal"], b["axes"], eps, nthreads=2)
    assert abs(mean - F.mean()) < 1e-15 and abs(var - F.var(ddof=1)) < 1e-15
    ideal = orc.run(M, b["ideal"])
    for t in (0, 4):
        noisy = orc.run(M, W.with_errors(b["ideal"], b["axes"], eps[t]))
        assert abs(orc.fidelity(ideal, noisy)[0] - F[t]) < 1e-12


def _decoherence_brute(M, recs, delta, r, gamma, psi):
    """The decoherence reading written out with 2^M x 2^M matrices and numpy
    sums: gate, Rz(delta) on the target, then the jump (r < gamma P1 / N) or
    no-jump operator scaled to keep the norm."""
    psi = psi.astype(np.complex128).copy()
    jumps = []
    for g in range(len(recs)):
        t = int(recs[g]["target"])
        ctl = tuple(int(c) for c in recs[g]["controls"][: int(recs[g]["ncontrols"])])
        psi = dense_gate(M, W.record_matrix(recs[g]), t, ctl) @ psi
        psi = dense_gate(M, W.mat_rz(delta[g]), t) @ psi
        ones = (np.arange(1 << M) >> t) & 1 == 1
        P1 = float(np.sum(np.abs(psi[ones]) ** 2))
        N = float(np.sum(np.abs(psi) ** 2))
        p = gamma * P1 / N
        if r[g] < p:
            K = np.array([[0, np.sqrt(gamma)], [0, 0]]) * np.sqrt(N / (gamma * P1))
        else:
            K = np.diag([1.0, np.sqrt(1 - gamma)]) * np.sqrt(N / (N - gamma * P1))
        psi = dense_gate(M, K, t) @ psi
        jumps.append(int(r[g] < p))
    return psi, np.array(jumps)


def pin_decoherence_brute_force(orc):
    """Decoherence (Section 3.4 reading): the oracle's run equals the same
    steps written with dense matrices, for random circuits and jump draws."""
    rng = np.random.default_rng(17)
    for M in (1, 3, 4):
        recs = W._pack([W.gate_record(*_rand_gate(rng, M)) for _ in range(10)])
        delta = rng.normal(0, 0.3, len(recs))
        r = rng.random(len(recs)) * 0.6
        psi0 = _rand_state(rng, M)
        ref, jref = _decoherence_brute(M, recs, delta, r, 0.4, psi0)
        got = psi0.astype(np.complex128).copy()
        jumps, p = orc.decoherence(got, recs, delta, r, 0.4)
        assert np.array_equal(jumps, jref)
        assert np.allclose(got, ref, atol=1e-12, rtol=0)
        assert abs(orc.norm(got) - orc.norm(psi0)) < 1e-12


def pin_decoherence_single_qubit(orc):
    """Closed forms on one qubit: X from |0> then damping gives |0> after a
    jump (r < gamma) and |1> after none; H gives p = gamma / 2 and, without a
    jump, (1, sqrt(1 - gamma)) / sqrt(2 - gamma); gamma = 0 with delta only is
    H then Rz(delta)."""
    g = 0.3
    for r, want in ((0.1, [1, 0]), (0.5, [0, 1])):
        psi = orc.zero_state(1)
        jumps, p = orc.decoherence(psi, W._pack([W.gate_record(W.mat_x(), 0)]), [0.0], [r], g)
        assert abs(p[0] - g) < 1e-15 and jumps[0] == int(r < g)
        assert np.allclose(psi, want, atol=1e-15)
    psi = orc.zero_state(1)
    jumps, p = orc.decoherence(psi, W._pack([W.gate_record(W.mat_h(), 0)]), [0.0], [0.9], g)
    assert abs(p[0] - g / 2) < 1e-15 and jumps[0] == 0
    assert np.allclose(psi, np.array([1.0, np.sqrt(1 - g)]) / np.sqrt(2 - g), atol=1e-15)
    psi = orc.zero_state(1)
    orc.decoherence(psi, W._pack([W.gate_record(W.mat_h(), 0)]), [0.8], [0.9], 0.0)
    assert np.allclose(psi, np.array([np.exp(-0.4j), np.exp(0.4j)]) / np.sqrt(2), atol=1e-15)


def pin_decoherence_channel(orc):
    """The two branches weighted by their probabilities give the amplitude-
    damping channel: p rho_jump + (1 - p) rho_nojump = K0 rho K0^+ + K1 rho K1^+
    (for a random 3-qubit state and each target), and gamma = delta = 0 is the
    plain circuit, bit for bit."""
    rng = np.random.default_rng(5)
    M, g = 3, 0.35
    psi0 = _rand_state(rng, M)
    rho = np.outer(psi0, psi0.conj())
    for t in range(M):
        ident = W._pack([W.gate_record(np.eye(2), t)])
        a = psi0.copy()
        ja, p = orc.decoherence(a, ident, [0.0], [0.0], g)
        b = psi0.copy()
        jb, _ = orc.decoherence(b, ident, [0.0], [1.0], g)
        assert ja[0] == 1 and jb[0] == 0
        mix = p[0] * np.outer(a, a.conj()) + (1 - p[0]) * np.outer(b, b.conj())
        K0 = dense_gate(M, np.diag([1.0, np.sqrt(1 - g)]), t)
        K1 = dense_gate(M, np.array([[0, np.sqrt(g)], [0, 0]]), t)
        assert np.allclose(mix, K0 @ rho @ K0.conj().T + K1 @ rho @ K1.conj().T, atol=1e-13)
    recs = W._pack([W.gate_record(*_rand_gate(rng, M)) for _ in range(8)])
    c = psi0.copy()
    orc.decoherence(c, recs, np.zeros(len(recs)), np.full(len(recs), 0.5), 0.0)
    assert np.array_equal(c, orc.run(M, recs, psi0))


def dense3(M: int, U: np.ndarray, target: int, controls=(), levels=()) -> np.ndarray:
    """The 3^M x 3^M matrix of one three-level transformation: I plus
    (U - I) on the target tensored with the projector on each control's
    level (digit q of the index = particle q, digit 0 least significant)."""
    factors = []
    for q in range(M - 1, -1, -1):
        if q == target:
            factors.append(np.asarray(U, dtype=np.complex128) - np.eye(3))
        elif q in controls:
            P = np.zeros((3, 3))
            v = levels[list(controls).index(q)]
            P[v, v] = 1.0
            factors.append(P)
        else:
            factors.append(np.eye(3))
    return np.eye(3 ** M, dtype=np.complex128) + reduce(np.kron, factors)


def pin_qutrit_brute_force(orc):
    """Three-state model: random pulses (controlled ones too) against dense
    3^M x 3^M products, M = 1, 2, 3."""
    for M in (1, 2, 3):
        c = W.circuit_qutrit(M, 25, seed_circuit=M)
        x = W.random_state3(M, seed=M, dtype=np.complex128)
        ref = x.copy()
        for rec in c["noisy"]:
            ctl = tuple(int(v) for v in rec["controls"][: int(rec["ncontrols"])])
            lev = tuple(int(v) for v in rec["levels"][: int(rec["ncontrols"])])
            ref = dense3(M, W.record3_matrix(rec), int(rec["target"]), ctl, lev) @ ref
        got = orc.qutrit_apply(x.copy(), c["noisy"])
        assert np.allclose(got, ref, atol=1e-13, rtol=0)
        assert abs(np.vdot(got, got).real - 1.0) < 1e-13


def pin_qutrit_special_cases(orc):
    """The discrete Fourier transform on every particle from |0...0> gives
    3^{-M/2} everywhere; the cyclic level shift applied three times returns
    the input bit for bit; pulses between levels 0 and 1 on a state without
    level 2 are the two-state simulation of the same pulses."""
    M = 4
    psi = np.zeros(3 ** M, dtype=np.complex128)
    psi[0] = 1.0
    orc.qutrit_apply(psi, W.pack3([W.gate3_record(W.mat_dft3(), q) for q in range(M)]))
    assert np.allclose(psi, 3.0 ** (-M / 2), atol=1e-15)
    shift = np.roll(np.eye(3), 1, axis=0)
    x = W.random_state3(M, seed=9, dtype=np.complex128)
    y = orc.qutrit_apply(x.copy(), W.pack3([W.gate3_record(shift, 2, (0,), (1,))] * 3))
    assert np.array_equal(x, y)
    rng = np.random.default_rng(4)
    recs3, recs2 = [], []
    for _ in range(12):
        t = int(rng.integers(M))
        th, ph = float(rng.uniform(0, 6.3)), float(rng.uniform(0, 6.3))
        U3 = W.mat_pulse3(0, 1, th, ph)
        ctl = (int(rng.choice([q for q in range(M) if q != t])),) if rng.random() < 0.5 else ()
        recs3.append(W.gate3_record(U3, t, ctl, (1,) * len(ctl)))
        recs2.append(W.gate_record(U3[:2, :2], t, ctl))
    x2 = _rand_state(rng, M)
    x3 = np.zeros(3 ** M, dtype=np.complex128)
    for i in range(1 << M):
        x3[sum(((i >> q) & 1) * 3 ** q for q in range(M))] = x2[i]
    orc.qutrit_apply(x3, W.pack3(recs3))
    y2 = orc.run(M, W._pack(recs2), x2)
    for i in range(1 << M):
        assert abs(x3[sum(((i >> q) & 1) * 3 ** q for q in range(M))] - y2[i]) < 1e-14


PINS = [v for k, v in sorted(globals().items()) if k.startswith("pin_")]
