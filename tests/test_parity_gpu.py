"""CUDA path against the CPU oracle, element by element (GPU only).

Tolerances (stated for the spec precisions):
  complex128: ||dpsi||_2 / ||psi||_2 <= 1e-12, F and norm to 1e-12 relative;
  complex64 : max_i |da_i| <= 1e-5 and ||dpsi||_2 <= 1e-5 against the
              complex128 oracle run on the same (upcast) input; |dF| <= 1e-6.
NOT / CNOT / Toffoli (U = X exactly) are permutations and must match bitwise.
"""

import math
import os

import numpy as np
import pytest

import paper_quant_ph_9804039_gb300 as qs
from workloads import generators as W

pytestmark = pytest.mark.gpu

NT = max(1, os.cpu_count() or 1)
TOL128 = 1e-12
TOL64_MAX, TOL64_L2, TOL64_F = 1e-5, 1e-5, 1e-6


def _close(got, ref, prec):
    got = np.asarray(got, dtype=np.complex128)
    if prec == "c128":
        err = np.linalg.norm(got - ref) / max(np.linalg.norm(ref), 1e-300)
        assert err <= TOL128, err
    else:
        d = np.abs(got - ref)
        assert d.max() <= TOL64_MAX, d.max()
        assert np.linalg.norm(got - ref) <= TOL64_L2, np.linalg.norm(got - ref)


def _input(M, prec, seed=2):
    x = W.random_state(M, seed=seed, dtype=np.complex64 if prec == "c64" else np.complex128)
    return x, x.astype(np.complex128)


def _rand_gates(rng, M, n, kinds=("dense", "diag", "phase", "x")):
    recs = []
    for _ in range(n):
        kind = kinds[int(rng.integers(len(kinds)))]
        t = int(rng.integers(M))
        nc = int(rng.integers(0, min(2, M - 1) + 1))
        others = [q for q in range(M) if q != t]
        ctl = [int(v) for v in rng.choice(others, size=nc, replace=False)] if nc else []
        if kind == "dense":
            U = W.mat_haar_su2(rng) * np.exp(1j * rng.uniform(0, 6.3))
        elif kind == "diag":
            U = np.diag(np.exp(1j * rng.uniform(0, 6.3, 2)))
        elif kind == "phase":
            U = W.mat_phase(float(rng.uniform(0, 6.3)))
        else:
            U = W.mat_x()
        recs.append(W.gate_record(U, t, ctl))
    return W._pack(recs)


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("M", [1, 2, 3, 5, 7, 8, 9, 12, 15])
def test_single_gates_every_target(orc, prec, M):
    """qsim_apply_gate for every kind, every target bit, random controls."""
    rng = np.random.default_rng(100 + M)
    x, x128 = _input(M, prec)
    st = qs.State(M, prec).set(x)
    ref = x128.copy()
    for t in range(M):
        for rec in _rand_gates(rng, M, 6):
            rec["target"] = t
            ctl = [int(c) for c in rec["controls"][: int(rec["ncontrols"])] if c != t]
            rec = W.gate_record(W.record_matrix(rec), t, ctl)
            U = W.record_matrix(rec)
            st.apply_gate(U, t, ctl)
            orc.apply_gate(ref, U, t, ctl)
    _close(st.get(), ref, prec)


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("M", [3, 8, 11, 16])
def test_not_gates_are_exact_permutations(orc, prec, M):
    """U = X with 0, 1, 2 controls moves amplitudes without arithmetic."""
    rng = np.random.default_rng(7 + M)
    x, x128 = _input(M, prec)
    recs = _rand_gates(rng, M, 60, kinds=("x",))
    for mode in ("unfused", "tiled"):
        st = qs.State(M, prec).set(x)
        st.apply_circuit(recs, mode=mode)
        ref = orc.run(M, recs, x128)
        assert np.array_equal(st.get(), ref.astype(x.dtype)), mode


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("mode,tile_bits", [("unfused", 0), ("tiled", 6), ("tiled", 9), ("tiled", 0), ("tiled", 11), ("tiled", 12), ("tiled", 13)])
@pytest.mark.parametrize("M", [4, 10, 13, 17])
def test_random_circuits(orc, prec, mode, tile_bits, M):
    if prec == "c128" and tile_bits > 12:
        pytest.skip("complex128 tiles hold at most 2^12 amplitudes")
    rng = np.random.default_rng(M * 31 + tile_bits)
    recs = _rand_gates(rng, M, 150)
    x, x128 = _input(M, prec)
    st = qs.State(M, prec).set(x)
    st.apply_circuit(recs, mode=mode, tile_bits=tile_bits)
    _close(st.get(), orc.run(M, recs, x128, nthreads=NT), prec)


@pytest.mark.parametrize("mode", ["unfused", "tiled"])
def test_c1_random_circuit_fp64(orc, mode):
    """M=10, complex128, 200 gates from seed 0, errors sigma=1e-3 from seed 1,
    start |0...0>: final states, norm and fidelity to 1e-12."""
    c = W.circuit_c1_random()
    M = c["M"]
    ideal = qs.State(M, "c128").apply_circuit(c["ideal"], mode=mode)
    noisy = qs.State(M, "c128").apply_circuit(c["noisy"], mode=mode)
    ri = orc.run(M, c["ideal"])
    rn = orc.run(M, c["noisy"])
    _close(ideal.get(), ri, "c128")
    _close(noisy.get(), rn, "c128")
    F, nrm = qs.fidelity(ideal, noisy)
    Fo, nrmo = orc.fidelity(ri, rn)
    assert abs(F - Fo) <= TOL128 * Fo and abs(nrm - nrmo) <= TOL128 * nrmo
    assert F < 1.0 - 1e-6  # the errors are visible


@pytest.mark.parametrize("M", [12, 17, 20])
@pytest.mark.parametrize("mode", ["unfused", "tiled"])
def test_qft_complex64(orc, M, mode):
    """The QFT workload (H + controlled R_k ladder + bit-reversal swaps, phase
    error sigma=1e-4) on a random normalised input, complex64 vs FP64."""
    c = W.circuit_c2_qft(M, sigma=1e-4)
    x, x128 = _input(M, "c64")
    ideal = qs.State(M).set(x).apply_circuit(c["ideal"], mode=mode)
    noisy = qs.State(M).set(x).apply_circuit(c["noisy"], mode=mode)
    ri = orc.run(M, c["ideal"], x128, nthreads=NT)
    rn = orc.run(M, c["noisy"], x128, nthreads=NT)
    _close(ideal.get(), ri, "c64")
    _close(noisy.get(), rn, "c64")
    F, nrm = qs.fidelity(ideal, noisy)
    Fo, nrmo = orc.fidelity(ri, rn)
    assert abs(F - Fo) <= TOL64_F and abs(nrm - nrmo) <= TOL64_F


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("M,tile_bits", [(9, 0), (13, 7), (16, 0), (19, 12)])
def test_phase_runs(orc, prec, M, tile_bits):
    """Long runs of diagonal gates (Rz-like diag(e^ia, e^ib), controlled
    phases, on qubits inside and outside the tile) between a few Hadamards:
    the tiled mode applies each run at once as a phase polynomial."""
    rng = np.random.default_rng(40 + M)
    recs = []
    for layer in range(5):
        for q in rng.choice(M, size=3, replace=False):
            recs.append(W.gate_record(W.mat_h(), int(q)))
        for _ in range(30):
            t = int(rng.integers(M))
            if rng.random() < 0.5:
                U = np.diag(np.exp(1j * rng.uniform(-7, 7, 2)))
                ctl = ()
            else:
                U = W.mat_phase(float(rng.uniform(-7, 7)))
                ctl = (int(rng.choice([q for q in range(M) if q != t])),)
            recs.append(W.gate_record(U, t, ctl))
    recs = W._pack(recs)
    x, x128 = _input(M, prec)
    st = qs.State(M, prec).set(x).apply_circuit(recs, mode="tiled", tile_bits=tile_bits)
    _close(st.get(), orc.run(M, recs, x128, nthreads=NT), prec)


@pytest.mark.parametrize("M,tile_bits", [(14, 12), (18, 12), (18, 11), (22, 12)])
def test_phase_runs_one_shared_qubit(orc, M, tile_bits):
    """Runs whose controlled phases all share one qubit q (the quantum FFT's
    ladder after a Hadamard), with q as target or as control, controls inside
    and outside the tile, and single-qubit phases on other qubits mixed in."""
    rng = np.random.default_rng(70 + M + tile_bits)
    recs = []
    for layer in range(6):
        q = int(rng.integers(M))
        recs.append(W.gate_record(W.mat_h(), q))
        for _ in range(25):
            o = int(rng.choice([v for v in range(M) if v != q]))
            r = rng.random()
            if r < 0.6:
                recs.append(W.gate_record(W.mat_phase(float(rng.uniform(-7, 7))), q, (o,)))
            elif r < 0.8:
                recs.append(W.gate_record(W.mat_phase(float(rng.uniform(-7, 7))), o, (q,)))
            else:
                recs.append(W.gate_record(np.diag(np.exp(1j * rng.uniform(-7, 7, 2))), o))
        recs.append(W.gate_record(W.mat_haar_su2(rng), int(rng.integers(M))))
    recs = W._pack(recs)
    x, x128 = _input(M, "c64")
    st = qs.State(M, "c64").set(x).apply_circuit(recs, mode="tiled", tile_bits=tile_bits)
    _close(st.get(), orc.run(M, recs, x128, nthreads=NT), "c64")


@pytest.mark.parametrize("M", [14, 18])
def test_brickwork_toffoli_complex64(orc, M):
    """The brickwork + Toffoli workload at reduced M, tiled and unfused."""
    c = W.circuit_c4_brickwork_toffoli(M, layers=8)
    x, x128 = _input(M, "c64")
    rn = orc.run(M, c["noisy"], x128, nthreads=NT)
    for mode in ("unfused", "tiled"):
        st = qs.State(M).set(x).apply_circuit(c["noisy"], mode=mode)
        _close(st.get(), rn, "c64")


@pytest.mark.parametrize("prec", ["c64", "c128"])
@pytest.mark.parametrize("M", [1, 2, 3, 4, 11, 20])
def test_reductions(orc, prec, M):
    """norm, fidelity and probabilities against the oracle's sums."""
    x, x128 = _input(M, prec, seed=3)
    y, y128 = _input(M, prec, seed=4)
    y = (0.6 * x + 0.8 * y).astype(x.dtype)
    y128 = y.astype(np.complex128)
    a = qs.State(M, prec).set(x)
    b = qs.State(M, prec).set(y)
    F, nrm = qs.fidelity(a, b)
    Fo, nrmo = orc.fidelity(x128, y128)
    tol = 1e-12 if prec == "c128" else 1e-6
    assert abs(F - Fo) <= tol * max(1.0, Fo) and abs(nrm - nrmo) <= tol * max(1.0, nrmo)
    assert abs(a.norm() - orc.norm(x128)) <= tol
    p = a.probabilities()
    po = orc.probabilities(x128)
    assert np.allclose(p, po, rtol=1e-6 if prec == "c64" else 1e-14, atol=0)
    pd = a.probabilities(on_device=True).cpu().numpy()
    assert np.array_equal(pd, p)


def test_reduction_is_deterministic():
    M = 22
    x, _ = _input(M, "c64")
    y, _ = _input(M, "c64", seed=5)
    a = qs.State(M).set(x)
    b = qs.State(M).set(y)
    vals = {qs.fidelity(a, b) for _ in range(5)}
    assert len(vals) == 1


def test_zero_state_and_hadamards():
    """|0...0> then H on every qubit: 2^{-M/2} everywhere (Section 1.2)."""
    for M, prec in ((1, "c64"), (6, "c128"), (15, "c64")):
        st = qs.State(M, prec)
        p = st.probabilities()
        assert p[0] == 1.0 and p[1:].sum() == 0.0
        recs = W._pack([W.gate_record(W.mat_h(), q) for q in range(M)])
        st.apply_circuit(recs)
        assert np.allclose(st.get(), 2.0 ** (-M / 2), atol=1e-7 if prec == "c64" else 1e-15, rtol=0)


def test_plan_out_of_place_and_graph(orc):
    """dst = circuit(src) leaves src alone; a graph replay equals direct launches."""
    import torch
    M = 16
    c = W.circuit_c2_qft(M, sigma=1e-4)
    x, x128 = _input(M, "c64")
    s = torch.cuda.Stream()
    src = qs.State(M, stream=s).set(x)
    dst = qs.State(M, stream=s)
    ref = orc.run(M, c["noisy"], x128, nthreads=NT)
    for use_graph in (False, True):
        plan = qs.Plan(M, c["noisy"], mode="tiled", use_graph=use_graph)
        for _ in range(2):
            plan.execute(dst, src)
            s.synchronize()
            _close(dst.get(), ref, "c64")
        assert np.array_equal(src.get(), x)
    st = plan.stats()
    assert st["n_gates"] == len(c["noisy"]) and st["n_passes"] < st["n_gates"]


def test_bad_gate_rejected():
    st = qs.State(5)
    with pytest.raises(qs.QsimError) as e:
        st.apply_gate(W.mat_x(), 5)
    assert e.value.code == qs.QSIM_EINVAL
    with pytest.raises(qs.QsimError):
        st.apply_gate(W.mat_x(), 1, (1,))


def test_full_size_qft_m28():
    """The benchmark configuration (M=28, complex64, 406 gates + 14 swaps, in
    the tiled mode the benchmark times).  With sigma=0 the result must equal
    sqrt(N) ifft(x) (numpy's FFT, the closed form of the circuit) within the
    complex64 tolerance; with sigma=1e-4 the norm stays 1 and the tiled and
    one-gate-per-launch runs agree."""
    M = 28
    x, _ = _input(M, "c64")
    c0 = W.circuit_c2_qft(M, sigma=0.0)
    st = qs.State(M).set(x)
    qs.Plan(M, c0["ideal"], mode="tiled").execute(st)
    got = st.get()
    ref = np.fft.ifft(x.astype(np.complex128)) * math.sqrt(1 << M)
    d = np.abs(got - ref)
    assert d.max() <= TOL64_MAX and np.linalg.norm(got - ref) <= TOL64_L2
    del got, ref, d
    c = W.circuit_c2_qft(M, sigma=1e-4)
    a = qs.State(M).set(x)
    b = qs.State(M).set(x)
    qs.Plan(M, c["noisy"], mode="tiled").execute(a)
    qs.Plan(M, c["noisy"], mode="unfused").execute(b)
    assert abs(a.norm() - 1.0) <= 1e-5
    ideal = qs.State(M).set(x)
    qs.Plan(M, c["ideal"], mode="tiled").execute(ideal)
    Fa, na = qs.fidelity(ideal, a)
    Fb, nb = qs.fidelity(ideal, b)
    assert abs(Fa - Fb) <= TOL64_F and 0.99 < Fa <= 1.0 + TOL64_F


# ---------------------------------------------------------------- fused mode
def _fused_case(orc, M, recs, k, x=None):
    if x is None:
        x, x128 = _input(M, "c64")
    else:
        x128 = x.astype(np.complex128)
    plan = qs.Plan(M, recs, mode="fused", fuse_k=k)
    st = qs.State(M).set(x)
    plan.execute(st)
    plan.status()
    assert plan.stats()["mode"] == qs.MODE_FUSED and plan.stats()["n_blocks"] >= 1
    _close(st.get(), orc.run(M, recs, x128, nthreads=NT), "c64")
    return plan


@pytest.mark.parametrize("k", [3, 4, 5])
@pytest.mark.parametrize("M", [12, 13, 16, 20])
def test_fused_random_circuits(orc, k, M):
    """Dense k-qubit blocks on the tensor cores (split FP16 with a power-of-two
    scale per sub-vector, FP32 accumulation); M = 12 is one tile."""
    rng = np.random.default_rng(300 + 7 * M + k)
    _fused_case(orc, M, _rand_gates(rng, M, 120), k)


@pytest.mark.parametrize("k", [3, 4, 5])
@pytest.mark.parametrize("qubits", [(0, 1, 2, 3, 4), (12, 13, 14, 15, 16), (0, 3, 7, 11, 16), (1, 2, 9, 10, 15),
                                    (5, 6, 7, 8, 9), (4, 11, 12, 13, 14)])
def test_fused_block_positions(orc, k, qubits):
    """One block on low, high and mixed qubit positions (tile layouts differ)."""
    M = 17
    rng = np.random.default_rng(sum(qubits) + k)
    qs_ = list(qubits[:k])
    recs = []
    for _ in range(40):
        t = int(rng.choice(qs_))
        others = [q for q in qs_ if q != t]
        nc = int(rng.integers(0, 3))
        ctl = [int(v) for v in rng.choice(others, size=nc, replace=False)] if nc else []
        recs.append(W.gate_record(W.mat_haar_su2(rng) * np.exp(1j * rng.uniform(0, 6.3)), t, ctl))
    plan = _fused_case(orc, M, W._pack(recs), k)
    assert plan.stats()["n_blocks"] == 1


@pytest.mark.parametrize("k", [3, 4, 5])
def test_fused_qft_and_brickwork(orc, k):
    M = 18
    c = W.circuit_c2_qft(M, sigma=1e-4)
    x, x128 = _input(M, "c64")
    ideal = qs.State(M).set(x)
    noisy = qs.State(M).set(x)
    qs.Plan(M, c["ideal"], mode="fused", fuse_k=k).execute(ideal)
    pn = qs.Plan(M, c["noisy"], mode="fused", fuse_k=k)
    pn.execute(noisy)
    pn.status()
    ri = orc.run(M, c["ideal"], x128, nthreads=NT)
    rn = orc.run(M, c["noisy"], x128, nthreads=NT)
    _close(ideal.get(), ri, "c64")
    _close(noisy.get(), rn, "c64")
    F, nrm = qs.fidelity(ideal, noisy)
    Fo, nrmo = orc.fidelity(ri, rn)
    assert abs(F - Fo) <= TOL64_F and abs(nrm - nrmo) <= TOL64_F
    b = W.circuit_c4_brickwork_toffoli(M, layers=8)
    _fused_case(orc, M, b["noisy"], k, x)


@pytest.mark.parametrize("k", [3, 5])
def test_fused_dynamic_range(orc, k):
    """Groups of 32 amplitudes whose magnitudes span 50 decades, a fifth of them
    zero, under gates on qubits 0..2 (each sub-vector stays inside its group):
    every sub-vector is scaled on its own before the FP16 split, so each group
    keeps its relative precision, and zero groups stay exactly zero."""
    M = 14
    rng = np.random.default_rng(93 + k)
    x = W.random_state(M, seed=5).astype(np.complex128).reshape(-1, 32)
    mag = 10.0 ** rng.uniform(-25, 25, size=x.shape[0])
    mag[rng.random(mag.size) < 0.2] = 0.0
    x = (x * mag[:, None]).astype(np.complex64).reshape(-1)
    recs = _rand_gates(rng, 3, 40)
    plan = qs.Plan(M, recs, mode="fused", fuse_k=k)
    st = qs.State(M).set(x)
    plan.execute(st)
    plan.status()
    assert plan.stats()["mode"] == qs.MODE_FUSED
    got = st.get().astype(np.complex128).reshape(-1, 32)
    ref = orc.run(M, recs, x.astype(np.complex128), nthreads=NT).reshape(-1, 32)
    assert np.all(np.isfinite(got))
    zero = mag == 0.0
    assert np.all(got[zero] == 0)
    gmax = np.abs(ref[~zero]).max(axis=1)
    err = np.abs(got[~zero] - ref[~zero]).max(axis=1) / gmax
    assert err.max() <= 2e-6, err.max()


def test_fused_non_unitary_block(orc):
    """A non-unitary block is applied as given (no norm correction)."""
    M = 14
    rng = np.random.default_rng(91)
    recs = []
    for _ in range(12):
        U = (rng.standard_normal((2, 2)) + 1j * rng.standard_normal((2, 2))) * 0.7
        recs.append(W.gate_record(U, int(rng.integers(0, 4)), ()))
    x, x128 = _input(M, "c64")
    ref = orc.run(M, W._pack(recs), x128)
    ref_scale = np.abs(ref).max()
    plan = qs.Plan(M, W._pack(recs), mode="fused", fuse_k=4)
    st = qs.State(M).set(x)
    plan.execute(st)
    plan.status()
    got = st.get().astype(np.complex128)
    assert np.abs(got - ref).max() <= 1e-5 * max(1.0, ref_scale)


def test_fused_out_of_place(orc):
    import torch
    M = 16
    rng = np.random.default_rng(77)
    recs = _rand_gates(rng, M, 60)
    x, x128 = _input(M, "c64")
    s = torch.cuda.Stream()
    src = qs.State(M, stream=s).set(x)
    dst = qs.State(M, stream=s)
    plan = qs.Plan(M, recs, mode="fused")
    plan.execute(dst, src)
    s.synchronize()
    plan.status()
    _close(dst.get(), orc.run(M, recs, x128, nthreads=NT), "c64")
    assert np.array_equal(src.get(), x)



# -------------------------------------------------- specialised tile passes
def _spec_circuit(kind, M, rng):
    if kind == "random":
        return _rand_gates(rng, M, 150)
    if kind == "qft":
        return W.circuit_c2_qft(M, sigma=1e-4)["noisy"]
    if kind == "brickwork":
        return W.circuit_c4_brickwork_toffoli(M, layers=6)["noisy"]
    recs = []  # phase runs between Hadamards, controls inside and outside the tile
    for _ in range(4):
        for q in rng.choice(M, size=3, replace=False):
            recs.append(W.gate_record(W.mat_h(), int(q)))
        for _ in range(25):
            t = int(rng.integers(M))
            c = int(rng.choice([q for q in range(M) if q != t]))
            recs.append(W.gate_record(W.mat_phase(float(rng.uniform(-7, 7))), t, (c,)))
    return W._pack(recs)


@pytest.mark.parametrize("kind", ["random", "qft", "brickwork", "phase"])
@pytest.mark.parametrize("M,tile_bits", [(12, 12), (16, 12), (20, 11), (20, 12)])
def test_specialised_passes(orc, kind, M, tile_bits):
    """Register tile passes generated as their own kernels (NVRTC) give the
    general kernel's results bit for bit, and the oracle's within tolerance."""
    rng = np.random.default_rng(500 + M + tile_bits)
    recs = _spec_circuit(kind, M, rng)
    x, x128 = _input(M, "c64")
    gen = qs.Plan(M, recs, mode="tiled", tile_bits=tile_bits)
    spec = qs.Plan(M, recs, mode="tiled", tile_bits=tile_bits, specialize=True)
    assert "specialised" in spec.describe(), spec.describe()[:400]
    a = qs.State(M).set(x)
    gen.execute(a)
    b = qs.State(M).set(x)
    spec.execute(b)
    assert np.array_equal(a.get(), b.get())
    _close(b.get(), orc.run(M, recs, x128, nthreads=NT), "c64")


def test_auto_mode_picks_by_time_model(orc):
    """AUTO keeps the tile passes for a phase-heavy circuit (the QFT) and takes
    the fused tensor-core blocks for a dense-heavy one (Haar brickwork); both
    results agree with the oracle."""
    M = 20
    x, x128 = _input(M, "c64")
    for recs, want in ((W.circuit_c2_qft(M, sigma=1e-4)["noisy"], qs.MODE_TILED),
                       (W.circuit_c4_brickwork_toffoli(M, layers=24)["noisy"], qs.MODE_FUSED)):
        plan = qs.Plan(M, recs, mode="auto")
        assert "auto: tiled" in plan.describe()
        assert plan.stats()["mode"] == want, plan.describe().splitlines()[:3]
        st = qs.State(M).set(x)
        plan.execute(st)
        _close(st.get(), orc.run(M, recs, x128, nthreads=NT), "c64")


@pytest.mark.parametrize("specialize", [True, False])
def test_front_permutation(orc, specialize):
    """The QFT's closing swap runs become one permutation at the front (the
    gates after them relabelled).  Out of place, a specialised first pass
    gathers it while reading the source and the permutation pass is skipped;
    in place, the permutation pass runs.  Both give the same amplitudes
    bitwise, and the oracle's within tolerance."""
    M = 20
    x, x128 = _input(M, "c64")
    recs = W.circuit_c2_qft(M, sigma=1e-4)["noisy"]
    plan = qs.Plan(M, recs, mode="tiled", specialize=specialize)
    desc = plan.describe()
    assert "moved to the front" in desc
    assert ("gathered by step 1" in desc) == specialize
    src = qs.State(M).set(x)
    out = qs.State(M)
    plan.set_timing(True)
    plan.execute(out, src)
    _, _, kinds, _ = plan.timing()
    plan.set_timing(False)
    assert (kinds[0] == 6) == specialize
    inp = qs.State(M).set(x)
    plan.execute(inp)
    a, b = out.get(), inp.get()
    assert np.array_equal(a, b)
    _close(a, orc.run(M, recs, x128, nthreads=NT), "c64")


def test_set_state_async_orders_with_later_work(orc):
    """qsim_set_state_async queues the host copy on the state's own stream and
    returns; a plan executed from that state on another stream runs after the
    copy (cross-stream event), and gives the synchronous copy's result."""
    torch = pytest.importorskip("torch")
    M = 18
    x, x128 = _input(M, "c64")
    recs = W.circuit_c2_qft(M, sigma=1e-4)["noisy"]
    plan = qs.Plan(M, recs, mode="tiled", specialize=True)
    h = torch.empty(1 << M, dtype=torch.complex64, pin_memory=True)
    h.numpy()[:] = x
    copy_stream = torch.cuda.Stream()
    src = qs.State(M, stream=copy_stream, zero=False)
    out = qs.State(M)
    src.set_async(h)
    plan.execute(out, src)
    got = out.get()
    ref = qs.State(M)
    plan.execute(ref, qs.State(M).set(x))
    assert np.array_equal(got, ref.get())
    _close(got, orc.run(M, recs, x128, nthreads=NT), "c64")
