"""Full-size parity: the benchmark's own kernels in the launch configurations
the benchmark times, against the CPU oracle (GPU only).

The persistent kernels walk many tiles per block only at large M: the fused
tensor-core pass keeps one CTA per SM and wraps its input, operand and TMEM
accumulator stages (mbarrier phases flip on every reuse) once a CTA handles
more than a few tiles, and the specialised register passes prefetch the next
tile with cp.async only when a block owns a second tile.  These cases run at
M >= 24, where every block handles many tiles, and at the benchmark's exact
calls (M=28 quantum FFT, out of place from a shared input with the front
permutation gathered by the first specialised pass; the brickwork with
Toffolis from |0...0>).

Tolerances as in the rest of the suite (complex64 against the complex128
oracle): max_i |da_i| <= 1e-5, ||dpsi||_2 <= 1e-5, |dF| <= 1e-6.  At M = 33
no CPU oracle fits: there the fused and the specialised tiled runs, which
share no kernel, must agree with each other on sampled amplitudes and in F
and the norm, and the norm must stay 1 (properties that hold at any size).
"""

import math
import os

import numpy as np
import pytest

import paper_quant_ph_9804039_gb300 as qs
from workloads import generators as W

pytestmark = pytest.mark.gpu

NT = max(1, os.cpu_count() or 1)
TOL64_MAX, TOL64_L2, TOL64_F = 1e-5, 1e-5, 1e-6
CHUNK = 1 << 24


def _host_bytes() -> int:
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError):
        return 0


def _need_host(gib: float):
    if _host_bytes() < gib * (1 << 30):
        pytest.skip(f"needs {gib:.0f} GiB of host memory for the oracle")


def _errors(got: np.ndarray, ref: np.ndarray):
    """(max_i |got_i - ref_i|, ||got - ref||_2), chunk by chunk."""
    mx, ss = 0.0, 0.0
    for o in range(0, ref.size, CHUNK):
        d = np.abs(got[o:o + CHUNK].astype(np.complex128) - ref[o:o + CHUNK])
        mx = max(mx, float(d.max()))
        ss += float(np.dot(d, d))
    return mx, math.sqrt(ss)


def _close(got, ref):
    mx, l2 = _errors(got, ref)
    assert mx <= TOL64_MAX, mx
    assert l2 <= TOL64_L2, l2


def _input(M, seed=2):
    x = W.random_state(M, seed=seed)
    return x, x.astype(np.complex128)


def _rand_gates(rng, M, n, lo=0):
    """n random gates (dense SU(2) times a phase, diagonal, phase, X) with
    0..2 controls on qubits lo..M-1."""
    recs = []
    qubits = list(range(lo, M))
    for _ in range(n):
        kind = int(rng.integers(4))
        t = int(rng.choice(qubits))
        others = [q for q in qubits if q != t]
        nc = int(rng.integers(0, 3))
        ctl = [int(v) for v in rng.choice(others, size=nc, replace=False)] if nc else []
        if kind == 0:
            U = W.mat_haar_su2(rng) * np.exp(1j * rng.uniform(0, 6.3))
        elif kind == 1:
            U = np.diag(np.exp(1j * rng.uniform(0, 6.3, 2)))
        elif kind == 2:
            U = W.mat_phase(float(rng.uniform(0, 6.3)))
        else:
            U = W.mat_x()
        recs.append(W.gate_record(U, t, ctl))
    return W._pack(recs)


# ------------------------------------------------ the benchmark's M=28 call
def test_bench_call_qft_m28(orc):
    """The exact benchmark step: M=28 quantum FFT (406 gates + 14 bit-reversal
    swaps, phase error sigma=1e-4), specialised tile passes, both circuits out
    of place from one resident input (the first pass gathers the front
    permutation), then F and the norm -- against the oracle's complex128 run
    of the same records from the same (upcast) input."""
    _need_host(40)
    M = 28
    c = W.circuit_c2_qft(M, sigma=1e-4)
    x, x128 = _input(M)
    xin = qs.State(M, zero=False).set(x)
    ideal = qs.State(M, zero=False)
    noisy = qs.State(M, zero=False)
    p_i = qs.Plan(M, c["ideal"], mode="tiled", specialize=True)
    p_n = qs.Plan(M, c["noisy"], mode="tiled", specialize=True)
    assert "gathered by step 1" in p_n.describe()
    p_i.set_timing(True)
    p_i.execute(ideal, xin)
    p_n.execute(noisy, xin)
    _, _, kinds, _ = p_i.timing()
    assert kinds[0] == 6  # the permutation was gathered by the first pass, not launched
    F, nrm = qs.fidelity(ideal, noisy)
    del xin
    gi, gn = ideal.get(), noisy.get()
    del ideal, noisy
    del x
    ri = orc.run(M, c["ideal"], x128, nthreads=NT)
    _close(gi, ri)
    del gi
    rn = orc.run(M, c["noisy"], x128, nthreads=NT)
    del x128
    _close(gn, rn)
    del gn
    Fo, nrmo = orc.fidelity(ri, rn)
    assert abs(F - Fo) <= TOL64_F, (F, Fo)
    assert abs(nrm - nrmo) <= TOL64_F, (nrm, nrmo)


# ------------------------------------------- fused blocks, many tiles per CTA
@pytest.mark.parametrize("k", [3, 4, 5])
def test_fused_many_tiles_per_cta(orc, k):
    """M=24 (4096 tiles of 2^12 amplitudes, ~27 per CTA): every input, operand
    and accumulator stage is reused many times.  Random gates over all 24
    qubits give blocks on low, high and mixed positions, qubits >= 20 among
    them."""
    M = 24
    rng = np.random.default_rng(900 + k)
    recs = _rand_gates(rng, M, 160)
    x, x128 = _input(M)
    plan = qs.Plan(M, recs, mode="fused", fuse_k=k)
    st = plan.stats()
    assert st["mode"] == qs.MODE_FUSED and st["n_blocks"] >= 8
    desc = plan.describe()
    qubits_used = set()
    for line in desc.splitlines():
        if " FUSED " in line:
            qubits_used.update(int(v) for v in line.split("qubits=")[1].split("(")[0].split())
    assert min(qubits_used) <= 4 and max(qubits_used) >= 20, sorted(qubits_used)
    a = qs.State(M).set(x)
    plan.execute(a)
    plan.status()
    _close(a.get(), orc.run(M, recs, x128, nthreads=NT))


@pytest.mark.parametrize("k", [3, 5])
def test_fused_high_qubits_many_tiles(orc, k):
    """Blocks only on qubits 20..25 of an M=26 state (16384 tiles), out of place."""
    M = 26
    rng = np.random.default_rng(950 + k)
    recs = _rand_gates(rng, M, 60, lo=20)
    x, x128 = _input(M)
    plan = qs.Plan(M, recs, mode="fused", fuse_k=k)
    assert plan.stats()["mode"] == qs.MODE_FUSED
    src = qs.State(M).set(x)
    dst = qs.State(M, zero=False)
    plan.execute(dst, src)
    plan.status()
    assert np.array_equal(src.get(), x)
    _close(dst.get(), orc.run(M, recs, x128, nthreads=NT))


@pytest.mark.parametrize("k", [3, 4, 5])
def test_fused_qft_and_brickwork_m24(orc, k):
    """The two benchmark circuits in fused mode at M=24: QFT (ideal, noisy, F)
    and the 24-layer brickwork with Toffolis."""
    M = 24
    c = W.circuit_c2_qft(M, sigma=1e-4)
    x, x128 = _input(M)
    ideal = qs.State(M).set(x)
    noisy = qs.State(M).set(x)
    qs.Plan(M, c["ideal"], mode="fused", fuse_k=k).execute(ideal)
    pn = qs.Plan(M, c["noisy"], mode="fused", fuse_k=k)
    pn.execute(noisy)
    pn.status()
    ri = orc.run(M, c["ideal"], x128, nthreads=NT)
    rn = orc.run(M, c["noisy"], x128, nthreads=NT)
    _close(ideal.get(), ri)
    _close(noisy.get(), rn)
    F, nrm = qs.fidelity(ideal, noisy)
    Fo, nrmo = orc.fidelity(ri, rn)
    assert abs(F - Fo) <= TOL64_F and abs(nrm - nrmo) <= TOL64_F
    b = W.circuit_c4_brickwork_toffoli(M, layers=24)
    st = qs.State(M).set(x)
    pb = qs.Plan(M, b["noisy"], mode="fused", fuse_k=k)
    pb.execute(st)
    pb.status()
    _close(st.get(), orc.run(M, b["noisy"], x128, nthreads=NT))


# ---------------------------------------- specialised passes, many tiles/block
@pytest.mark.parametrize("kind", ["random", "qft", "brickwork", "phase"])
@pytest.mark.parametrize("tile_bits", [11, 12])
def test_specialised_many_tiles_per_block(orc, kind, tile_bits):
    """M=24: 8192 or 4096 tiles for 456 resident blocks, so every block runs
    the cp.async prefetch of its next tile.  Bitwise equal to the general
    kernel and within tolerance of the oracle."""
    M = 24
    rng = np.random.default_rng(1000 + tile_bits)
    if kind == "random":
        recs = _rand_gates(rng, M, 150)
    elif kind == "qft":
        recs = W.circuit_c2_qft(M, sigma=1e-4)["noisy"]
    elif kind == "brickwork":
        recs = W.circuit_c4_brickwork_toffoli(M, layers=12)["noisy"]
    else:
        recs = []
        for _ in range(4):
            for q in rng.choice(M, size=3, replace=False):
                recs.append(W.gate_record(W.mat_h(), int(q)))
            for _ in range(25):
                t = int(rng.integers(M))
                cq = int(rng.choice([q for q in range(M) if q != t]))
                recs.append(W.gate_record(W.mat_phase(float(rng.uniform(-7, 7))), t, (cq,)))
        recs = W._pack(recs)
    x, x128 = _input(M)
    gen = qs.Plan(M, recs, mode="tiled", tile_bits=tile_bits)
    spec = qs.Plan(M, recs, mode="tiled", tile_bits=tile_bits, specialize=True)
    assert "specialised" in spec.describe()
    a = qs.State(M).set(x)
    gen.execute(a)
    b = qs.State(M).set(x)
    spec.execute(b)
    gb = b.get()
    assert np.array_equal(a.get(), gb)
    _close(gb, orc.run(M, recs, x128, nthreads=NT))


@pytest.mark.parametrize("M", [16, 20])
@pytest.mark.parametrize("specialize", [False, True])
def test_deferred_hadamard_scale_mid_plan(orc, M, specialize):
    """Layers of Hadamards on every qubit with phase gates between them:
    more than 48 deferred 1/sqrt(2) factors, so a pass before the last one
    applies the carried factor (the 2^-24 threshold), and the last pass the
    rest.  General and specialised kernels agree bitwise; both match the
    oracle."""
    rng = np.random.default_rng(60 + M)
    recs = []
    for layer in range(5):
        for q in range(M):
            recs.append(W.gate_record(W.mat_h(), q))
        for _ in range(M):
            t = int(rng.integers(M))
            cq = int(rng.choice([q for q in range(M) if q != t]))
            recs.append(W.gate_record(W.mat_phase(float(rng.uniform(-7, 7))), t, (cq,)))
    recs = W._pack(recs)
    x, x128 = _input(M)
    plan = qs.Plan(M, recs, mode="tiled", specialize=specialize)
    tiles = [ln for ln in plan.describe().splitlines() if " TILE " in ln]
    scaled = [i for i, ln in enumerate(tiles) if "deferred-scale" in ln]
    assert len(scaled) >= 2 and scaled[0] < len(tiles) - 1, tiles
    a = qs.State(M).set(x)
    plan.execute(a)
    got = a.get()
    _close(got, orc.run(M, recs, x128, nthreads=NT))
    if specialize:
        ref = qs.State(M).set(x)
        qs.Plan(M, recs, mode="tiled").execute(ref)
        assert np.array_equal(ref.get(), got)


# ------------------------------------- the brickwork workload at M=26 and 28
@pytest.mark.parametrize("M,mode", [(26, "fused"), (26, "tiled"), (28, "fused")])
def test_brickwork_toffoli(orc, M, mode):
    """The 24-layer brickwork with a Toffoli after every 4th layer (over-
    rotation sigma=1e-3), from |0...0>, in place, as the benchmark runs it at
    M=33: ideal and noisy states, F and norm against the oracle at M=26, and
    at M=28, where the fused grouping is the beam search the benchmark's
    plans use."""
    _need_host(8 if M <= 26 else 32)
    c = W.circuit_c4_brickwork_toffoli(M, layers=24, sigma=1e-3)
    spec = mode == "tiled"
    ideal = qs.State(M)
    noisy = qs.State(M)
    p_i = qs.Plan(M, c["ideal"], mode=mode, specialize=spec)
    p_n = qs.Plan(M, c["noisy"], mode=mode, specialize=spec)
    if spec:
        assert "specialised" in p_n.describe()
    if M >= 28 and mode == "fused":  # the window grouping alone makes 66 blocks here
        assert p_n.stats()["n_blocks"] < 66, p_n.stats()["n_blocks"]
    p_i.execute(ideal)
    p_n.execute(noisy)
    p_n.status()
    F, nrm = qs.fidelity(ideal, noisy)
    ri = orc.run(M, c["ideal"], nthreads=NT)
    _close(ideal.get(), ri)
    rn = orc.run(M, c["noisy"], nthreads=NT)
    _close(noisy.get(), rn)
    Fo, nrmo = orc.fidelity(ri, rn)
    assert abs(F - Fo) <= TOL64_F, (F, Fo)
    assert abs(nrm - nrmo) <= TOL64_F, (nrm, nrmo)
    assert F < 1.0 - 1e-5  # the errors are visible


# ---------------------------------------------- M=33: properties at any size
def test_brickwork_m33_fused_vs_tiled():
    """M=33 (64 GiB per state; no CPU oracle fits): the fused tensor-core run
    and the specialised tiled run of the benchmark's brickwork agree on 32
    sampled runs of 2^16 amplitudes (each within the complex64 tolerance of
    the truth, so within twice it of each other), in F and in the norm; the
    norm stays 1."""
    import torch
    M = 33
    free, _ = torch.cuda.mem_get_info()
    if free < (2 << M) * 8 + (4 << 30):
        pytest.skip("needs 2 x 64 GiB of device memory")
    c = W.circuit_c4_brickwork_toffoli(M, layers=24, sigma=1e-3)
    ideal = qs.State(M)
    noisy = qs.State(M)
    rng = np.random.default_rng(33)
    offs = sorted(int(o) * (1 << 16) for o in rng.choice(1 << (M - 16), size=32, replace=False))
    res = {}
    for mode in ("fused", "tiled"):
        spec = mode == "tiled"
        p_i = qs.Plan(M, c["ideal"], mode=mode, specialize=spec)
        p_n = qs.Plan(M, c["noisy"], mode=mode, specialize=spec)
        ideal.reset()
        noisy.reset()
        p_i.execute(ideal)
        p_n.execute(noisy)
        p_n.status()
        F, nrm = qs.fidelity(ideal, noisy)
        samp = np.concatenate([noisy.tensor[o:o + (1 << 16)].cpu().numpy() for o in offs])
        res[mode] = (F, nrm, samp)
        del p_i, p_n
    (Ff, nf, sf), (Ft, nt, st) = res["fused"], res["tiled"]
    assert abs(nf - 1.0) <= 1e-5 and abs(nt - 1.0) <= 1e-5, (nf, nt)
    assert abs(Ff - Ft) <= 2 * TOL64_F, (Ff, Ft)
    assert np.abs(sf.astype(np.complex128) - st).max() <= 2 * TOL64_MAX
