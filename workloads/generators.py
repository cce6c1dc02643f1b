"""Seeded circuit, error and state generators.

Conventions (the paper leaves these open; both the CUDA path and the oracle
receive the records built here, so a convention can never break parity):

* Qubit ``q`` is bit ``q`` of the amplitude index (bit 0 = least significant).
  Section 1.2 fixes only "bit value = index of the state"; with control A =
  qubit 1 and resultant B = qubit 0, the CNOT of Table 1 / Figure 2 swaps
  amplitudes 2 and 3, as printed.
* Every gate is a controlled single-target gate: a 2x2 complex matrix ``U``,
  a target qubit and 0-2 control qubits (Section 2.0: one-, two- and three-bit
  controlled-NOTs and rotation gates).  X, CNOT and Toffoli are ``U = X``
  with 0, 1, 2 controls.  A SWAP is three exact CNOTs.
* ``Rz(t) = diag(e^{-it/2}, e^{it/2})``, ``Ry(t) = [[c, -s], [s, c]]``,
  ``Rx(t) = [[c, -is], [-is, c]]`` with ``c = cos(t/2)``, ``s = sin(t/2)``;
  ``H = [[1, 1], [1, -1]] / sqrt(2)``; ``phase(p) = diag(1, e^{ip})``.
* Operational error (Sections 1.4, 2.0: a deviation of the rotation angle):
  a rotation gate's angle becomes ``theta + eps``; a gate with a rotation axis
  ``n`` becomes ``U . exp(-i eps/2 n.sigma)`` (an over-rotation about the
  gate's own axis, or ``X . Rx(eps)`` for NOT-type gates); fixed gates of the
  random circuit get an extra ``Rz(eps)`` after them; QFT gates get a phase
  error ``diag(1, e^{i eps})``.
* Random numbers: numpy ``default_rng`` (PCG64); circuit structure from seed
  0, errors from seed 1, input states from seed 2, the served request stream
  from seed 3; per-trajectory errors from ``SeedSequence(1).spawn(T)``.

Gate records use ``GATE_DTYPE`` (80 bytes: ``U`` as 8 doubles, row-major
``U00, U01, U10, U11`` with interleaved real/imaginary parts, then int32
``target``, ``ncontrols``, ``controls[2]``).  The record is an interface
format: the C ABI declares the same layout in its own header.
"""

from __future__ import annotations

import math

import numpy as np

GATE_DTYPE = np.dtype(
    [("U", "<f8", (8,)), ("target", "<i4"), ("ncontrols", "<i4"), ("controls", "<i4", (2,))]
)
assert GATE_DTYPE.itemsize == 80

_SQ2 = 1.0 / math.sqrt(2.0)


# ---------------------------------------------------------------- matrices ---
def mat_h() -> np.ndarray:
    return np.array([[_SQ2, _SQ2], [_SQ2, -_SQ2]], dtype=np.complex128)


def mat_x() -> np.ndarray:
    return np.array([[0, 1], [1, 0]], dtype=np.complex128)


def mat_rx(t: float) -> np.ndarray:
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -1j * s], [-1j * s, c]], dtype=np.complex128)


def mat_ry(t: float) -> np.ndarray:
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array([[c, -s], [s, c]], dtype=np.complex128)


def mat_rz(t: float) -> np.ndarray:
    return np.array([[np.exp(-0.5j * t), 0], [0, np.exp(0.5j * t)]], dtype=np.complex128)


def mat_phase(p: float) -> np.ndarray:
    return np.array([[1, 0], [0, np.exp(1j * p)]], dtype=np.complex128)


def mat_rot_axis(n, t: float) -> np.ndarray:
    """exp(-i t/2 n.sigma) for a unit axis n = (nx, ny, nz)."""
    nx, ny, nz = (float(v) for v in n)
    c, s = math.cos(t / 2), math.sin(t / 2)
    return np.array(
        [[c - 1j * s * nz, -s * ny - 1j * s * nx], [s * ny - 1j * s * nx, c + 1j * s * nz]],
        dtype=np.complex128,
    )


def mat_haar_su2(rng: np.random.Generator) -> np.ndarray:
    """Haar-random SU(2): a normalised complex Gaussian pair (a, b) -> [[a, -b*], [b, a*]]."""
    v = rng.standard_normal(4)
    a = complex(v[0], v[1])
    b = complex(v[2], v[3])
    r = math.sqrt(abs(a) ** 2 + abs(b) ** 2)
    a, b = a / r, b / r
    return np.array([[a, -b.conjugate()], [b, a.conjugate()]], dtype=np.complex128)


def su2_axis(U: np.ndarray):
    """Angle and unit axis of U = cos(t/2) I - i sin(t/2) n.sigma (U in SU(2))."""
    c = U[0, 0].real
    sz = -U[0, 0].imag
    sy = U[1, 0].real
    sx = -U[1, 0].imag
    s = math.sqrt(sx * sx + sy * sy + sz * sz)
    t = 2.0 * math.atan2(s, c)
    if s == 0.0:
        return t, (0.0, 0.0, 1.0)
    return t, (sx / s, sy / s, sz / s)


# ----------------------------------------------------------------- records ---
def gate_record(U: np.ndarray, target: int, controls=()) -> np.ndarray:
    rec = np.zeros((), dtype=GATE_DTYPE)
    U = np.asarray(U, dtype=np.complex128).reshape(2, 2)
    flat = U.reshape(4)
    rec["U"][0::2] = flat.real
    rec["U"][1::2] = flat.imag
    rec["target"] = int(target)
    controls = [int(c) for c in controls]
    if len(controls) > 2:
        raise ValueError("at most two controls")
    rec["ncontrols"] = len(controls)
    for i, c in enumerate(controls):
        rec["controls"][i] = c
    return rec


def _pack(recs) -> np.ndarray:
    out = np.zeros(len(recs), dtype=GATE_DTYPE)
    for i, r in enumerate(recs):
        out[i] = r
    return out


def record_matrix(rec) -> np.ndarray:
    u = np.asarray(rec["U"], dtype=np.float64)
    return (u[0::2] + 1j * u[1::2]).reshape(2, 2)


def records_to_arrays(recs: np.ndarray):
    """Split gate records into plain arrays (U[n,8], target[n], nctl[n], ctl[n,2])."""
    recs = np.ascontiguousarray(recs, dtype=GATE_DTYPE)
    return (
        np.ascontiguousarray(recs["U"], dtype=np.float64),
        np.ascontiguousarray(recs["target"], dtype=np.int32),
        np.ascontiguousarray(recs["ncontrols"], dtype=np.int32),
        np.ascontiguousarray(recs["controls"], dtype=np.int32),
    )


def inverse_circuit(recs: np.ndarray) -> np.ndarray:
    """The gates in reverse order with U replaced by its conjugate transpose."""
    out = np.zeros(len(recs), dtype=GATE_DTYPE)
    for i, r in enumerate(recs[::-1]):
        U = record_matrix(r).conj().T
        out[i] = gate_record(U, int(r["target"]), list(r["controls"][: int(r["ncontrols"])]))
    return out


def with_errors(recs: np.ndarray, axes: np.ndarray, eps: np.ndarray) -> np.ndarray:
    """Noisy copy of an ideal circuit: U -> U . exp(-i eps/2 n.sigma) per gate.

    ``axes[g] == (0, 0, 0)`` marks a gate that takes no error.
    """
    out = recs.copy()
    for g in range(len(recs)):
        n = axes[g]
        if not np.any(n):
            continue
        U = record_matrix(recs[g]) @ mat_rot_axis(n, float(eps[g]))
        out[g] = gate_record(U, int(recs[g]["target"]), list(recs[g]["controls"][: int(recs[g]["ncontrols"])]))
    return out


# ------------------------------------------------------------------ states ---
def random_state(M: int, seed: int = 2, dtype=np.complex64) -> np.ndarray:
    """Normalised complex Gaussian state of 2^M amplitudes (seeded).

    The values are drawn in float32 and normalised in float64, then stored in
    ``dtype``; the oracle receives the same (upcast) amplitudes.
    """
    rng = np.random.default_rng(seed)
    N = 1 << M
    re = rng.standard_normal(N, dtype=np.float32)
    im = rng.standard_normal(N, dtype=np.float32)
    nrm = math.sqrt(float(np.dot(re.astype(np.float64), re)) + float(np.dot(im.astype(np.float64), im)))
    x = np.empty(N, dtype=dtype)
    x.real = re / nrm
    x.imag = im / nrm
    return x


# ---------------------------------------------------------------- circuits ---
def circuit_c1_random(M: int = 10, n_gates: int = 200, sigma: float = 1e-3,
                      seed_circuit=0, seed_err=1):
    """Random circuit: each gate uniform over {H, X, Rz(t), Ry(t), CNOT}.

    t ~ U[0, 2pi); CNOT on a random ordered pair of distinct qubits
    (control, target).  One Gaussian error per gate: rotations take t + eps,
    H and X take an extra Rz(eps) after the gate, CNOT becomes a controlled
    Rz(eps).X on the target.
    """
    rng = np.random.default_rng(seed_circuit)
    spec = []
    for _ in range(n_gates):
        kind = int(rng.integers(5))
        if kind == 4:
            c, t = (int(v) for v in rng.choice(M, size=2, replace=False))
            spec.append((kind, t, (c,), 0.0))
        else:
            t = int(rng.integers(M))
            theta = float(rng.uniform(0.0, 2.0 * math.pi)) if kind in (2, 3) else 0.0
            spec.append((kind, t, (), theta))
    eps = np.random.default_rng(seed_err).normal(0.0, sigma, size=n_gates)
    ideal, noisy = [], []
    for g, (kind, t, ctl, theta) in enumerate(spec):
        e = float(eps[g])
        if kind == 0:
            Ui, Un = mat_h(), mat_rz(e) @ mat_h()
        elif kind == 1:
            Ui, Un = mat_x(), mat_rz(e) @ mat_x()
        elif kind == 2:
            Ui, Un = mat_rz(theta), mat_rz(theta + e)
        elif kind == 3:
            Ui, Un = mat_ry(theta), mat_ry(theta + e)
        else:
            Ui, Un = mat_x(), mat_rz(e) @ mat_x()
        ideal.append(gate_record(Ui, t, ctl))
        noisy.append(gate_record(Un, t, ctl))
    return {"M": M, "ideal": _pack(ideal), "noisy": _pack(noisy), "eps": eps,
            "kinds": np.array([s[0] for s in spec], dtype=np.int32)}


def circuit_c2_qft(M: int = 28, sigma: float = 1e-4, seed_err=1, swaps: bool = True):
    """Quantum FFT circuit with a Gaussian phase error on every H and R_k.

    For q = M-1 down to 0: H on q, then for k = 2..q+1 the controlled phase
    R_k = diag(1, e^{2 pi i / 2^k}) with control q-k+1 and target q; then the
    bit-reversal swaps (q, M-1-q), each three exact CNOTs.  With sigma = 0
    the circuit maps x to sqrt(N) * ifft(x) (numpy's convention).
    Noisy H = diag(1, e^{i eps}) . H, noisy R_k = diag(1, e^{i(2pi/2^k + eps)}).
    """
    n_err = M + M * (M - 1) // 2
    eps = np.random.default_rng(seed_err).normal(0.0, sigma, size=n_err)
    ideal, noisy = [], []
    e = 0
    for q in range(M - 1, -1, -1):
        ideal.append(gate_record(mat_h(), q))
        noisy.append(gate_record(mat_phase(float(eps[e])) @ mat_h(), q))
        e += 1
        for k in range(2, q + 2):
            phi = 2.0 * math.pi / float(1 << k)
            c = q - k + 1
            ideal.append(gate_record(mat_phase(phi), q, (c,)))
            noisy.append(gate_record(mat_phase(phi + float(eps[e])), q, (c,)))
            e += 1
    assert e == n_err
    n_logical = n_err
    if swaps:
        for q in range(M // 2):
            p = M - 1 - q
            for (c, t) in ((q, p), (p, q), (q, p)):
                ideal.append(gate_record(mat_x(), t, (c,)))
                noisy.append(gate_record(mat_x(), t, (c,)))
        n_logical += M // 2
    return {"M": M, "ideal": _pack(ideal), "noisy": _pack(noisy), "eps": eps,
            "n_logical_gates": n_logical}


def circuit_brickwork(M: int, layers: int, seed_circuit=0, toffoli_every: int = 0):
    """Brickwork circuit: per layer a Haar SU(2) on every qubit, then CNOTs on
    alternating neighbour pairs (even layers (0,1),(2,3),...; odd layers
    (1,2),(3,4),...; control = lower qubit).  With ``toffoli_every = k`` a
    Toffoli on a random distinct triple (c1, c2, t) follows layers k-1,
    2k-1, ...

    Returns the ideal records and the per-gate error axes: the SU(2)'s own
    rotation axis (over-rotation), x for CNOT and Toffoli (X . Rx(eps)).
    """
    rng = np.random.default_rng(seed_circuit)
    recs, axes = [], []
    for L in range(layers):
        for q in range(M):
            U = mat_haar_su2(rng)
            _, n = su2_axis(U)
            recs.append(gate_record(U, q))
            axes.append(n)
        for q in range(L % 2, M - 1, 2):
            recs.append(gate_record(mat_x(), q + 1, (q,)))
            axes.append((1.0, 0.0, 0.0))
        if toffoli_every and (L % toffoli_every) == toffoli_every - 1:
            c1, c2, t = (int(v) for v in rng.choice(M, size=3, replace=False))
            recs.append(gate_record(mat_x(), t, (c1, c2)))
            axes.append((1.0, 0.0, 0.0))
    return {"M": M, "ideal": _pack(recs), "axes": np.array(axes, dtype=np.float64)}


def circuit_c4_brickwork_toffoli(M: int = 33, layers: int = 24, sigma: float = 1e-3,
                                 seed_circuit=0, seed_err=1):
    """Brickwork of ``layers`` layers with a Toffoli after every 4th layer and a
    Gaussian over-rotation error on every gate."""
    c = circuit_brickwork(M, layers, seed_circuit, toffoli_every=4)
    eps = np.random.default_rng(seed_err).normal(0.0, sigma, size=len(c["ideal"]))
    c["eps"] = eps
    c["noisy"] = with_errors(c["ideal"], c["axes"], eps)
    return c


def trajectory_eps(n_gates: int, T: int, sigma: float, seed: int = 1) -> np.ndarray:
    """Per-trajectory Gaussian errors eps[T, n_gates] from SeedSequence(seed).spawn(T)."""
    out = np.empty((T, n_gates), dtype=np.float64)
    for t, ss in enumerate(np.random.SeedSequence(seed).spawn(T)):
        out[t] = np.random.default_rng(ss).normal(0.0, sigma, size=n_gates)
    return out


def serving_requests(n_requests: int = 2000, m_lo: int = 12, m_hi: int = 26,
                     len_lo: int = 50, len_hi: int = 500, seed: int = 3):
    """The served request stream: per request a qubit count M ~ U{m_lo..m_hi},
    a length ~ U{len_lo..len_hi}, a log-uniform sigma in [1e-5, 1e-2] and a
    unit-rate exponential inter-arrival gap (scale it by 1/lambda)."""
    rng = np.random.default_rng(seed)
    reqs = []
    for r in range(n_requests):
        M = int(rng.integers(m_lo, m_hi + 1))
        n = int(rng.integers(len_lo, len_hi + 1))
        sigma = float(10.0 ** rng.uniform(-5.0, -2.0))
        gap = float(rng.exponential(1.0))
        reqs.append({"id": r, "M": M, "n_gates": n, "sigma": sigma, "gap": gap,
                     "seed_circuit": (3, r, 0), "seed_err": (3, r, 1)})
    return reqs


def request_circuit(req):
    """Circuit of one served request (drawn as the random circuit above)."""
    return circuit_c1_random(req["M"], req["n_gates"], req["sigma"],
                             seed_circuit=list(req["seed_circuit"]), seed_err=list(req["seed_err"]))


def circuit_gradual(M: int, start: int = 4, per_qubit: int = 16, sigma: float = 1e-3, order=None,
                    seed_circuit=0, seed_err=1):
    """A circuit that touches its qubits one at a time, as the modular
    arithmetic of the paper's factoring circuits reaches its work registers
    late (Section 3.2, Figure 7): Hadamards on the first ``start`` qubits of
    ``order`` (default 0, 1, ..., M-1); then for each further qubit q of
    ``order`` a CNOT from a random touched qubit onto q, followed by
    ``per_qubit`` gates drawn among: a Haar SU(2) on a touched qubit, a
    controlled phase between touched qubits, a Toffoli on touched qubits, a
    CNOT controlled by a qubit not touched yet (the identity at that point),
    and an Rz on a qubit not touched yet (a phase on its 0 component).  Every
    gate carries a Gaussian over-rotation error (sigma) about its own axis
    (x for the X-type gates, z for the diagonal ones)."""
    rng = np.random.default_rng(seed_circuit)
    order = list(range(M)) if order is None else [int(q) for q in order]
    assert sorted(order) == list(range(M)) and 1 <= start <= M
    recs, axes = [], []

    def add(U, t, ctl=(), ax=(0.0, 0.0, 1.0)):
        recs.append(gate_record(U, t, ctl))
        axes.append(ax)

    for q in order[:start]:
        add(mat_h(), q, (), (1.0 / np.sqrt(2.0), 0.0, 1.0 / np.sqrt(2.0)))
    touched = list(order[:start])
    for q in order[start:]:
        add(mat_x(), q, (int(rng.choice(touched)),), (1.0, 0.0, 0.0))
        touched.append(q)
        rest = [v for v in order if v not in touched]
        for _ in range(per_qubit):
            r = rng.random()
            if r < 0.45:
                U = mat_haar_su2(rng)
                add(U, int(rng.choice(touched)), (), su2_axis(U)[1])
            elif r < 0.75 and len(touched) >= 2:
                a, b = (int(v) for v in rng.choice(touched, size=2, replace=False))
                add(mat_phase(float(rng.uniform(0, 2 * np.pi))), a, (b,))
            elif r < 0.85 and len(touched) >= 3:
                a, b, c = (int(v) for v in rng.choice(touched, size=3, replace=False))
                add(mat_x(), a, (b, c), (1.0, 0.0, 0.0))
            elif r < 0.93 and rest:
                add(mat_x(), int(rng.choice(touched)), (int(rng.choice(rest)),), (1.0, 0.0, 0.0))
            elif rest:
                add(mat_rz(float(rng.uniform(0, 2 * np.pi))), int(rng.choice(rest)))
            else:
                U = mat_haar_su2(rng)
                add(U, int(rng.choice(touched)), (), su2_axis(U)[1])
    ideal = _pack(recs)
    ax = np.array(axes, dtype=np.float64)
    eps = np.random.default_rng(seed_err).normal(0.0, sigma, size=len(recs))
    return {"M": M, "ideal": ideal, "axes": ax, "eps": eps, "noisy": with_errors(ideal, ax, eps)}


# ------------------------------------------------------------------ qutrits
# The three-state model (Section 2.0): 3^M amplitudes, digit q of the base-3
# index = the level of particle q.  One transformation record: a 3x3 matrix on
# a target particle, applied where each control particle is at its level.
GATE3_DTYPE = np.dtype(
    [("U", "<f8", (18,)), ("target", "<i4"), ("ncontrols", "<i4"), ("controls", "<i4", (2,)),
     ("levels", "<i4", (2,))]
)
assert GATE3_DTYPE.itemsize == 168


def mat_pulse3(j: int, k: int, theta: float, phi: float = 0.0) -> np.ndarray:
    """A laser pulse between levels j and k of one particle (a rotation by
    theta with phase phi in that two-level subspace; the third level
    untouched)."""
    U = np.eye(3, dtype=np.complex128)
    c, s = np.cos(theta / 2), np.sin(theta / 2)
    U[j, j] = c
    U[k, k] = c
    U[j, k] = -1j * np.exp(-1j * phi) * s
    U[k, j] = -1j * np.exp(1j * phi) * s
    return U


def mat_dft3() -> np.ndarray:
    w = np.exp(2j * np.pi / 3)
    return np.array([[1, 1, 1], [1, w, w * w], [1, w * w, w]], dtype=np.complex128) / np.sqrt(3)


def gate3_record(U: np.ndarray, target: int, controls=(), levels=()) -> np.ndarray:
    rec = np.zeros((), dtype=GATE3_DTYPE)
    U = np.asarray(U, dtype=np.complex128).reshape(9)
    rec["U"][0::2] = U.real
    rec["U"][1::2] = U.imag
    rec["target"] = target
    rec["ncontrols"] = len(controls)
    for i, (c, v) in enumerate(zip(controls, levels)):
        rec["controls"][i] = c
        rec["levels"][i] = v
    return rec


def pack3(recs) -> np.ndarray:
    out = np.zeros(len(recs), dtype=GATE3_DTYPE)
    for i, r in enumerate(recs):
        out[i] = r
    return out


def record3_matrix(rec) -> np.ndarray:
    u = rec["U"]
    return (u[0::2] + 1j * u[1::2]).reshape(3, 3)


def records3_to_arrays(recs: np.ndarray):
    recs = np.ascontiguousarray(recs, dtype=GATE3_DTYPE)
    return (np.ascontiguousarray(recs["U"]), np.ascontiguousarray(recs["target"]),
            np.ascontiguousarray(recs["ncontrols"]), np.ascontiguousarray(recs["controls"]),
            np.ascontiguousarray(recs["levels"]))


def circuit_qutrit(M: int, n_gates: int, sigma: float = 1e-3, seed_circuit=0, seed_err=1):
    """Random laser pulses on M three-level particles (as the detailed model
    of Section 2.0 runs its gates): each a rotation between two levels of a
    random particle by theta ~ U[0, 2 pi) with phase phi ~ U[0, 2 pi), a third
    of them conditioned on another particle being at level 1 or 2.  The noisy
    copy deviates every angle by a Gaussian eps (sigma)."""
    rng = np.random.default_rng(seed_circuit)
    eps = np.random.default_rng(seed_err).normal(0.0, sigma, size=n_gates)
    ideal, noisy = [], []
    pairs = [(0, 1), (1, 2), (0, 2)]
    for g in range(n_gates):
        t = int(rng.integers(M))
        j, k = pairs[int(rng.integers(3))]
        theta = float(rng.uniform(0, 2 * np.pi))
        phi = float(rng.uniform(0, 2 * np.pi))
        ctl, lev = (), ()
        if M > 1 and rng.random() < 1 / 3:
            ctl = (int(rng.choice([q for q in range(M) if q != t])),)
            lev = (int(rng.integers(1, 3)),)
        ideal.append(gate3_record(mat_pulse3(j, k, theta, phi), t, ctl, lev))
        noisy.append(gate3_record(mat_pulse3(j, k, theta + eps[g], phi), t, ctl, lev))
    return {"M": M, "ideal": pack3(ideal), "noisy": pack3(noisy), "eps": eps}


def random_state3(M: int, seed: int = 2, dtype=np.complex64) -> np.ndarray:
    """A random normalised complex Gaussian vector of 3^M amplitudes."""
    rng = np.random.default_rng(seed)
    n = 3 ** M
    x = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x /= np.linalg.norm(x)
    return x.astype(dtype)
