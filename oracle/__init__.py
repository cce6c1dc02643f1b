"""CPU complex128 oracle of the error-injecting state-vector simulator.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.
The arithmetic lives in ``qsim_oracle.c`` (plain C, compiled with gcc); this
module compiles it on first use and marshals numpy arrays to it.  It shares
no code with the CUDA path: only the seeded inputs from ``workloads`` reach
both.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qsim_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-fcx-limited-range"]


def compile_oracle(src: str = _SRC, out: str = _LIB_PATH, extra=()) -> str:
    """Compile the oracle C file into a shared library (gcc)."""
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", *CFLAGS, *extra, src, "-o", tmp, "-lm", "-lpthread"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    os.replace(tmp, out)
    return out


def _declare(lib):
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    lib.orc_apply_gate.argtypes = [dp, ctypes.c_int, dp, ctypes.c_int, ip, ctypes.c_int, ctypes.c_int]
    lib.orc_apply_gate.restype = ctypes.c_int
    lib.orc_apply_gates.argtypes = [dp, ctypes.c_int, ctypes.c_int64, dp, ip, ip, ip, ctypes.c_int]
    lib.orc_apply_gates.restype = ctypes.c_int
    lib.orc_norm.argtypes = [dp, ctypes.c_int64]
    lib.orc_norm.restype = ctypes.c_double
    lib.orc_overlap.argtypes = [dp, dp, ctypes.c_int64, dp]
    lib.orc_overlap.restype = None
    lib.orc_fidelity.argtypes = [dp, dp, ctypes.c_int64, dp, dp]
    lib.orc_fidelity.restype = None
    lib.orc_probabilities.argtypes = [dp, ctypes.c_int64, dp]
    lib.orc_probabilities.restype = None
    lib.orc_error_gate.argtypes = [dp, dp, ctypes.c_double, dp]
    lib.orc_error_gate.restype = None
    lib.orc_trajectories.argtypes = [ctypes.c_int, ctypes.c_int64, dp, ip, ip, ip, dp, dp,
                                     ctypes.c_int, dp, dp, dp, ctypes.c_int]
    lib.orc_trajectories.restype = ctypes.c_int
    lib.orc_decoherence.argtypes = [dp, ctypes.c_int, ctypes.c_int64, dp, ip, ip, ip, dp, dp, ctypes.c_double, ip,
                                    dp, ctypes.c_int]
    lib.orc_decoherence.restype = ctypes.c_int
    lib.orc_qutrit_apply.argtypes = [dp, ctypes.c_int, ctypes.c_int64, dp, ip, ip, ip, ip]
    lib.orc_qutrit_apply.restype = ctypes.c_int
    return lib


def load(path: str | None = None):
    """Load (compiling if needed) the oracle library.  ``path`` loads another
    build of it (the mutant tests use this)."""
    global _lib
    if path is not None:
        return _declare(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            if (not os.path.exists(_LIB_PATH)
                    or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC)):
                compile_oracle()
            _lib = _declare(ctypes.CDLL(_LIB_PATH))
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def _arrays(recs):
    from workloads.generators import records_to_arrays
    return records_to_arrays(recs)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


class Oracle:
    """numpy front end of one build of the oracle library."""

    def __init__(self, lib=None):
        self.lib = lib if lib is not None else load()

    # state ------------------------------------------------------------------
    @staticmethod
    def zero_state(M: int) -> np.ndarray:
        psi = np.zeros(1 << M, dtype=np.complex128)
        psi[0] = 1.0
        return psi

    def apply_gate(self, psi: np.ndarray, U, target: int, controls=(), nthreads: int = 1):
        assert psi.dtype == np.complex128 and psi.flags.c_contiguous
        M = int(psi.size).bit_length() - 1
        Uf = np.ascontiguousarray(np.asarray(U, dtype=np.complex128).reshape(4).view(np.float64))
        ctl = np.zeros(2, dtype=np.int32)
        ctl[: len(controls)] = controls
        rc = self.lib.orc_apply_gate(_dp(psi.view(np.float64)), M, _dp(Uf), int(target), _ip(ctl),
                                     len(controls), int(nthreads))
        if rc:
            raise ValueError("oracle rejected the gate")
        return psi

    def apply_circuit(self, psi: np.ndarray, recs, nthreads: int = 1):
        """Apply the gate records in order, in place."""
        assert psi.dtype == np.complex128 and psi.flags.c_contiguous
        M = int(psi.size).bit_length() - 1
        U, t, nc, c = _arrays(recs)
        rc = self.lib.orc_apply_gates(_dp(psi.view(np.float64)), M, len(t), _dp(U), _ip(t), _ip(nc),
                                      _ip(c), int(nthreads))
        if rc:
            raise ValueError("oracle rejected a gate")
        return psi

    # reductions -------------------------------------------------------------
    def norm(self, psi):
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        return float(self.lib.orc_norm(_dp(psi.view(np.float64)), psi.size))

    def overlap(self, a, b):
        a = np.ascontiguousarray(a, dtype=np.complex128)
        b = np.ascontiguousarray(b, dtype=np.complex128)
        out = np.zeros(2)
        self.lib.orc_overlap(_dp(a.view(np.float64)), _dp(b.view(np.float64)), a.size, _dp(out))
        return complex(out[0], out[1])

    def fidelity(self, ideal, noisy):
        a = np.ascontiguousarray(ideal, dtype=np.complex128)
        b = np.ascontiguousarray(noisy, dtype=np.complex128)
        F = np.zeros(1)
        nrm = np.zeros(1)
        self.lib.orc_fidelity(_dp(a.view(np.float64)), _dp(b.view(np.float64)), a.size, _dp(F), _dp(nrm))
        return float(F[0]), float(nrm[0])

    def probabilities(self, psi):
        psi = np.ascontiguousarray(psi, dtype=np.complex128)
        p = np.empty(psi.size, dtype=np.float64)
        self.lib.orc_probabilities(_dp(psi.view(np.float64)), psi.size, _dp(p))
        return p

    def error_gate(self, U, axis, eps: float) -> np.ndarray:
        Uf = np.ascontiguousarray(np.asarray(U, dtype=np.complex128).reshape(4).view(np.float64))
        ax = np.ascontiguousarray(axis, dtype=np.float64)
        out = np.zeros(8)
        self.lib.orc_error_gate(_dp(Uf), _dp(ax), float(eps), _dp(out))
        return (out[0::2] + 1j * out[1::2]).reshape(2, 2)

    def trajectories(self, M: int, recs, axes, eps, nthreads: int = 1):
        """Fidelity of every error trajectory; returns (F[T], mean, var)."""
        U, t, nc, c = _arrays(recs)
        axes = np.ascontiguousarray(axes, dtype=np.float64)
        eps = np.ascontiguousarray(eps, dtype=np.float64)
        T = eps.shape[0]
        assert eps.shape[1] == len(t)
        F = np.zeros(T)
        mean = np.zeros(1)
        var = np.zeros(1)
        rc = self.lib.orc_trajectories(M, len(t), _dp(U), _ip(t), _ip(nc), _ip(c), _dp(axes), _dp(eps),
                                       T, _dp(F), _dp(mean), _dp(var), int(nthreads))
        if rc:
            raise ValueError("oracle rejected the trajectory batch")
        return F, float(mean[0]), float(var[0])

    def decoherence(self, psi: np.ndarray, recs, delta, r, gamma: float, nthreads: int = 1):
        """Gates with dephasing and amplitude-damping jumps after each one, in
        place; returns (jumps[n], p[n])."""
        assert psi.dtype == np.complex128 and psi.flags.c_contiguous
        M = int(psi.size).bit_length() - 1
        U, t, nc, c = _arrays(recs)
        delta = np.ascontiguousarray(delta, dtype=np.float64)
        r = np.ascontiguousarray(r, dtype=np.float64)
        assert delta.size == len(t) and r.size == len(t)
        jumps = np.zeros(len(t), dtype=np.int32)
        p = np.zeros(len(t))
        rc = self.lib.orc_decoherence(_dp(psi.view(np.float64)), M, len(t), _dp(U), _ip(t), _ip(nc), _ip(c),
                                      _dp(delta), _dp(r), float(gamma), _ip(jumps), _dp(p), int(nthreads))
        if rc:
            raise ValueError("oracle rejected the decoherence run")
        return jumps, p

    def qutrit_apply(self, psi: np.ndarray, recs3):
        """Three-level transformation records applied in order to 3^M
        amplitudes, in place."""
        from workloads.generators import records3_to_arrays
        assert psi.dtype == np.complex128 and psi.flags.c_contiguous
        M = round(np.log(psi.size) / np.log(3))
        assert 3 ** M == psi.size
        U, t, nc, c, lv = records3_to_arrays(recs3)
        rc = self.lib.orc_qutrit_apply(_dp(psi.view(np.float64)), M, len(t), _dp(U), _ip(t), _ip(nc), _ip(c),
                                       _ip(lv))
        if rc:
            raise ValueError("oracle rejected a qutrit transformation")
        return psi

    # whole runs ------------------------------------------------------------
    def run(self, M: int, recs, psi0=None, nthreads: int = 1) -> np.ndarray:
        psi = self.zero_state(M) if psi0 is None else np.array(psi0, dtype=np.complex128, copy=True)
        return self.apply_circuit(psi, recs, nthreads)
