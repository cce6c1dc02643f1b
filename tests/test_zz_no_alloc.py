"""qsim_fidelity_noalloc: the fidelity and norm for callers that cannot
allocate device memory (plugins whose host application owns all GPU memory
through its own pool, latency-critical loops that must never enter the
allocator).  It takes raw device pointers and keeps its scratch in a fixed
device array, so it must give what qsim_fidelity gives, call after call.

This file sorts last so that a run stopping at its first failure has already
run every other test; it also passes on its own in a fresh process.
"""

import ctypes

import numpy as np
import pytest

import paper_quant_ph_9804039_gb300 as qs
from workloads import generators as W

pytestmark = pytest.mark.gpu


def _noalloc(lib, a, b, M, prec, stream):
    F = ctypes.c_double()
    n = ctypes.c_double()
    rc = lib.qsim_fidelity_noalloc(ctypes.c_void_p(a), ctypes.c_void_p(b), M, prec, ctypes.c_void_p(stream),
                                   ctypes.byref(F), ctypes.byref(n))
    return rc, F.value, n.value


@pytest.mark.parametrize("M,prec", [(1, "c64"), (3, "c64"), (12, "c128"), (17, "c64"), (22, "c64")])
def test_noalloc_matches_qsim_fidelity(M, prec):
    import torch
    lib = qs.load_library()
    dt = np.complex64 if prec == "c64" else np.complex128
    x = W.random_state(M, seed=11, dtype=dt)
    y = (0.6 * x + 0.8 * W.random_state(M, seed=12, dtype=dt)).astype(dt)
    a = qs.State(M, prec).set(x)
    b = qs.State(M, prec).set(y)
    F_ref, n_ref = qs.fidelity(a, b)
    tol = 1e-6 if prec == "c64" else 1e-12
    stream = torch.cuda.current_stream().cuda_stream
    p = qs._prec(prec)
    for _ in range(2):  # two calls in a row share the fixed scratch
        rc, F, n = _noalloc(lib, a.tensor.data_ptr(), b.tensor.data_ptr(), M, p, stream)
        assert rc == qs.QSIM_OK, lib.qsim_last_error()
        assert abs(F - F_ref) <= tol * max(1.0, F_ref) and abs(n - n_ref) <= tol * max(1.0, n_ref)
    rc, F, n = _noalloc(lib, 0, b.tensor.data_ptr(), M, p, stream)  # norm alone
    assert rc == qs.QSIM_OK and F == 0.0 and abs(n - n_ref) <= tol * max(1.0, n_ref)


def test_noalloc_rejects_states_beyond_its_scratch():
    lib = qs.load_library()
    t = qs.State(4).tensor
    rc, _, _ = _noalloc(lib, t.data_ptr(), t.data_ptr(), 33, qs.QSIM_C64, 0)
    assert rc == qs.QSIM_EINVAL
    assert b"fixed scratch" in lib.qsim_last_error()
