"""The C-ABI library loads and exports every function include/qsim.h declares
(CPU only: no compute call is made)."""

import ctypes
import os
import re

import numpy as np

import paper_quant_ph_9804039_gb300 as qs
from workloads.generators import GATE_DTYPE

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(qsim_\w+)\s*\(", text))
    return names


def test_library_builds_and_loads():
    lib = qs.load_library()
    assert b"sm_103a" in lib.qsim_version()


def test_every_declared_symbol_is_exported():
    lib = qs.load_library()
    names = declared_functions()
    assert len(names) >= 20
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_covers_the_header():
    assert {s[0] for s in qs.SIGNATURES} == declared_functions()


def test_gate_record_layout_matches_workloads():
    assert qs.GATE_DTYPE == GATE_DTYPE and qs.GATE_DTYPE.itemsize == 80


def test_last_error_empty_at_start():
    lib = qs.load_library()
    assert lib.qsim_last_error() == b""


def test_invalid_arguments_rejected_on_host():
    """Argument checks happen before any CUDA call, so they run without a GPU."""
    lib = qs.load_library()
    h = ctypes.c_void_p()
    assert lib.qsim_alloc(0, 0, ctypes.byref(h)) == qs.QSIM_EINVAL
    assert lib.qsim_alloc(qs.MAX_QUBITS + 1, 0, ctypes.byref(h)) == qs.QSIM_EINVAL
    assert lib.qsim_alloc(4, 7, ctypes.byref(h)) == qs.QSIM_EINVAL
    assert b"precision" in lib.qsim_last_error()
    g = np.zeros(1, dtype=GATE_DTYPE)
    g["target"] = 5
    o = qs.Opts(2, 0, 0, 0)
    assert lib.qsim_plan_create(4, 0, ctypes.c_void_p(g.ctypes.data), 1, ctypes.byref(o),
                                ctypes.byref(h)) == qs.QSIM_EINVAL
    assert b"target" in lib.qsim_last_error()
    g["target"] = 0
    g["ncontrols"] = 1
    g["controls"][0][0] = 0
    assert lib.qsim_plan_create(4, 0, ctypes.c_void_p(g.ctypes.data), 1, ctypes.byref(o),
                                ctypes.byref(h)) == qs.QSIM_EINVAL
    g["ncontrols"] = 0
    g["U"][0][0] = np.nan
    assert lib.qsim_plan_create(4, 0, ctypes.c_void_p(g.ctypes.data), 1, ctypes.byref(o),
                                ctypes.byref(h)) == qs.QSIM_EINVAL
    o = qs.Opts(2, 0, 14, 0)
    g["U"][0][0] = 1.0
    assert lib.qsim_plan_create(4, 0, ctypes.c_void_p(g.ctypes.data), 1, ctypes.byref(o),
                                ctypes.byref(h)) == qs.QSIM_EINVAL


def test_async_copy_rejects_null_on_host():
    lib = qs.load_library()
    assert lib.qsim_set_state_async(None, None, 0) == qs.QSIM_EINVAL
    assert b"NULL" in lib.qsim_last_error()


def test_set_allocator_host_checks():
    """qsim_set_allocator takes both functions or neither (no CUDA call)."""
    lib = qs.load_library()
    fa = qs.ALLOC_FN(lambda n, s, c: None)
    assert lib.qsim_set_allocator(ctypes.cast(fa, ctypes.c_void_p), None, None) == qs.QSIM_EINVAL
    assert b"both" in lib.qsim_last_error()
    assert lib.qsim_set_allocator(None, None, None) == qs.QSIM_OK


def test_gate3_record_layout_matches_workloads():
    from workloads.generators import GATE3_DTYPE
    assert qs.GATE3_DTYPE == GATE3_DTYPE and qs.GATE3_DTYPE.itemsize == 168


def test_qutrit_and_decoherence_host_checks():
    """Argument checks before any CUDA call."""
    lib = qs.load_library()
    assert lib.qsim_qutrit_apply(None, 3, 0, None, 0, None) == qs.QSIM_EINVAL
    assert lib.qsim_qutrit_apply(ctypes.c_void_p(16), 22, 0, None, 0, None) == qs.QSIM_EINVAL
    assert b"particles" in lib.qsim_last_error()
    from workloads.generators import gate3_record, pack3
    import numpy as np
    g = pack3([gate3_record(np.eye(3), 0, (0,), (1,))])  # control == target
    assert lib.qsim_qutrit_apply(ctypes.c_void_p(16), 3, 0, ctypes.c_void_p(g.ctypes.data), 1, None) == qs.QSIM_EINVAL
    g = pack3([gate3_record(np.eye(3), 1, (0,), (3,))])  # level 3
    assert lib.qsim_qutrit_apply(ctypes.c_void_p(16), 3, 0, ctypes.c_void_p(g.ctypes.data), 1, None) == qs.QSIM_EINVAL
    assert lib.qsim_run_decoherence(None, None, 0, None, None, 0.1, None, None) == qs.QSIM_EINVAL
