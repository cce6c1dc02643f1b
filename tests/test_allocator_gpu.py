"""qsim_set_allocator: every device allocation of the library goes through the
caller's hook (here PyTorch's caching allocator, with counters), each object
frees through the pair it was created with, and results do not change."""

import ctypes

import numpy as np
import pytest

import paper_quant_ph_9804039_gb300 as qs
from workloads import generators as W

pytestmark = pytest.mark.gpu


class Counting:
    def __init__(self):
        import torch
        self.torch = torch
        self.live = {}
        self.n_alloc = self.n_free = 0
        self.streams = set()

    def alloc(self, nbytes, stream):
        p = self.torch.cuda.caching_allocator_alloc(nbytes, stream=stream)
        self.live[p] = nbytes
        self.n_alloc += 1
        self.streams.add(stream)
        return p

    def free(self, ptr, nbytes, stream):
        assert self.live.pop(ptr) == nbytes
        self.n_free += 1
        self.torch.cuda.caching_allocator_delete(ptr)


def _run_all(lib):
    """States from qsim_alloc, a tiled and a fused plan, a trajectory plan
    and a server; returns every result."""
    M = 14
    out = {}
    c = W.circuit_c2_qft(M, sigma=1e-4)
    h = ctypes.c_void_p()
    qs._check(lib.qsim_alloc(M, qs.QSIM_C64, ctypes.byref(h)))
    g = np.ascontiguousarray(c["noisy"], dtype=qs.GATE_DTYPE)
    for mode in (qs.MODE_TILED, qs.MODE_FUSED):
        o = qs.Opts(mode, 0, 0, 0, 0)
        qs._check(lib.qsim_reset(h))
        qs._check(lib.qsim_apply_circuit(h, ctypes.c_void_p(g.ctypes.data), len(g), ctypes.byref(o)))
        amps = np.empty(1 << M, dtype=np.complex64)
        qs._check(lib.qsim_get_state(h, ctypes.c_void_p(amps.ctypes.data), 0))
        out[f"state{mode}"] = amps
    p = np.empty(1 << M, dtype=np.float32)
    qs._check(lib.qsim_probabilities(h, ctypes.c_void_p(p.ctypes.data), 0))
    out["probs"] = p
    lib.qsim_free(h)
    b = W.circuit_brickwork(10, 6)
    eps = W.trajectory_eps(len(b["ideal"]), 64, 5e-3)
    out["traj"] = qs.TrajPlan(10, b["ideal"], b["axes"], max_T=64, use_graph=False, kernel="smem").run(eps)[0]
    srv = qs.Server(hbm_budget=1 << 30, max_slots=4, mode="tiled")
    reqs = W.serving_requests(6, m_lo=10, m_hi=14, len_lo=20, len_hi=40)
    for r in reqs:
        cc = W.request_circuit(r)
        srv.submit(r["M"], cc["ideal"], cc["noisy"])
    done = []
    while len(done) < len(reqs):
        done += srv.poll(16, wait_ms=100)
    srv.close()
    out["served"] = sorted((d["id"], d["F"], d["norm"]) for d in done)
    return out


def test_allocator_hook_routes_every_allocation():
    import torch
    lib = qs.load_library()
    ref = _run_all(lib)
    cnt = Counting()
    qs.set_allocator(cnt.alloc, cnt.free)
    try:
        got = _run_all(lib)
    finally:
        qs.set_allocator(None, None)
    torch.cuda.synchronize()
    # states (amplitudes + scratch), plan tables, probabilities staging,
    # trajectory workspaces and tables, served states, slot scratch
    assert cnt.n_alloc >= 20, cnt.n_alloc
    assert cnt.n_free == cnt.n_alloc and not cnt.live, (cnt.n_alloc, cnt.n_free, cnt.live)
    assert len(cnt.streams) >= 2  # the server's slot streams as well as the default stream
    for k in ref:
        if k == "served":
            assert got[k] == ref[k]
        else:
            assert np.array_equal(np.asarray(got[k]), np.asarray(ref[k])), k


def test_allocator_hook_failure_is_enomem():
    lib = qs.load_library()
    qs.set_allocator(lambda n, s: 0, lambda p, n, s: None)
    try:
        h = ctypes.c_void_p()
        assert lib.qsim_alloc(10, qs.QSIM_C64, ctypes.byref(h)) == qs.QSIM_ENOMEM
    finally:
        qs.set_allocator(None, None)
    h = ctypes.c_void_p()
    qs._check(lib.qsim_alloc(10, qs.QSIM_C64, ctypes.byref(h)))
    lib.qsim_free(h)
