"""GB300 error-injecting state-vector simulator (Obenland & Despain, quant-ph/9804039).

A thin ctypes binding of the C ABI in ``include/qsim.h``: the same entry
points, argument marshalling only.  Every step of the simulation runs in the
library's CUDA kernels (``_lib/libqsim.so``, built for sm_103a by
``build.py``).  PyTorch provides device memory and streams: a ``State`` keeps
its amplitudes in a torch tensor on the GPU and runs on a torch stream.

Importing this package fails loudly when the library is missing; there is no
CPU path.
"""

from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB_PATH = _build.LIB

QSIM_OK = 0
QSIM_EINVAL = -1
QSIM_ENOMEM = -2
QSIM_ECUDA = -3
QSIM_ETIMEOUT = -4
QSIM_EBUSY = -5
QSIM_EUNSUPPORTED = -6
QSIM_C64 = 0
QSIM_C128 = 1
MODE_AUTO, MODE_UNFUSED, MODE_TILED, MODE_FUSED = 0, 1, 2, 3
MAX_QUBITS = 34

_MODES = {"auto": MODE_AUTO, "unfused": MODE_UNFUSED, "tiled": MODE_TILED, "fused": MODE_FUSED}


class QsimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"qsim error {code}: {msg}")
        self.code = code


class Opts(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("fuse_k", ctypes.c_int32), ("tile_bits", ctypes.c_int32),
                ("use_graph", ctypes.c_int32), ("specialize", ctypes.c_int32), ("wait_us", ctypes.c_int32),
                ("subspace", ctypes.c_int32)]


class PlanStats(ctypes.Structure):
    _fields_ = [("n_gates", ctypes.c_int64), ("n_passes", ctypes.c_int64), ("n_launches", ctypes.c_int64),
                ("mode", ctypes.c_int32), ("tile_bits", ctypes.c_int32), ("fuse_k", ctypes.c_int32),
                ("n_blocks", ctypes.c_int32), ("algo_bytes", ctypes.c_double), ("amp_updates", ctypes.c_double),
                ("table_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class TrajOpts(ctypes.Structure):
    _fields_ = [("fuse_k", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_uint64), ("max_slots", ctypes.c_int32), ("mode", ctypes.c_int32)]


class RequestResult(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("status", ctypes.c_int32), ("M", ctypes.c_int32),
                ("n_gates", ctypes.c_int32), ("pad", ctypes.c_int32), ("F", ctypes.c_double),
                ("norm", ctypes.c_double), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class ServerStats(ctypes.Structure):
    _fields_ = [("n_submitted", ctypes.c_uint64), ("n_completed", ctypes.c_uint64), ("n_pending", ctypes.c_uint64),
                ("bytes_in_use", ctypes.c_uint64), ("peak_bytes", ctypes.c_uint64), ("max_active", ctypes.c_int32),
                ("pad", ctypes.c_int32), ("now", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


_vp = ctypes.c_void_p
_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)

# (name, restype, argtypes) for every function of include/qsim.h
SIGNATURES = [
    ("qsim_alloc", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)]),
    ("qsim_wrap", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(_vp)]),
    ("qsim_free", None, [_vp]),
    ("qsim_set_stream", ctypes.c_int, [_vp, _vp]),
    ("qsim_state_info", ctypes.c_int, [_vp, _ip, _ip, ctypes.POINTER(_vp)]),
    ("qsim_reset", ctypes.c_int, [_vp]),
    ("qsim_set_state", ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    ("qsim_set_state_async", ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    ("qsim_get_state", ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    ("qsim_copy_state", ctypes.c_int, [_vp, _vp]),
    ("qsim_apply_gate", ctypes.c_int, [_vp, _dp, ctypes.c_int, _ip, ctypes.c_int]),
    ("qsim_apply_circuit", ctypes.c_int, [_vp, _vp, ctypes.c_size_t, ctypes.POINTER(Opts)]),
    ("qsim_plan_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t, ctypes.POINTER(Opts),
                                        ctypes.POINTER(_vp)]),
    ("qsim_plan_execute", ctypes.c_int, [_vp, _vp, _vp]),
    ("qsim_plan_stats_get", ctypes.c_int, [_vp, ctypes.POINTER(PlanStats)]),
    ("qsim_plan_describe", ctypes.c_int, [_vp, ctypes.c_char_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    ("qsim_plan_status", ctypes.c_int, [_vp]),
    ("qsim_plan_destroy", None, [_vp]),
    ("qsim_plan_set_timing", ctypes.c_int, [_vp, ctypes.c_int]),
    ("qsim_plan_timing", ctypes.c_int, [_vp, ctypes.c_int64, _dp, _dp, ctypes.POINTER(ctypes.c_int32),
                                        ctypes.POINTER(ctypes.c_int64)]),
    ("qsim_fidelity", ctypes.c_int, [_vp, _vp, _dp, _dp]),
    ("qsim_overlap", ctypes.c_int, [_vp, _vp, _dp]),
    ("qsim_norm", ctypes.c_int, [_vp, _dp]),
    ("qsim_probabilities", ctypes.c_int, [_vp, _vp, ctypes.c_int]),
    ("qsim_fidelity_noalloc", ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _dp, _dp]),
    ("qsim_run_trajectories", ctypes.c_int, [ctypes.c_int, _vp, _dp, ctypes.c_size_t, _dp, ctypes.c_int,
                                             ctypes.POINTER(TrajOpts), _dp, _dp, _dp]),
    ("qsim_traj_plan_create", ctypes.c_int, [ctypes.c_int, _vp, _dp, ctypes.c_size_t, ctypes.c_int,
                                             ctypes.POINTER(TrajOpts), ctypes.POINTER(_vp)]),
    ("qsim_traj_plan_run", ctypes.c_int, [_vp, _dp, ctypes.c_int, _dp, _dp, _dp]),
    ("qsim_traj_plan_info", ctypes.c_int, [_vp, _ip, _ip, _ip]),
    ("qsim_traj_plan_describe", ctypes.c_int, [_vp, ctypes.c_char_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]),
    ("qsim_traj_plan_destroy", None, [_vp]),
    ("qsim_server_create", ctypes.c_int, [ctypes.POINTER(ServerOpts), ctypes.POINTER(_vp)]),
    ("qsim_server_submit", ctypes.c_int, [_vp, ctypes.c_int, _vp, _vp, ctypes.c_size_t,
                                          ctypes.POINTER(ctypes.c_uint64)]),
    ("qsim_server_poll", ctypes.c_int, [_vp, ctypes.POINTER(RequestResult), ctypes.c_int, _ip, ctypes.c_int]),
    ("qsim_server_get_stats", ctypes.c_int, [_vp, ctypes.POINTER(ServerStats)]),
    ("qsim_server_destroy", None, [_vp]),
    ("qsim_set_allocator", ctypes.c_int, [_vp, _vp, _vp]),
    ("qsim_qutrit_apply", ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t, _vp]),
    ("qsim_qutrit_overlap", ctypes.c_int, [_vp, _vp, ctypes.c_int, ctypes.c_int, _vp, _dp]),
    ("qsim_run_decoherence", ctypes.c_int, [_vp, _vp, ctypes.c_size_t, _dp, _dp, ctypes.c_double,
                                            ctypes.POINTER(ctypes.c_int32), _dp]),
    ("qsim_shard_plan_create", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, ctypes.c_size_t,
                                              ctypes.c_int, ctypes.POINTER(_vp)]),
    ("qsim_shard_plan_info", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                            _dp]),
    ("qsim_shard_step", ctypes.c_int, [_vp, ctypes.c_int64, _ip, ctypes.POINTER(ctypes.c_int64), _ip, _ip]),
    ("qsim_shard_step_gates", ctypes.c_int, [_vp, ctypes.c_int64, _vp, ctypes.c_size_t]),
    ("qsim_shard_plan_destroy", None, [_vp]),
    ("qsim_tune_set_cache", ctypes.c_int, [ctypes.c_char_p]),
    ("qsim_tune_rates", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_char_p, ctypes.c_int64,
                                       ctypes.POINTER(ctypes.c_int64)]),
    ("qsim_last_error", ctypes.c_char_p, []),
    ("qsim_version", ctypes.c_char_p, []),
]

_lib = None


def library_path() -> str:
    return _LIB_PATH


def load_library(build_if_missing: bool = True):
    """Load libqsim.so (building it with nvcc first when it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing and not _build.up_to_date():
        _build.build()
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"the CUDA library {_LIB_PATH} is missing; run build.py (nvcc, sm_103a)")
    lib = ctypes.CDLL(_LIB_PATH)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    if not os.environ.get("QSIM_TUNE_CACHE"):
        lib.qsim_tune_set_cache(DEFAULT_TUNE_CACHE.encode())
    return lib


# the tuning cache next to the built library (ignored by version control)
DEFAULT_TUNE_CACHE = os.path.join(os.path.dirname(_LIB_PATH), "qsim_tune.json")


def set_tune_cache(path):
    """qsim_tune_set_cache: the JSON file of measured rates and timed
    trajectory configurations (None: memory only)."""
    _check(load_library().qsim_tune_set_cache(None if path is None else str(path).encode()))


def tune_rates(prec="c64", specialize=True) -> dict:
    """The measured rates QSIM_MODE_AUTO uses (qsim_tune_rates)."""
    import json
    lib = load_library()
    n = ctypes.c_int64(0)
    buf = ctypes.create_string_buffer(4096)  # one call: a second one could read the cache and differ
    _check(lib.qsim_tune_rates(_prec(prec), int(bool(specialize)), buf, len(buf), ctypes.byref(n)))
    assert n.value <= len(buf)
    return json.loads(buf.value.decode())


def _check(rc: int):
    if rc != QSIM_OK:
        raise QsimError(rc, _lib.qsim_last_error().decode())


# qsim_gate of include/qsim.h: U[8] doubles, int32 target, ncontrols, controls[2]
GATE_DTYPE = np.dtype(
    [("U", "<f8", (8,)), ("target", "<i4"), ("ncontrols", "<i4"), ("controls", "<i4", (2,))]
)
assert GATE_DTYPE.itemsize == 80


def _records(gates) -> np.ndarray:
    return np.ascontiguousarray(gates, dtype=GATE_DTYPE)


def _opts(mode="auto", fuse_k=0, tile_bits=0, use_graph=False, specialize=False, wait_us=0, subspace=False) -> Opts:
    m = _MODES[mode] if isinstance(mode, str) else int(mode)
    return Opts(m, int(fuse_k), int(tile_bits), int(bool(use_graph)), int(bool(specialize)), int(wait_us),
                int(bool(subspace)))


def _torch():
    import torch
    return torch


def _prec(prec) -> int:
    if prec in ("c64", "complex64", QSIM_C64):
        return QSIM_C64
    if prec in ("c128", "complex128", QSIM_C128):
        return QSIM_C128
    raise ValueError(f"unknown precision {prec!r}")


class State:
    """A 2^M-amplitude state vector on the GPU (amplitudes in a torch tensor)."""

    def __init__(self, M: int, prec="c64", device=None, stream=None, zero=True):
        torch = _torch()
        lib = load_library()
        self.M = int(M)
        self.prec = _prec(prec)
        dtype = torch.complex64 if self.prec == QSIM_C64 else torch.complex128
        device = torch.device(device if device is not None else "cuda")
        self.tensor = torch.empty(1 << self.M, dtype=dtype, device=device)
        h = _vp()
        _check(lib.qsim_wrap(_vp(self.tensor.data_ptr()), self.M, self.prec, ctypes.byref(h)))
        self._h = h
        self.set_stream(stream if stream is not None else torch.cuda.current_stream(device))
        if zero:
            self.reset()

    @property
    def handle(self):
        return self._h

    def set_stream(self, stream):
        self.stream = stream
        _check(_lib.qsim_set_stream(self._h, _vp(stream.cuda_stream)))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.qsim_free(h)
            self._h = None

    def reset(self):
        _check(_lib.qsim_reset(self._h))
        return self

    def set(self, amps):
        """Copy amplitudes in (numpy array on the host, or a CUDA tensor)."""
        torch = _torch()
        if isinstance(amps, torch.Tensor) and amps.is_cuda:
            a = amps.to(self.tensor.dtype).contiguous()
            _check(_lib.qsim_set_state(self._h, _vp(a.data_ptr()), 1))
            self.stream.synchronize()
        else:
            a = np.ascontiguousarray(amps, dtype=np.complex64 if self.prec == QSIM_C64 else np.complex128)
            assert a.size == (1 << self.M)
            _check(_lib.qsim_set_state(self._h, _vp(a.ctypes.data), 0))
        return self

    def set_async(self, amps):
        """Queue a copy in from a pinned host tensor (or a CUDA tensor) on this
        state's stream and return (qsim_set_state_async); `amps` must stay
        unchanged until later work that waits for this state."""
        torch = _torch()
        assert isinstance(amps, torch.Tensor) and amps.dtype == self.tensor.dtype and amps.is_contiguous()
        assert amps.numel() == (1 << self.M) and (amps.is_cuda or amps.is_pinned())
        _check(_lib.qsim_set_state_async(self._h, _vp(amps.data_ptr()), 1 if amps.is_cuda else 0))
        return self

    def get(self) -> np.ndarray:
        out = np.empty(1 << self.M, dtype=np.complex64 if self.prec == QSIM_C64 else np.complex128)
        _check(_lib.qsim_get_state(self._h, _vp(out.ctypes.data), 0))
        return out

    def copy_from(self, other: "State"):
        _check(_lib.qsim_copy_state(self._h, other._h))
        return self

    def apply_gate(self, U, target: int, controls=()):
        Uf = np.ascontiguousarray(np.asarray(U, dtype=np.complex128).reshape(4).view(np.float64))
        ctl = np.zeros(2, dtype=np.int32)
        ctl[: len(controls)] = controls
        _check(_lib.qsim_apply_gate(self._h, Uf.ctypes.data_as(_dp), int(target), ctl.ctypes.data_as(_ip),
                                    len(controls)))
        return self

    def apply_circuit(self, gates, mode="auto", fuse_k=0, tile_bits=0, use_graph=False):
        g = _records(gates)
        o = _opts(mode, fuse_k, tile_bits, use_graph)
        _check(_lib.qsim_apply_circuit(self._h, _vp(g.ctypes.data), len(g), ctypes.byref(o)))
        return self

    def norm(self) -> float:
        v = ctypes.c_double()
        _check(_lib.qsim_norm(self._h, ctypes.byref(v)))
        return v.value

    def probabilities(self, on_device: bool = False):
        if on_device:
            torch = _torch()
            dt = torch.float32 if self.prec == QSIM_C64 else torch.float64
            out = torch.empty(1 << self.M, dtype=dt, device=self.tensor.device)
            _check(_lib.qsim_probabilities(self._h, _vp(out.data_ptr()), 1))
            return out
        out = np.empty(1 << self.M, dtype=np.float32 if self.prec == QSIM_C64 else np.float64)
        _check(_lib.qsim_probabilities(self._h, _vp(out.ctypes.data), 0))
        return out


def fidelity(ideal: State, noisy: State):
    """(F, norm_noisy) with F = |<ideal|noisy>|^2."""
    F = ctypes.c_double()
    n = ctypes.c_double()
    _check(_lib.qsim_fidelity(ideal._h, noisy._h, ctypes.byref(F), ctypes.byref(n)))
    return F.value, n.value


class Plan:
    """A compiled circuit for states of M qubits (qsim_plan_create)."""

    def __init__(self, M: int, gates, prec="c64", mode="auto", fuse_k=0, tile_bits=0, use_graph=False,
                 specialize=False, wait_us=0, subspace=False):
        lib = load_library()
        self.M = int(M)
        self.prec = _prec(prec)
        g = _records(gates)
        self.n_gates = len(g)
        o = _opts(mode, fuse_k, tile_bits, use_graph, specialize, wait_us, subspace)
        h = _vp()
        _check(lib.qsim_plan_create(self.M, self.prec, _vp(g.ctypes.data), len(g), ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def execute(self, dst: State, src: State | None = None):
        _check(_lib.qsim_plan_execute(self._h, dst._h, src._h if src is not None else None))
        return dst

    def status(self):
        """Raise if a kernel of this plan gave up a bounded wait (waits for the device)."""
        _check(_lib.qsim_plan_status(self._h))

    def set_timing(self, enable: bool = True):
        _check(_lib.qsim_plan_set_timing(self._h, int(bool(enable))))

    def timing(self):
        """(ms[j] summed over timed executions, bytes[j], kind[j], executions) per launch j."""
        n = int(self.stats()["n_launches"])
        ms = np.zeros(n)
        by = np.zeros(n)
        kd = np.zeros(n, dtype=np.int32)
        ex = ctypes.c_int64()
        _check(_lib.qsim_plan_timing(self._h, n, ms.ctypes.data_as(_dp), by.ctypes.data_as(_dp),
                                     kd.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), ctypes.byref(ex)))
        return ms, by, kd, ex.value

    def stats(self) -> dict:
        s = PlanStats()
        _check(_lib.qsim_plan_stats_get(self._h, ctypes.byref(s)))
        return s.as_dict()

    def describe(self) -> str:
        """Text description of the passes, rounds and op kinds."""
        n = ctypes.c_int64(0)
        _check(_lib.qsim_plan_describe(self._h, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(int(n.value))
        _check(_lib.qsim_plan_describe(self._h, buf, n.value, ctypes.byref(n)))
        return buf.value.decode()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.qsim_plan_destroy(h)
            self._h = None


class TrajPlan:
    """A circuit compiled for batches of error trajectories (qsim_traj_plan_create)."""

    def __init__(self, M: int, gates, err_axis, max_T: int, use_graph: bool = True, kernel: str = "auto"):
        lib = load_library()
        g = _records(gates)
        ax = np.ascontiguousarray(err_axis, dtype=np.float64)
        assert ax.shape == (len(g), 3)
        self.M, self.n, self.max_T = int(M), len(g), int(max_T)
        o = TrajOpts(0, int(bool(use_graph)), {"auto": 0, "smem": 1, "register": 2}[kernel], 0)
        h = _vp()
        _check(lib.qsim_traj_plan_create(self.M, _vp(g.ctypes.data), ax.ctypes.data_as(_dp), len(g), self.max_T,
                                         ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def run(self, eps):
        e = np.ascontiguousarray(eps, dtype=np.float64)
        T = e.shape[0]
        assert e.shape[1] == self.n
        F = np.zeros(T)
        mean, var = ctypes.c_double(), ctypes.c_double()
        _check(_lib.qsim_traj_plan_run(self._h, e.ctypes.data_as(_dp), T, F.ctypes.data_as(_dp), ctypes.byref(mean),
                                       ctypes.byref(var)))
        return F, mean.value, var.value

    def info(self) -> dict:
        tb, npass, grid = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        _check(_lib.qsim_traj_plan_info(self._h, ctypes.byref(tb), ctypes.byref(npass), ctypes.byref(grid)))
        return {"tile_bits": tb.value, "n_passes": npass.value, "grid": grid.value}

    def describe(self) -> str:
        """The chosen kernel and the autotuner's candidate timings."""
        n = ctypes.c_int64(0)
        _check(_lib.qsim_traj_plan_describe(self._h, None, 0, ctypes.byref(n)))
        buf = ctypes.create_string_buffer(int(n.value))
        _check(_lib.qsim_traj_plan_describe(self._h, buf, n.value, ctypes.byref(n)))
        return buf.value.decode()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.qsim_traj_plan_destroy(h)
            self._h = None


class Server:
    """Continuous-batching request loop (qsim_server_*)."""

    def __init__(self, hbm_budget: int, max_slots: int = 8, mode="tiled"):
        lib = load_library()
        m = _MODES[mode] if isinstance(mode, str) else int(mode)
        o = ServerOpts(int(hbm_budget), int(max_slots), m)
        h = _vp()
        _check(lib.qsim_server_create(ctypes.byref(o), ctypes.byref(h)))
        self._h = h

    def submit(self, M: int, ideal, noisy) -> int:
        gi, gn = _records(ideal), _records(noisy)
        assert len(gi) == len(gn)
        rid = ctypes.c_uint64()
        _check(_lib.qsim_server_submit(self._h, int(M), _vp(gi.ctypes.data), _vp(gn.ctypes.data), len(gi),
                                       ctypes.byref(rid)))
        return rid.value

    def poll(self, max_results: int = 256, wait_ms: int = 0):
        buf = (RequestResult * max_results)()
        n = ctypes.c_int()
        _check(_lib.qsim_server_poll(self._h, buf, max_results, ctypes.byref(n), int(wait_ms)))
        return [buf[i].as_dict() for i in range(n.value)]

    def stats(self) -> dict:
        s = ServerStats()
        _check(_lib.qsim_server_get_stats(self._h, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and _lib is not None:
            _lib.qsim_server_destroy(h)
            self._h = None

    def __del__(self):
        self.close()


def run_trajectories(M: int, gates, err_axis, eps, fuse_k: int = 0, use_graph: bool = False):
    """Fidelities of T error trajectories of one circuit: (F[T], mean, var)."""
    lib = load_library()
    g = _records(gates)
    ax = np.ascontiguousarray(err_axis, dtype=np.float64)
    e = np.ascontiguousarray(eps, dtype=np.float64)
    T = e.shape[0]
    assert e.shape[1] == len(g) and ax.shape == (len(g), 3)
    F = np.zeros(T)
    mean = ctypes.c_double()
    var = ctypes.c_double()
    o = TrajOpts(int(fuse_k), int(bool(use_graph)), 0, 0)
    _check(lib.qsim_run_trajectories(int(M), _vp(g.ctypes.data), ax.ctypes.data_as(_dp), len(g),
                                     e.ctypes.data_as(_dp), T, ctypes.byref(o), F.ctypes.data_as(_dp),
                                     ctypes.byref(mean), ctypes.byref(var)))
    return F, mean.value, var.value


def version() -> str:
    return load_library().qsim_version().decode()


# qsim_gate3 of include/qsim.h: U[18] doubles, int32 target, ncontrols, controls[2], levels[2]
GATE3_DTYPE = np.dtype(
    [("U", "<f8", (18,)), ("target", "<i4"), ("ncontrols", "<i4"), ("controls", "<i4", (2,)),
     ("levels", "<i4", (2,))]
)
assert GATE3_DTYPE.itemsize == 168


class QutritState:
    """3^M amplitudes of M three-level particles on the GPU (a torch tensor);
    qsim_qutrit_apply / qsim_qutrit_overlap work on its device pointer."""

    def __init__(self, M: int, prec="c64", device=None, stream=None):
        torch = _torch()
        load_library()
        self.M = int(M)
        self.prec = _prec(prec)
        dtype = torch.complex64 if self.prec == QSIM_C64 else torch.complex128
        self.tensor = torch.zeros(3 ** self.M, dtype=dtype, device=device if device is not None else "cuda")
        self.tensor[0] = 1.0
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.tensor.device)

    def set(self, amps):
        torch = _torch()
        a = np.ascontiguousarray(amps, dtype=np.complex64 if self.prec == QSIM_C64 else np.complex128)
        assert a.size == 3 ** self.M
        self.tensor.copy_(torch.from_numpy(a))
        return self

    def get(self) -> np.ndarray:
        with _torch().cuda.stream(self.stream):
            return self.tensor.cpu().numpy()

    def apply(self, gates3):
        g = np.ascontiguousarray(gates3, dtype=GATE3_DTYPE)
        _check(_lib.qsim_qutrit_apply(_vp(self.tensor.data_ptr()), self.M, self.prec, _vp(g.ctypes.data), len(g),
                                      _vp(self.stream.cuda_stream)))
        return self


def qutrit_overlap(ideal: QutritState | None, noisy: QutritState):
    """(norm of noisy, Re, Im of <ideal|noisy>) over 3^M amplitudes."""
    out = np.zeros(3)
    _check(load_library().qsim_qutrit_overlap(_vp(ideal.tensor.data_ptr()) if ideal is not None else None,
                                              _vp(noisy.tensor.data_ptr()), noisy.M, noisy.prec,
                                              _vp(noisy.stream.cuda_stream), out.ctypes.data_as(_dp)))
    return out


def run_decoherence(state: State, gates, delta, r, gamma: float):
    """qsim_run_decoherence on `state` in place: returns (jumps[n], p[n])."""
    lib = load_library()
    g = _records(gates)
    d = np.ascontiguousarray(delta, dtype=np.float64)
    rr = np.ascontiguousarray(r, dtype=np.float64)
    assert d.size == len(g) and rr.size == len(g)
    jumps = np.zeros(len(g), dtype=np.int32)
    p = np.zeros(len(g))
    _check(lib.qsim_run_decoherence(state.handle, _vp(g.ctypes.data), len(g), d.ctypes.data_as(_dp),
                                    rr.ctypes.data_as(_dp), float(gamma),
                                    jumps.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), p.ctypes.data_as(_dp)))
    return jumps, p


# qsim_device_alloc_fn / qsim_device_free_fn of include/qsim.h
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_hooks = None  # the registered callbacks, kept alive while the library may call them


def set_allocator(alloc=None, free=None):
    """qsim_set_allocator with Python callables: alloc(bytes, stream) -> device
    address (int, 0 on failure) and free(ptr, bytes, stream); None, None
    restores the CUDA runtime.  Objects created under a pair keep calling it
    until they are released, so the callables are kept alive here."""
    global _hooks
    lib = load_library()
    if alloc is None and free is None:
        _check(lib.qsim_set_allocator(None, None, None))
        return

    def _a(nbytes, stream, ctx):
        try:
            return int(alloc(int(nbytes), int(stream or 0))) or None
        except Exception:  # reported to the library as an allocation failure
            return None

    def _f(ptr, nbytes, stream, ctx):
        free(int(ptr), int(nbytes), int(stream or 0))

    ca, cf = ALLOC_FN(_a), FREE_FN(_f)
    _check(lib.qsim_set_allocator(ctypes.cast(ca, _vp), ctypes.cast(cf, _vp), None))
    _hooks = (_hooks or ()) + ((ca, cf),)  # earlier pairs stay alive for the objects made under them


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching
    allocator (torch.cuda.caching_allocator_alloc / _delete), so that its
    states, plan tables and workspaces share torch's memory pool."""
    torch = _torch()

    def alloc(nbytes, stream):
        return torch.cuda.caching_allocator_alloc(nbytes, stream=stream)

    def free(ptr, nbytes, stream):
        torch.cuda.caching_allocator_delete(ptr)

    set_allocator(alloc, free)
