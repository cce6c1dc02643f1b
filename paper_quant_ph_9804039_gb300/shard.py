"""One state vector split over ranks (Section 3.1; Section 3.3, Figure 8).

The library plans, for each rank, the local gate steps and the
redistributions (``qsim_shard_plan_*``); this module marshals those records
and carries the chunks of a redistribution between ranks with
``torch.distributed`` point-to-point calls (NCCL between GPUs, gloo between
CPU processes).  The local gate steps run as the library's plans on the
rank's shard, a state of ``L = M - n_global`` qubits.  Fidelity and norm of
a split state are the sum over ranks of ``qsim_overlap`` (an all-reduce of
three doubles, EQ 3's global sum).
"""

from __future__ import annotations

import ctypes

import numpy as np

from . import GATE_DTYPE, Plan, State, _check, _dp, _records, _vp, load_library


class ShardPlan:
    """qsim_shard_plan_create for one rank: a list of steps, each
    ("local", gate records on the L local qubits) or ("exchange", rank bits)."""

    def __init__(self, M: int, n_global: int, rank: int, gates, restore_order: bool = True):
        lib = load_library()
        g = _records(gates)
        h = _vp()
        _check(lib.qsim_shard_plan_create(int(M), int(n_global), int(rank), _vp(g.ctypes.data), len(g),
                                          int(bool(restore_order)), ctypes.byref(h)))
        self._h = h
        self.M, self.n_global, self.rank = int(M), int(n_global), int(rank)
        self.L = self.M - self.n_global
        ns, nx, mv = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        _check(lib.qsim_shard_plan_info(h, ctypes.byref(ns), ctypes.byref(nx), ctypes.byref(mv)))
        self.n_exchanges, self.moved = int(nx.value), float(mv.value)
        self.steps = []
        for i in range(ns.value):
            kind, ng, npairs = ctypes.c_int(), ctypes.c_int64(), ctypes.c_int()
            bits = (ctypes.c_int * max(1, self.n_global))()
            _check(lib.qsim_shard_step(h, i, ctypes.byref(kind), ctypes.byref(ng), ctypes.byref(npairs), bits))
            if kind.value == 0:
                out = np.zeros(ng.value, dtype=GATE_DTYPE)
                _check(lib.qsim_shard_step_gates(h, i, _vp(out.ctypes.data), ng.value))
                self.steps.append(("local", out))
            else:
                self.steps.append(("exchange", [int(bits[k]) for k in range(npairs.value)]))

    def __del__(self):
        h = getattr(self, "_h", None)
        lib = load_library()
        if h is not None:
            lib.qsim_shard_plan_destroy(h)
            self._h = None


def chunk_schedule(rank: int, L: int, gbits):
    """The chunk swaps of one redistribution for this rank, in the order every
    rank follows (round d pairs the ranks whose pair bits differ by d, so no
    exchange waits on another): (chunk index, partner rank, first amplitude,
    amplitudes)."""
    nc = len(gbits)
    C = 1 << (L - nc)
    own = sum(((rank >> j) & 1) << i for i, j in enumerate(gbits))
    out = []
    for d in range(1, 1 << nc):
        b = own ^ d
        partner = rank
        for i, j in enumerate(gbits):
            partner = (partner & ~(1 << j)) | (((b >> i) & 1) << j)
        out.append((b, partner, b * C, C))
    return out


def exchange_chunks(amps, rank: int, L: int, gbits, group=None):
    """One redistribution on this rank's shard (a 1-D complex torch tensor of
    2^L amplitudes, on the device for NCCL or on the host for gloo): for each
    round, send the chunk to the partner and receive the partner's chunk into
    its place."""
    import torch
    import torch.distributed as dist
    C = 1 << (L - len(gbits))
    tmp = torch.empty(C, dtype=amps.dtype, device=amps.device)
    for _, partner, off, n in chunk_schedule(rank, L, gbits):
        chunk = amps[off:off + n]
        reqs = [dist.isend(torch.view_as_real(chunk).contiguous(), partner, group=group),
                dist.irecv(torch.view_as_real(tmp), partner, group=group)]
        for r in reqs:
            r.wait()
        chunk.copy_(tmp)


class ShardedCircuit:
    """A circuit for this rank's shard: the library's plans (L qubits) for the
    local steps, made once; run() applies them to a State of L qubits and
    carries the redistributions over torch.distributed."""

    def __init__(self, M: int, n_global: int, rank: int, gates, mode="auto", specialize=False,
                 restore_order: bool = True):
        self.plan = ShardPlan(M, n_global, rank, gates, restore_order)
        self.L = self.plan.L
        self.rank = rank
        self.local = [Plan(self.L, g, mode=mode, specialize=specialize) if kind == "local" and len(g) else None
                      for kind, g in self.plan.steps]

    def run(self, state: State, group=None):
        assert state.M == self.L
        for (kind, arg), plan in zip(self.plan.steps, self.local):
            if kind == "local":
                if plan is not None:
                    plan.execute(state)
            else:
                state.stream.synchronize()
                exchange_chunks(state.tensor, self.rank, self.L, arg, group)
        return state


def overlap(ideal: State, noisy: State):
    """qsim_overlap: (norm of noisy, Re, Im of <ideal|noisy>) over this shard."""
    out = np.zeros(3)
    _check(load_library().qsim_overlap(ideal.handle, noisy.handle, out.ctypes.data_as(_dp)))
    return out


def sharded_fidelity(ideal: State, noisy: State, group=None):
    """F and the norm of a split state: the shards' three sums all-reduced."""
    import torch
    import torch.distributed as dist
    s = torch.tensor(overlap(ideal, noisy), dtype=torch.float64,
                     device=ideal.tensor.device if dist.get_backend(group) == "nccl" else "cpu")
    dist.all_reduce(s, group=group)
    n, re, im = (float(v) for v in s.cpu())
    return re * re + im * im, n
