#!/usr/bin/env python
"""Benchmark of the error-injecting state-vector simulator on GB300.

Workload (default): the 33-qubit brickwork, complex64, both state vectors
resident (2 x 64 GiB): 24 layers of a Haar-random SU(2) on every qubit and
CNOTs on alternating neighbour pairs, a Toffoli on a random triple after
every 4th layer (1182 gates), every gate over-rotated by a Gaussian angle
(sigma = 1e-3).  One step = both states reset to |0...0>, the error-free and
the noisy circuit applied in place, then the fidelity |<ideal|noisy>|^2 and
the noisy norm read back to the host.  The plans are made in the library's
AUTO mode (the execution form is chosen when the plan is made); the fused
tensor-core, tiled and one-gate-per-launch forms are each timed beside it.

Extra keys: the M=28 quantum FFT (the tiled register passes' workload), one
dense gate per launch at M=30, batched error trajectories (M=16, T=4096),
the served request stream, and the CPU oracle on a bounded sample.

metric: amplitude-updates/s = (logical gates applied) * 2^M / second, summed
over ranks.  Per-launch CUDA events (recorded by the library on the launching
stream inside the timed region) give the dominant kernel's roofline figures.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun (N > 1) every rank runs an independent replica (no collective
on the data path: the per-rank work is fixed, weak scaling).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOADS = {
    # 33-qubit brickwork (24 layers, Haar SU(2) + CNOT, Toffoli every 4th layer,
    # over-rotation sigma=1e-3) from |0...0>, both states resident (128 GiB)
    "brickwork-m33-c64": dict(M=33, sigma=1e-3, circuit="brickwork"),
    # the same circuit at M=26 (512 MiB per state, > L2) for ncu captures
    "brickwork-m26-c64": dict(M=26, sigma=1e-3, circuit="brickwork"),
    # quantum FFT on M=28 qubits from a random normalised input
    "qft-m28-c64": dict(M=28, sigma=1e-4, circuit="qft"),
    # smaller case of the same circuit for ncu captures (512 MiB per state, > L2)
    "qft-m26-c64": dict(M=26, sigma=1e-4, circuit="qft"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 4 for the 33-qubit brickwork, 40 otherwise)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="brickwork-m33-c64", choices=sorted(WORKLOADS))
    ap.add_argument("--mode", default=None, choices=["auto", "tiled", "unfused", "fused"],
                    help="execution form of the headline (default: auto for the brickwork, tiled for the QFT)")
    ap.add_argument("--modes", default="fused,tiled,unfused",
                    help="brickwork: the forms timed beside the headline")
    ap.add_argument("--tile-bits", type=int, default=0)
    ap.add_argument("--no-specialize", action="store_true",
                    help="keep the general register kernel instead of one generated kernel per tile pass")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-unfused", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-qft", action="store_true", help="brickwork: skip the M=28 quantum-FFT key")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the single-gate, batched-trajectory and serving measurements")
    ap.add_argument("--serve-requests", type=int, default=2000)
    a = ap.parse_args()
    if a.steps is None:
        a.steps = 4 if WORKLOADS[a.workload]["M"] >= 30 else 40
    if a.mode is None:
        a.mode = "auto" if WORKLOADS[a.workload]["circuit"] == "brickwork" else "tiled"
    return a


# ------------------------------------------------------------------ ranks ---
def dist_setup():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world, local, backend="nccl"):
    """One process per GPU; the process group only carries the barrier and the
    max-over-ranks of the timings (no collective on the data path).  The gloo
    backend runs the same host logic on CPU ranks."""
    import torch
    if backend == "nccl":
        torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        if backend == "nccl":
            dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        else:
            dist.init_process_group(backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v: float, world: int) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job rate of independent replicas: the units all ranks processed
    over the slowest rank's time (weak scaling)."""
    return units_per_rank * world / (ms_max / 1e3)


# ----------------------------------------------------------------- clocks ---
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.start = 0

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts once nvidia-smi is sampling: earlier lines
            # are not counted
            t0 = time.time()
            while not self.lines and self.proc.poll() is None and time.time() - t0 < 5.0:
                time.sleep(0.01)
            self.start = len(self.lines)
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines[self.start:] or self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = float(parts[1])
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# GB300: 152 SMs, 128 FP32 lanes per SM, one FMA (2 flop) per lane per clock.
GB300_SMS, FP32_LANES_PER_SM = 152, 128


def derived_fp32_peak(sm_mhz: float) -> float:
    """FP32 FMA peak in flop/s derived from the unit counts and an SM clock."""
    return GB300_SMS * FP32_LANES_PER_SM * 2.0 * sm_mhz * 1e6


# plan timing kinds (qsim_plan_timing) -> kernel names
KIND_NAME = {0: "k_gate (one gate per launch)", 1: "k_tile_pass", 2: "k_fused_tc", 3: "k_permute",
             4: "k_tile_reg", 5: "qs_pass (specialised register tile pass)", 6: "none (gathered permutation)"}
KIND_KEY = {0: "k_gate", 1: "k_tile_pass", 2: "k_fused_tc", 3: "k_permute", 4: "k_tile_reg", 5: "qs_pass"}
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "dram_traffic.txt")


def _src_sha16(paths) -> str:
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str, M: int):
    """DRAM bytes (read + write) per launch of `kernel` from the committed ncu
    summary, scaled from the captured state size to 2^M amplitudes (each of
    these passes moves every amplitude once, so its traffic is proportional to
    2^M).  None when there is no capture or the kernel's source changed since
    it was taken.  Returns (bytes or None, where from, tensor-pipe % or None)."""
    if not os.path.exists(PROFILE_TRAFFIC):
        return None, "no ncu capture", None
    with open(PROFILE_TRAFFIC) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            fld = line.split()
            # kernel workload M launches dram_bytes_per_launch tensor_pipe_pct sources sha16
            if fld[0] != kernel:
                continue
            if _src_sha16(fld[6].split(",")) != fld[7]:
                return None, f"kernel source changed since the ncu capture ({fld[1]})", None
            shift = M - int(fld[2])
            tensor = None if fld[5] == "-" else float(fld[5])
            return float(fld[4]) * 2.0 ** shift, f"ncu {fld[1]}, {fld[3]} launches, scaled by 2^{shift}", tensor
    return None, "no ncu capture", None


def plan_roofline(plans, ms_step, steps, M):
    """Roofline of the dominant kernel of the timed plans from the library's
    per-launch CUDA events (qsim_plan_timing, recorded on the launching
    stream): algorithmic bytes per launch over the average launch time,
    against the measured copy bandwidth."""
    kinds = {}
    launches_step = 0
    bytes_step = 0.0
    per_plan_launches = []
    for p in plans:
        t_ms, t_bytes, t_kind, execs = p.timing()
        nl = int(np.sum(t_kind != 6))  # 6: a permutation gathered by the next pass, no launch
        per_plan_launches.append(nl)
        launches_step += nl
        bytes_step += float(np.sum(t_bytes))
        for j in range(len(t_ms)):
            k = int(t_kind[j])
            if k == 6:
                continue
            d = kinds.setdefault(k, [0.0, 0.0, 0])
            d[0] += t_ms[j]
            d[1] += t_bytes[j] * execs
            d[2] += execs
    top = max(kinds, key=lambda k: kinds[k][0])
    tot_ms, tot_bytes, n_launch = kinds[top]
    peak, peak_src = measured_peaks()
    achieved = tot_bytes / (tot_ms / 1e3) / 1e9
    traffic, t_src, tensor = profiled_traffic(KIND_KEY.get(top, "?"), M)
    roof = {"bound": "hbm", "kernel": KIND_NAME[top], "achieved": round(achieved, 1), "peak": peak,
            "peak_source": peak_src, "unit": "GB/s", "frac": round(achieved / peak, 4),
            "traffic": traffic, "traffic_source": t_src,
            "algo_bytes_per_launch": tot_bytes / max(1, n_launch), "launches_timed": n_launch,
            "avg_launch_ms": round(tot_ms / max(1, n_launch), 4),
            "kernel_share_of_step": round(tot_ms / (ms_step * steps), 4)}
    if top == 2:
        roof["tensor_pipe_active_pct_ncu"] = tensor
    return roof, launches_step, bytes_step, per_plan_launches


# ------------------------------------------------------------ cpu baseline ---
def _host_available_bytes() -> int:
    try:
        return os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_AVPHYS_PAGES")
    except (ValueError, OSError):
        return 0


def oracle_size(M: int) -> int:
    """The largest qubit count <= M whose complex128 state fits in a third of
    the host's free memory (the oracle runs at the workload's own M when it
    fits)."""
    avail = _host_available_bytes()
    m = M
    while m > 20 and (16 << m) * 3 > avail:
        m -= 1
    return m


def oracle_sample(M, gates, x, budget_s: float, min_gates: int = 3, nthreads=None, max_M=None):
    """Time the CPU oracle (all host threads, or nthreads) on the first gates
    of the noisy circuit, at the workload's M if the host has the memory
    (else the largest M that fits, or max_M), for about budget_s seconds after
    one untimed gate (which touches every page of the state).  Returns
    (amp-updates/s, gates applied, seconds, threads, M used)."""
    import oracle
    orc = oracle.Oracle()
    nt = nthreads or oracle.default_threads()
    Ms = oracle_size(M) if max_M is None else min(oracle_size(M), max_M)
    if x is not None and Ms == M:
        psi = x.astype(np.complex128)
    else:
        psi = np.zeros(1 << Ms, dtype=np.complex128)
        psi[0] = 1.0
    gates = gates[[i for i in range(len(gates)) if gates[i]["target"] < Ms
                   and all(c < Ms for c in gates[i]["controls"][: int(gates[i]["ncontrols"])])]]
    orc.apply_circuit(psi, gates[:1], nthreads=nt)
    t0 = time.perf_counter()
    n = 1
    while n < len(gates) and (n < min_gates + 1 or time.perf_counter() - t0 < budget_s):
        orc.apply_circuit(psi, gates[n:n + 1], nthreads=nt)
        n += 1
    dt = time.perf_counter() - t0
    return (n - 1) * float(1 << Ms) / dt, n - 1, dt, nt, Ms


def workload_circuit(wl):
    from workloads import generators as W
    if wl["circuit"] == "brickwork":
        c = W.circuit_c4_brickwork_toffoli(wl["M"], layers=24, sigma=wl["sigma"])
        c["n_logical_gates"] = len(c["ideal"])
        return c, None
    c = W.circuit_c2_qft(wl["M"], sigma=wl["sigma"])
    return c, W.random_state(wl["M"], seed=2)


# ---------------------------------------------------------------- ours ---
def _timed_steps(step, plans, steps, warm, stream, world, local, M):
    """Run `warm` untimed steps, then time exactly `steps` with CUDA events on
    the launching stream (barrier and synchronisation on both sides), with the
    plans' per-launch timing on.  Returns (ms per step, last result, roofline,
    launches per step, algorithmic bytes per step, launches per plan, clocks)."""
    import torch
    out = None
    for _ in range(warm):
        out = step()
    torch.cuda.synchronize()
    for p in plans:
        p.set_timing(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        e0.record(stream)
        for _ in range(steps):
            out = step()
        e1.record(stream)
        torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(e0.elapsed_time(e1) / steps, world)
    roof, launches, bytes_step, per_plan = plan_roofline(plans, ms, steps, M)
    for p in plans:
        p.set_timing(False)
    return ms, out, roof, launches, bytes_step, per_plan, clk.summary()


def run_brickwork(args, rank, world, local):
    """The brickwork from |0...0>: one step = reset both states, the error-free
    and the noisy circuit in place, fidelity and norm read back.  The headline
    uses the plans made in args.mode (AUTO by default); each other form in
    args.modes is timed the same way beside it."""
    import ctypes

    import torch

    import paper_quant_ph_9804039_gb300 as qs

    wl = WORKLOADS[args.workload]
    M = wl["M"]
    c, _ = workload_circuit(wl)
    n = len(c["ideal"])
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    ideal = qs.State(M, device=dev, stream=stream)
    noisy = qs.State(M, device=dev, stream=stream)
    spec = not args.no_specialize
    amp_step = 2.0 * n * float(1 << M)
    mode_names = {qs.MODE_UNFUSED: "unfused", qs.MODE_TILED: "tiled", qs.MODE_FUSED: "fused"}

    def make(mode):
        t = time.perf_counter()
        p_i = qs.Plan(M, c["ideal"], mode=mode, specialize=spec and mode != "unfused")
        p_n = qs.Plan(M, c["noisy"], mode=mode, specialize=spec and mode != "unfused")
        return p_i, p_n, time.perf_counter() - t

    def stepper(p_i, p_n):
        def step():
            ideal.reset()
            noisy.reset()
            p_i.execute(ideal)
            p_n.execute(noisy)
            return qs.fidelity(ideal, noisy)
        return step

    p_i, p_n, t_plan = make(args.mode)
    head = mode_names[p_n.stats()["mode"]]
    auto_line = next((ln for ln in p_n.describe().splitlines() if ln.startswith("auto:")), None)
    ms, (F, nrm), roof, launches, bytes_step, per_plan, clocks = _timed_steps(
        stepper(p_i, p_n), [p_i, p_n], args.steps, args.warmup, stream, world, local, M)
    value = job_throughput(amp_step, world, ms)
    st = p_n.stats()
    modes = {head: {"amp_updates_per_s": value, "ms_per_step": ms, "steps": args.steps, "warmup": args.warmup,
                    "passes_per_circuit": per_plan[1], "blocks_per_circuit": st["n_blocks"],
                    "specialised_passes": "specialised" in p_n.describe(), "plan_create_s": round(t_plan, 3),
                    "roofline": roof, "F": F, "norm": nrm}}
    result = {
        "metric": "amplitude-updates/s", "value": value, "unit": "amp-updates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "complex64", "data": "synthetic",
        "config": {"workload": args.workload, "M": M, "circuit": "brickwork+toffoli", "layers": 24,
                   "sigma": wl["sigma"], "gates_per_circuit": n, "circuits_per_step": 2, "input": "|0...0>",
                   "mode": args.mode, "executed_as": head, "auto_choice": auto_line,
                   "l2": f"inputs larger than L2 ({(8 << M) >> 20} MiB per state)",
                   "parallelism": f"replicas{world}"},
        "roofline": roof,
        "fidelity": F, "norm": nrm,
        "hbm_gbs_step": (bytes_step + 2 * 8 * float(1 << M) + 16 * float(1 << M)) / (ms / 1e3) / 1e9,
        "clocks": clocks,
    }
    # launches per step: the plans' own + 2 resets + the reduction's 2 kernels
    result["gpu_launches"] = int((launches + 4) * args.steps)

    # end to end through the C ABI: host gate records in, F and the norm out.
    # Each step resets both states, plans and applies both circuits from the
    # host records (qsim_apply_circuit: the plan's tables are built on the
    # host and copied to the device inside the call) and reads F back.
    if not args.no_e2e:
        lib = qs.load_library()
        gi = np.ascontiguousarray(c["ideal"], dtype=qs.GATE_DTYPE)
        gn = np.ascontiguousarray(c["noisy"], dtype=qs.GATE_DTYPE)
        o = qs._opts("auto", 0, 0, False, False)
        Fv, Nv = ctypes.c_double(), ctypes.c_double()

        def e2e_step():
            qs._check(lib.qsim_reset(ideal.handle))
            qs._check(lib.qsim_reset(noisy.handle))
            qs._check(lib.qsim_apply_circuit(ideal.handle, gi.ctypes.data_as(ctypes.c_void_p), len(gi),
                                             ctypes.byref(o)))
            qs._check(lib.qsim_apply_circuit(noisy.handle, gn.ctypes.data_as(ctypes.c_void_p), len(gn),
                                             ctypes.byref(o)))
            qs._check(lib.qsim_fidelity(ideal.handle, noisy.handle, ctypes.byref(Fv), ctypes.byref(Nv)))

        ke = max(1, min(args.steps, 2))
        e2e_step()
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        for _ in range(ke):
            e2e_step()
        torch.cuda.synchronize()
        dt = max_over_ranks((time.perf_counter() - t0) / ke, world)
        tables = qs.Plan(M, c["noisy"], mode="auto").stats()["table_bytes"] * 2
        result["e2e"] = {"value": job_throughput(amp_step, world, dt * 1e3), "unit": "amp-updates/s",
                         "ms_per_step": dt * 1e3, "steps": ke,
                         "h2d_bytes_per_step": int(gi.nbytes + gn.nbytes + tables), "d2h_bytes_per_step": 24,
                         "path": "qsim_reset x2, qsim_apply_circuit x2 from host gate records (plan built and "
                                 "its tables copied in the call), qsim_fidelity",
                         "F": Fv.value}

    del p_i, p_n
    for mode in [m for m in args.modes.split(",") if m and m != head]:
        if mode == "unfused" and args.no_unfused:
            continue
        q_i, q_n, t_plan = make(mode)
        steps, warm = (1, 0) if mode == "unfused" else (max(1, min(args.steps, 2)), 1)
        msm, (Fm, nm), roofm, _, _, per_plan, clk = _timed_steps(
            stepper(q_i, q_n), [q_i, q_n], steps, warm, stream, world, local, M)
        modes[mode] = {"amp_updates_per_s": job_throughput(amp_step, world, msm), "ms_per_step": msm,
                       "steps": steps, "warmup": warm, "passes_per_circuit": per_plan[1],
                       "specialised_passes": "specialised" in q_n.describe(), "plan_create_s": round(t_plan, 3),
                       "roofline": roofm, "F": Fm, "norm": nm, "clocks": clk}
        del q_i, q_n
    for m, d in modes.items():
        d["speedup_of_unfused"] = (modes["unfused"]["ms_per_step"] / d["ms_per_step"]) if "unfused" in modes else None
    result["modes"] = modes
    if args.mode == "auto":
        try:
            result["auto_rates"] = qs.tune_rates("c64", specialize=spec)
        except qs.QsimError as e:
            result["auto_rates"] = {"error": str(e)}
    del ideal, noisy
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return result, c, None


def run_qft(args, world, local, workload, mode, steps, warmup):
    """The quantum FFT: one step = the error-free and the noisy circuit, both
    out of place from the resident input state, then the fidelity and norm."""
    import ctypes

    import torch

    import paper_quant_ph_9804039_gb300 as qs

    wl = WORKLOADS[workload]
    M = wl["M"]
    c, x = workload_circuit(wl)
    n_logical = c["n_logical_gates"]
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    xin = qs.State(M, device=dev, stream=stream, zero=False).set(x)
    ideal = qs.State(M, device=dev, stream=stream, zero=False)
    noisy = qs.State(M, device=dev, stream=stream, zero=False)
    spec = not args.no_specialize
    t_plan = time.perf_counter()
    p_ideal = qs.Plan(M, c["ideal"], mode=mode, tile_bits=args.tile_bits, specialize=spec)
    p_noisy = qs.Plan(M, c["noisy"], mode=mode, tile_bits=args.tile_bits, specialize=spec)
    t_plan = time.perf_counter() - t_plan
    specialised = "specialised" in p_noisy.describe()
    st_n = p_noisy.stats()
    amp_updates_step = 2.0 * n_logical * float(1 << M)

    def step():
        p_ideal.execute(ideal, xin)
        p_noisy.execute(noisy, xin)
        return qs.fidelity(ideal, noisy)

    ms, (F, nrm), roof, launches, bytes_step, per_plan, clocks = _timed_steps(
        step, [p_ideal, p_noisy], steps, warmup, stream, world, local, M)
    value = job_throughput(amp_updates_step, world, ms)
    result = {
        "metric": "amplitude-updates/s", "value": value, "unit": "amp-updates/s", "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "complex64", "data": "synthetic",
        "config": {"workload": workload, "M": M, "circuit": "qft", "sigma": wl["sigma"],
                   "gates_per_circuit": n_logical, "gate_records_per_circuit": int(len(c["noisy"])),
                   "circuits_per_step": 2, "mode": mode, "tile_bits": st_n["tile_bits"],
                   "passes_per_circuit": per_plan[1], "specialised_passes": specialised,
                   "plan_create_s": round(t_plan, 3),
                   "l2": f"inputs larger than L2 ({(8 << M) >> 20} MiB per state)",
                   "parallelism": f"replicas{world}"},
        "roofline": roof,
        "gpu_launches": int((launches + 2) * steps),  # + the overlap reduction's two kernels
        "fidelity": F, "norm": nrm,
        "hbm_gbs_step": (bytes_step + 2 * 8 * float(1 << M)) / (ms / 1e3) / 1e9,
        "clocks": clocks,
    }

    # end to end through the C ABI with host buffers: every step copies its
    # input from pinned host memory and reads F and the norm back.  Pipelined
    # over two input states on a copy stream: step k+1's copy is queued
    # (qsim_set_state_async) before step k's fidelity is read, so it overlaps
    # step k's passes; the synchronous read of step k orders the reuse of the
    # buffer that step k+1 will overwrite two steps later.
    if not args.no_e2e:
        xh = [torch.empty(1 << M, dtype=torch.complex64, pin_memory=True) for _ in range(2)]
        for h in xh:
            h.numpy()[:] = x
        ke = max(2, min(steps, 10))
        lib = qs.load_library()
        Fv, Nv = ctypes.c_double(), ctypes.c_double()
        copy_stream = torch.cuda.Stream(device=dev)
        xq = [qs.State(M, device=dev, stream=copy_stream, zero=False) for _ in range(2)]

        def e2e_run(k_steps):
            xq[0].set_async(xh[0])
            for k in range(k_steps):
                p_ideal.execute(ideal, xq[k % 2])
                p_noisy.execute(noisy, xq[k % 2])
                if k + 1 < k_steps:
                    xq[(k + 1) % 2].set_async(xh[(k + 1) % 2])
                qs._check(lib.qsim_fidelity(ideal.handle, noisy.handle, ctypes.byref(Fv), ctypes.byref(Nv)))

        e2e_run(2)
        torch.cuda.synchronize()
        barrier(world)
        t0 = time.perf_counter()
        e2e_run(ke)
        torch.cuda.synchronize()
        dt = max_over_ranks((time.perf_counter() - t0) / ke, world)
        assert abs(Fv.value - F) < 1e-9, (Fv.value, F)
        result["e2e"] = {"value": job_throughput(amp_updates_step, world, dt * 1e3), "unit": "amp-updates/s",
                         "ms_per_step": dt * 1e3, "h2d_bytes_per_step": int(x.nbytes),
                         "d2h_bytes_per_step": 24, "steps": ke,
                         "pipelined": "input copy of step k+1 overlaps the passes of step k (two input states)"}
        del xq, xh

    # one-gate-per-launch form on the same GPU
    if not args.no_unfused and mode != "unfused":
        pu_i = qs.Plan(M, c["ideal"], mode="unfused")
        pu_n = qs.Plan(M, c["noisy"], mode="unfused")

        def ustep():
            pu_i.execute(ideal, xin)
            pu_n.execute(noisy, xin)
            return qs.fidelity(ideal, noisy)

        ku = max(1, min(steps, 3))
        msu, (Fu, _), _, lu, _, _, _ = _timed_steps(ustep, [pu_i, pu_n], ku, 1, stream, world, local, M)
        result["unfused"] = {"value": job_throughput(amp_updates_step, world, msu), "ms_per_step": msu,
                             "launches_per_step": lu + 2, "fidelity": Fu, "speedup_of_value": msu / ms}
        del pu_i, pu_n
    del xin, ideal, noisy, p_ideal, p_noisy
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    return result, c, x


def run_ours(args, rank, world, local):
    wl = WORKLOADS[args.workload]
    if wl["circuit"] == "brickwork":
        result, c, x = run_brickwork(args, rank, world, local)
        if not args.no_qft:
            q, _, _ = run_qft(args, world, local, "qft-m28-c64", "tiled", 20, 3)
            result["qft_m28"] = {k: q[k] for k in ("value", "unit", "ms_per_step", "steps", "warmup", "config",
                                                   "roofline", "e2e", "unfused", "fidelity", "norm", "clocks",
                                                   "gpu_launches", "hbm_gbs_step") if k in q}
    else:
        result, c, x = run_qft(args, world, local, args.workload, args.mode, args.steps, args.warmup)
    if not args.no_extras:
        import torch
        stream = torch.cuda.current_stream()
        result["single_gate"] = bench_single_gate(stream)
        result["batched"] = bench_trajectories(world, result["clocks"].get("sm_mhz"))
        result["subspace"] = bench_subspace(world, stream)
        result["decoherence"] = bench_decoherence(world, stream)
        result["qutrit"] = bench_qutrit(world, stream)
        result["serving"] = bench_serving(args.serve_requests, world)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, ng, dt, nt, Ms = oracle_sample(wl["M"], c["noisy"], x, budget_s=15.0)
        v1, ng1, dt1, _, Ms1 = oracle_sample(wl["M"], c["noisy"], None, budget_s=5.0, nthreads=1, max_M=26)
        result["cpu_baseline"] = {"value": v, "unit": "amp-updates/s", "cores": nt, "kind": "oracle",
                                  "sample": f"first {ng} gates of the noisy circuit at M={Ms} "
                                            f"(complex128), {dt:.1f} s",
                                  "one_core": {"value": v1, "unit": "amp-updates/s", "cores": 1,
                                               "sample": f"first {ng1} gates of the noisy circuit at M={Ms1} "
                                                         f"(complex128), {dt1:.1f} s"}}
    if rank == 0:
        print(json.dumps(result), flush=True)


# ------------------------------------------------------------------ extras ---
def _events_ms(fn, reps, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    fn()
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def bench_single_gate(stream):
    """One dense gate per launch (k_gate_*) on an M=30 complex64 state (8 GiB):
    algorithmic bytes 16 * 2^30 per launch; targets below and above the
    512-byte warp chunk."""
    import torch
    import paper_quant_ph_9804039_gb300 as qs
    from workloads import generators as W
    M = 30
    st = qs.State(M, stream=stream)
    U = W.mat_haar_su2(np.random.default_rng(9))
    peak, _ = measured_peaks()
    out = {"M": M, "bytes_per_launch": 16 << M, "targets": {}}
    for t in (0, 3, 7, 20, 29):
        ms = _events_ms(lambda: st.apply_gate(U, t), 5, stream)
        gbs = (16 << M) / (ms / 1e3) / 1e9
        out["targets"][str(t)] = {"ms": round(ms, 4), "GB/s": round(gbs, 1), "frac": round(gbs / peak, 4)}
    ms = _events_ms(lambda: st.apply_gate(W.mat_x(), 17, (25,)), 5, stream)
    out["cnot_17_ctl25"] = {"ms": round(ms, 4), "GB/s": round((8 << M) / (ms / 1e3) / 1e9, 1)}
    del st
    torch.cuda.empty_cache()
    return out


def bench_trajectories(world, sm_mhz=None):
    """Batched error trajectories: M=16, T=4096, 20-layer brickwork, sigma=5e-3,
    one persistent launch replayed from a CUDA graph; against running the
    same trajectories one circuit at a time, one gate per launch (their
    plans made before the timed loop).

    Roofline (ALU-bound: every trajectory lives on chip): algorithmic flops
    = 16 per amplitude per dense 2x2 complex gate (8 FMA: two complex
    products and a sum per output), 0 for the CNOTs (a permutation), against
    the FP32 FMA peak derived from 152 SMs x 128 lanes x 2 flop x the SM
    clock sampled during the timed region."""
    import paper_quant_ph_9804039_gb300 as qs
    from workloads import generators as W
    M, T = 16, 4096
    b = W.circuit_brickwork(M, 20)
    eps = W.trajectory_eps(len(b["ideal"]), T, 5e-3)
    plan = qs.TrajPlan(M, b["ideal"], b["axes"], max_T=T, use_graph=True)
    plan.run(eps)
    t0 = time.perf_counter()
    reps = 3
    for _ in range(reps):
        F, mean, var = plan.run(eps)
    dt = (time.perf_counter() - t0) / reps
    n_dense = int(sum(1 for r in b["ideal"] if int(r["ncontrols"]) == 0))
    flops = T * n_dense * 16.0 * float(1 << M)
    mhz = sm_mhz or 2070.0
    peak = derived_fp32_peak(mhz)
    # sequential one-gate-per-launch form on a sample of trajectories
    ideal = qs.State(M)
    qs.Plan(M, b["ideal"], mode="unfused").execute(ideal)
    noisy = qs.State(M)
    ns = 16
    plans = [qs.Plan(M, W.with_errors(b["ideal"], b["axes"], eps[t]), mode="unfused") for t in range(ns)]
    plans[0].execute(noisy)
    qs.fidelity(ideal, noisy)
    t0 = time.perf_counter()
    for t in range(ns):
        noisy.reset()
        plans[t].execute(noisy)
        qs.fidelity(ideal, noisy)
    dts = (time.perf_counter() - t0) / ns
    info = plan.info()
    return {"workload": "brickwork-m16-t4096", "trajectories_per_s": world * T / dt, "s_per_batch": dt,
            "mean_F": mean, "var_F": var, "tile_bits": info["tile_bits"], "passes": info["n_passes"],
            "grid": info["grid"], "gates": int(len(b["ideal"])), "dense_gates": n_dense,
            "amp_updates_per_s": world * T * len(b["ideal"]) * float(1 << M) / dt,
            "roofline": {"bound": "alu", "achieved": flops / dt, "peak": peak, "unit": "FLOP/s",
                         "frac": round(flops / dt / peak, 4),
                         "peak_source": f"derived: {GB300_SMS} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x "
                                        f"{mhz:.0f} MHz" + (" (sampled)" if sm_mhz else " (maximum clock)"),
                         "flops": "16 per amplitude per dense complex 2x2 gate, 0 per CNOT"},
            "sequential_unfused_trajectories_per_s": 1.0 / dts,
            "sequential_sample": f"{ns} trajectories, one gate per launch, plans made before the timed loop",
            "speedup_of_sequential": (T / dt) * dts}


def bench_subspace(world, stream):
    """Touched-qubit subspace (Section 3.2, EQ 6): a circuit that touches its
    30 qubits one at a time (Hadamards on 4, then per further qubit a CNOT
    onto it and 16 gates among the touched ones; over-rotation sigma=1e-3),
    from |0...0>, complex64.  One step = the error-free and the noisy circuit
    and F.  The flat plans run every gate on all 2^30 amplitudes; the
    subspace plans run each segment on the prefix its touched qubits span and
    restore the qubit order at the end."""
    import torch
    import paper_quant_ph_9804039_gb300 as qs
    from workloads import generators as W
    M = 30
    c = W.circuit_gradual(M, start=4, per_qubit=16)
    n = len(c["ideal"])
    a = qs.State(M, stream=stream)
    b = qs.State(M, stream=stream)
    out = {"workload": "gradual-m30-c64", "M": M, "gates_per_circuit": n}
    for name, sub in (("flat", False), ("subspace", True)):
        t = time.perf_counter()
        # the general register kernel: plan creation stays short (no NVRTC per segment)
        pi = qs.Plan(M, c["ideal"], mode="tiled", subspace=sub)
        pn = qs.Plan(M, c["noisy"], mode="tiled", subspace=sub)
        t = time.perf_counter() - t
        res = {}

        def step():
            if not sub:
                a.reset()
                b.reset()
            pi.execute(a)
            pn.execute(b)
            res["F"] = qs.fidelity(a, b)

        ms = _events_ms(step, 3, stream)
        entry = {"ms_per_step": ms, "amp_updates_per_s": world * 2.0 * n * float(1 << M) / (ms / 1e3),
                 "passes_per_circuit": pn.stats()["n_passes"], "F": res["F"][0], "norm": res["F"][1],
                 "plan_create_s": round(t, 3)}
        if sub:
            line = pn.describe().split("subspace: ")[1].splitlines()[0]
            entry["planned"] = line
        out[name] = entry
        del pi, pn
    out["speedup"] = out["flat"]["ms_per_step"] / out["subspace"]["ms_per_step"]
    out["F_difference"] = abs(out["flat"]["F"] - out["subspace"]["F"])
    del a, b
    torch.cuda.empty_cache()
    return out


def bench_decoherence(world, stream):
    """Decoherence after every operation (Section 3.4 reading): M=28,
    complex64, 100 random gates with dephasing kicks (sigma 1e-3) and
    amplitude damping gamma = 1e-3; one pass over the vector per operation
    (16 bytes per amplitude), timed with CUDA events."""
    import torch
    import paper_quant_ph_9804039_gb300 as qs
    from workloads import generators as W
    M, n = 28, 100
    c = W.circuit_c1_random(M, n, 1e-3, seed_circuit=5, seed_err=6)
    rng = np.random.default_rng(7)
    delta = rng.normal(0.0, 1e-3, n)
    r = rng.random(n)
    st = qs.State(M, stream=stream).set(W.random_state(M, seed=2))
    qs.run_decoherence(st, c["noisy"][:4], delta[:4], r[:4], 1e-3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    jumps, p = qs.run_decoherence(st, c["noisy"], delta, r, 1e-3)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    peak, _ = measured_peaks()
    gbs = (n + 1) * 16.0 * float(1 << M) / (ms / 1e3) / 1e9
    out = {"workload": "decoherence-m28-c64", "M": M, "operations": n, "gamma": 1e-3, "ms": ms,
           "ms_per_operation": ms / n, "launches": n + 1, "GB/s": round(gbs, 1), "frac": round(gbs / peak, 4),
           "jumps": int(jumps.sum()), "amp_updates_per_s": world * n * float(1 << M) / (ms / 1e3),
           "passes_per_operation": 1.0, "paper_transformations_per_operation": 3}
    del st
    torch.cuda.empty_cache()
    return out


def bench_qutrit(world, stream):
    """The three-state model: M=18 particles (3^18 complex64 amplitudes,
    3.1 GB), 40 laser pulses (a third controlled), one launch per pulse;
    algorithmic bytes 16 per amplitude per uncontrolled pulse (a controlled
    pulse reads and writes the third of the triples its control selects)."""
    import torch
    import paper_quant_ph_9804039_gb300 as qs
    from workloads import generators as W
    M = 18
    c = W.circuit_qutrit(M, 40, seed_circuit=18)
    st = qs.QutritState(M, stream=stream)
    st.apply(c["noisy"][:2])
    ms = _events_ms(lambda: st.apply(c["noisy"]), 3, stream)
    nct = int(np.sum(c["noisy"]["ncontrols"] > 0))
    byts = 16.0 * 3 ** M * ((len(c["noisy"]) - nct) + nct / 3.0)
    peak, _ = measured_peaks()
    gbs = byts / (ms / 1e3) / 1e9
    out = {"workload": "qutrit-m18-c64", "M": M, "pulses": len(c["noisy"]), "controlled": nct, "ms": ms,
           "GB/s": round(gbs, 1), "frac": round(gbs / peak, 4),
           "amp_updates_per_s": world * len(c["noisy"]) * float(3 ** M) / (ms / 1e3)}
    del st
    torch.cuda.empty_cache()
    return out


def bench_serving(n_requests, world):
    """Served stream: Poisson arrivals, M ~ U{12..26}, 50..500 gates, sigma
    log-uniform in [1e-5, 1e-2], 160 GiB budget.  The base offered rate is
    the measured capacity of the sequential one-gate-per-launch loop (load
    1.0 for it).  Latency = completion - arrival.  The sequential loop serves
    a sample of the stream live (one request at a time, in arrival order);
    the continuous-batching server serves the whole stream at the base rate,
    then again at 4x and 16x the base rate to find its saturation
    throughput, and once with every request submitted at t = 0."""
    import paper_quant_ph_9804039_gb300 as qs
    from workloads import generators as W
    reqs = W.serving_requests(n_requests)
    circs = [W.request_circuit(r) for r in reqs]

    def serve_one(r, c):
        a = qs.State(r["M"])
        b = qs.State(r["M"])
        qs.Plan(r["M"], c["ideal"], mode="unfused").execute(a)
        qs.Plan(r["M"], c["noisy"], mode="unfused").execute(b)
        return qs.fidelity(a, b)

    serve_one(reqs[0], circs[0])
    t0 = time.perf_counter()
    ncal = min(len(reqs), 50)
    for r, c in zip(reqs[:ncal], circs[:ncal]):
        serve_one(r, c)
    lam = ncal / (time.perf_counter() - t0)  # sequential capacity, requests/s
    # sequential loop under the stream (sample)
    ns = min(len(reqs), 200)
    seq_lat = []
    t_start = time.perf_counter()
    t_arr = 0.0
    for r, c in zip(reqs[:ns], circs[:ns]):
        t_arr += r["gap"] / lam
        now = time.perf_counter() - t_start
        if now < t_arr:
            time.sleep(t_arr - now)
        serve_one(r, c)
        seq_lat.append(time.perf_counter() - t_start - t_arr)
    seq_rate = ns / (time.perf_counter() - t_start)

    def serve_stream(rate, sel):
        """The server under the requests `sel` arriving at `rate` (None: all at once)."""
        srv = qs.Server(hbm_budget=160 << 30, max_slots=16, mode="tiled")
        t_start = time.perf_counter()
        t_arr = 0.0
        done = []
        for r, c in sel:
            if rate is not None:
                t_arr += r["gap"] / rate
                while time.perf_counter() - t_start < t_arr:
                    done += srv.poll(256, wait_ms=0)
                    time.sleep(0.0002)
            srv.submit(r["M"], c["ideal"], c["noisy"])
        while len(done) < len(sel):
            done += srv.poll(256, wait_ms=100)
        t_end = time.perf_counter()
        st = srv.stats()
        srv.close()
        lat = np.array([d["t_done"] - d["t_submit"] for d in done])
        return {"offered_rate": rate, "requests": len(sel), "ok": sum(1 for d in done if d["status"] == 0),
                "requests_per_s": world * len(sel) / (t_end - t_start),
                "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                "max_active": st["max_active"], "peak_state_bytes": st["peak_bytes"]}

    pairs = list(zip(reqs, circs))
    base = serve_stream(lam, pairs)
    loads = {}
    for mult in (4, 16):
        loads[f"{mult}x"] = serve_stream(lam * mult, pairs)
    loads["all_at_t0"] = serve_stream(None, pairs)
    sat = max(v["requests_per_s"] for v in loads.values())
    out = {"workload": "served-stream", "requests": len(reqs), "ok": base["ok"], "offered_rate": lam,
           "requests_per_s": base["requests_per_s"], "p50_ms": base["p50_ms"], "p99_ms": base["p99_ms"],
           "max_active": base["max_active"], "peak_state_bytes": base["peak_state_bytes"],
           "higher_loads": loads, "saturation_requests_per_s": sat,
           "sequential_unfused": {"requests_per_s": seq_rate, "capacity_requests_per_s": lam, "sample": ns,
                                  "p50_ms": float(np.percentile(seq_lat, 50) * 1e3),
                                  "p99_ms": float(np.percentile(seq_lat, 99) * 1e3)},
           "saturation_over_sequential_capacity": sat / lam}
    return out


# ---------------------------------------------------------- reference arm ---
def run_reference(args, rank, world):
    """The CPU oracle as it stands, on the host cores, same metric and config;
    each step is a bounded sample (consecutive gates of the noisy circuit, at
    the workload's M when the host has the memory)."""
    if rank != 0:
        return
    import oracle

    wl = WORKLOADS[args.workload]
    c, x = workload_circuit(wl)
    M = oracle_size(wl["M"])
    gates = c["noisy"]
    gates = gates[[i for i in range(len(gates)) if gates[i]["target"] < M
                   and all(q < M for q in gates[i]["controls"][: int(gates[i]["ncontrols"])])]]
    orc = oracle.Oracle()
    nt = oracle.default_threads()
    if x is not None and M == wl["M"]:
        psi = x.astype(np.complex128)
    else:
        psi = np.zeros(1 << M, dtype=np.complex128)
        psi[0] = 1.0
    orc.apply_circuit(psi, gates[:1], nthreads=nt)  # touches every page
    t0 = time.perf_counter()
    orc.apply_circuit(psi, gates[1:2], nthreads=nt)
    t1 = time.perf_counter() - t0
    total_steps = args.steps + args.warmup
    per_step = max(1, int(min(8.0, 150.0 / max(1, total_steps)) / max(t1, 1e-6)))
    g = 2
    for _ in range(args.warmup):
        orc.apply_circuit(psi, gates[g:g + per_step], nthreads=nt)
        g = (g + per_step) % len(gates)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sel = gates[g:g + per_step]
        if len(sel) < per_step:
            g = 0
            sel = gates[:per_step]
        orc.apply_circuit(psi, sel, nthreads=nt)
        g += per_step
    dt = (time.perf_counter() - t0) / args.steps
    v = per_step * float(1 << M) / dt
    sample = f"{per_step} consecutive gates of the noisy circuit per step at M={M} (complex128)"
    print(json.dumps({
        "impl": "reference", "metric": "amplitude-updates/s", "value": v, "unit": "amp-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "complex128",
        "data": "synthetic",
        "config": {"workload": args.workload, "M": wl["M"], "circuit": wl["circuit"], "sigma": wl["sigma"],
                   "oracle_M": M},
        "cpu_baseline": {"value": v, "unit": "amp-updates/s", "cores": nt, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "amp-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    rank, world, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    dist_init(world, local)
    run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
