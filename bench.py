#!/usr/bin/env python
"""Benchmark: noisy density-matrix evolution of a 15-qubit ring transverse-
field Ising Trotter circuit on one GB300 (sm_103a).

One step = one Trotter step (30 noisy gates: 15 RZZ(0.2) with 2-qubit
depolarising 5e-4 on the ring, 15 RX(0.1) with 1-qubit depolarising 5e-4)
through the whole hot path -- superoperator build (FP64, GPU), fusion (FP64,
GPU), apply passes over all 4^15 entries of vec(rho), and the FP64 <Z0 Z1>
reduction -- with rho carried from step to step.

  value      noisy gates/s of the FP64 path, inputs resident in device memory
             (a compiled program re-run each step; readout to device memory)
  e2e        the same through the public C-ABI call with host buffers: each
             step copies the step's op tables host-to-device (tq_run_circuit)
             and reads <Z0 Z1> back to the host (tq_expect_z)
  split      the split-precision path (complex64 rho, FP32 products, FP64
             build/fusion/reductions) on the same workload, with its error
             against the FP64 path
  roofline   dominant kernel of the FP64 path (and of the split path),
             algorithmic flops or bytes per launch over CUDA-event-timed
             launch durations inside the timed region
  cpu_baseline  the FP64 CPU oracle on a bounded sample (see cpu_baseline())

--impl reference times the CPU oracle (there is no reference code) on the
same workload and metric, one bounded sample per step.

Multi-GPU: the path does not shard (one 16 GiB density matrix per GPU); with
--gpus N each rank runs an independent replica and value sums the ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "superoperator gates/s at 15q (FP64 vs split), served circuits/s + p99 latency"
UNIT = "noisy gates/s"
N_QUBITS = 15
ZZ_MASK = 0b11
SAMPLE_QUBITS = 12      # register size of the CPU-oracle sample
SEED_SERVE = 2404_13184 + 5


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


def device_sms() -> int:
    """Multiprocessor count of the current device (152 on a GB300)."""
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def fp64_peak_tflops(sm_mhz: float, sms: int | None = None) -> float:
    """Nominal FP64 (DFMA) rate from unit counts and clock: 4 FP64 flops (2
    DFMA) per SM per clock (1.26 TFLOP/s on 152 SMs at 2070 MHz)."""
    return (sms or device_sms()) * 4 * sm_mhz * 1e6 / 1e12


_PIPE_CACHE = {}


def measured_pipe(tq, pipe: str) -> float:
    """Measured rate of an arithmetic pipe (tq_pipe_rate), in TFLOP/s (FMA and
    MMA pipes) or T ops/s (conversions); measured once per process."""
    iters = {"dfma": 2048, "dmma": 512, "ffma": 65536, "cvt_f64_s64": 8192, "cvt_f64_f32": 8192}[pipe]
    if pipe not in _PIPE_CACHE:
        rate, _ = tq.pipe_rate(pipe, iters)
        _PIPE_CACHE[pipe] = rate / 1e12
    return _PIPE_CACHE[pipe]


def host_cpu() -> dict:
    """Threads available to this process and the CPU model of the host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            model = "unknown"
    return {"nproc": os.cpu_count(), "cpu_model": model}


def kernel_source_sha(symbol: str):
    """sha256 (first 16 hex digits) of a kernel's definition in csrc/ (from its
    `__global__` to the closing brace of its body) together with the shared
    device types and helpers of tq_device.cuh (the part before its launcher
    declarations, #include lines left out): changes when the kernel's code
    does."""
    csrc = os.path.join(ROOT, "paper_2404_13184_gb300", "csrc")
    for name in sorted(os.listdir(csrc)):
        if not name.endswith((".cu", ".cuh")):
            continue
        text = open(os.path.join(csrc, name)).read()
        at = text.find(" " + symbol + "(")
        if at < 0:
            continue
        start = text.rfind("__global__", 0, at)
        start = text.rfind("template", 0, start) if text.rfind("template", 0, start) > text.rfind(";", 0, start) else start
        brace = text.find("{", at)
        depth, k = 0, brace
        while k < len(text):
            depth += {"{": 1, "}": -1}.get(text[k], 0)
            if depth == 0:
                break
            k += 1
        helpers = open(os.path.join(csrc, "tq_device.cuh")).read().split("// --- kernel launchers")[0]
        helpers = "\n".join(l for l in helpers.splitlines() if not l.startswith("#include"))
        return hashlib.sha256((text[start:k + 1] + helpers).encode()).hexdigest()[:16]
    return None


def traffic_from_profile(kernel: str):
    """dram read+write bytes per launch from the committed ncu summary of
    `kernel`, if the kernel's source is unchanged since the capture (the
    summary names the kernel's symbol and the hash kernel_source_sha gave)."""
    path = os.path.join(ROOT, "profiles", f"{kernel}.txt")
    try:
        fields = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                fields[k.strip()] = v.split("#")[0].strip()
        sym = fields.get("kernel_symbol")
        if not sym or fields.get("source_sha256_16") != kernel_source_sha(sym):
            return None
        return float(fields["dram_bytes_per_full_launch"])
    except Exception:
        return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=self.file,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.file.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(v, world, device="cuda"):
    """Max of a per-rank time over all ranks (the job takes as long as its
    slowest replica); identity on one rank."""
    if world == 1 or v is None:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, max_ms, world):
    """Whole-job rate: units processed by all ranks over the slowest rank's time."""
    return world * units_per_rank / (max_ms / 1e3)


def step_ops():
    from paper_2404_13184_gb300 import workloads
    return workloads.tfim_ring(N_QUBITS, steps=1).ops


def run_device_leg(tq, torch, precision, steps, warmup, world, clocks=None, engine="auto"):
    """K timed steps from device-resident inputs; returns timings and stats."""
    import torch.distributed as dist
    st = tq.State(N_QUBITS, precision, engine=engine)
    on_tensor = st.fp64_on_tensor() if precision == "fp64" else False
    prog = tq.DeviceProgram(N_QUBITS, step_ops(), width=-1, precision=precision)
    masks = torch.tensor([ZZ_MASK], dtype=torch.int64, device="cuda")
    out = torch.zeros(warmup + steps, dtype=torch.float64, device="cuda")
    for w in range(warmup):
        st.run_program(prog)
        st.expect_z_device(masks.data_ptr(), 1, out[w:].data_ptr())
    torch.cuda.synchronize()
    st.profile(True)
    launches0 = st.launch_count()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if clocks:
        clocks.start()
    e0.record(stream)
    for i in range(steps):
        st.run_program(prog)
        st.expect_z_device(masks.data_ptr(), 1, out[warmup + i:].data_ptr())
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop() if clocks else None
    if world > 1:
        dist.barrier()
    ms = e0.elapsed_time(e1)
    launches = st.launch_count() - launches0
    stats = st.profile_stats()
    st.profile(False)
    zz = out.cpu().tolist()
    res = {"ms": ms, "launches": launches, "stats": stats, "zz": zz, "blocks": prog.n_blocks,
           "max_width": prog.max_width, "table_bytes": prog.table_bytes, "clocks": clk, "on_tensor": on_tensor}
    prog.free()
    st.free()
    return res


def run_e2e_leg(tq, torch, precision, steps, warmup, world, engine="auto", profile=False):
    """The public host-buffer API: tq_run_circuit + tq_expect_z per step.
    Returns ms for the K steps (and, with profile, the per-kernel stats and
    the <Z0 Z1> of every step)."""
    import torch.distributed as dist
    st = tq.State(N_QUBITS, precision, engine=engine)
    prog = tq.Program(step_ops())
    for _ in range(warmup):
        st.run(prog, width=-1)
        st.expect_z([ZZ_MASK])
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if profile:
        st.profile(True)
    zz = []
    t0 = time.perf_counter()
    for _ in range(steps):
        st.run(prog, width=-1)
        zz.append(float(st.expect_z([ZZ_MASK])[0]))
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    if world > 1:
        dist.barrier()
    stats = st.profile_stats() if profile else None
    st.free()
    if profile:
        return dt * 1e3, stats, zz
    return dt * 1e3


def fp64_roofline(name, st, pipes, sm_max, sm_mhz, sms, hbm_gbs, peak_src):
    """Roofline of the dominant FP64 apply kernel: the tensor-core engine's
    passes are bound by HBM (algorithmic bytes: one read and one write of
    every canonical entry), the DFMA kernels by the FP64 pipe (algorithmic
    flops: 8 per applied complex multiply-add)."""
    avg_ms = st["total_ms"] / st["launches"]
    if "f64tc" in name:
        ach = st["bytes"] / (avg_ms / 1e3) / 1e9
        return {"kernel": name, "bound": "hbm", "achieved": ach, "peak": hbm_gbs, "unit": "GB/s",
                "frac": ach / hbm_gbs, "traffic": traffic_from_profile(name),
                "algorithmic_bytes_per_launch": st["bytes"], "algorithmic_flops_per_launch": st["flops"],
                "launches": st["launches"], "avg_launch_ms": avg_ms, "peak_source": f"{peak_src} HBM copy bandwidth"}
    ach = st["flops"] / (avg_ms / 1e3) / 1e12
    peak = fp64_peak_tflops(sm_max, sms)
    return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
            "traffic": traffic_from_profile(name),
            "algorithmic_bytes_per_launch": st["bytes"], "algorithmic_flops_per_launch": st["flops"],
            "flops_count": "8 per nonzero of the row lists the kernel applied (read back from the device), per "
                           "canonical group" if "sparse" in name else "dense 8 x 16^w per canonical group",
            "launches": st["launches"], "avg_launch_ms": avg_ms,
            "peak_source": f"DFMA pipe, nominal: {sms} SMs x 4 FP64 flop/clk x {sm_max:.0f} MHz",
            "frac_at_measured_clock": ach / fp64_peak_tflops(sm_mhz, sms),
            "peak_measured_dfma": pipes["dfma"], "frac_of_measured_dfma": ach / pipes["dfma"]}


def dominant(stats: dict):
    apply = {k: v for k, v in stats.items() if k.startswith("apply")}
    name = max(apply, key=lambda k: apply[k]["total_ms"])
    return name, apply[name]


def cpu_sample_rate(pairs: int = 1):
    """Oracle rate on a bounded sample of the workload: `pairs` x (RZZ + 2q
    depolarising, RX + 1q depolarising) of the ring TFIM step, on a
    SAMPLE_QUBITS-qubit register, scaled by 4^-(15 - SAMPLE_QUBITS) to the
    15-qubit register (the oracle's cost per op is proportional to 4^n).
    Returns (scaled gates/s, raw gates/s, seconds)."""
    import numpy as np
    from oracle import dm_oracle
    from paper_2404_13184_gb300 import workloads
    n = SAMPLE_QUBITS
    ops = workloads.tfim_ring(n, steps=1).ops
    pair_ops = ops[0:2] + ops[2 * n:2 * n + 2]
    rho = dm_oracle.zero_state(n)
    t0 = time.perf_counter()
    for _ in range(pairs):
        for op in pair_ops:
            rho = dm_oracle.apply_op(rho, op)
    dt = time.perf_counter() - t0
    raw = 2 * pairs / dt
    return raw * 4.0 ** (-(N_QUBITS - n)), raw, dt


def oracle_prefix_time(n, ops, budget_s, min_ops=3):
    """The CPU oracle run op by op from |0><0| on an n-qubit register until
    `budget_s` seconds have passed (and at least `min_ops` ops ran) or the
    ops run out: (ops done, seconds; the initial state is not timed)."""
    from oracle import dm_oracle
    rho = dm_oracle.zero_state(n)
    t0 = time.perf_counter()
    done = 0
    for op in ops:
        rho = dm_oracle.apply_op(rho, op)
        done += 1
        if done >= min_ops and time.perf_counter() - t0 >= budget_s:
            break
    return done, time.perf_counter() - t0


def cpu_baseline_circuits(circuits, budget_per_n=1.5, masks=(1, 3), full_max_n=6, full_count=8):
    """Oracle time of a set of circuits, estimated from a bounded sample.
    First the first `full_count` circuits of at most `full_max_n` qubits run
    whole (their trace and <Z_mask> are kept, so the GPU results of those
    circuits can be held to the oracle). Then per remaining register size n,
    the first ops of the first circuit of that size run until
    `budget_per_n` seconds (or the circuit ends). The estimate is the
    oracle's time per op at each n x the ops of every circuit of size n.
    Returns (estimated seconds for all circuits, sample text, {circuit index:
    [Re tr, Im tr, <Z_m>...]})."""
    import numpy as np
    from oracle import dm_oracle
    per_op, parts, full = {}, [], {}
    spent = {}
    for idx, c in enumerate(circuits):
        if len(full) >= full_count:
            break
        if c.n > full_max_n:
            continue
        t0 = time.perf_counter()
        rho = dm_oracle.run_circuit(c.n, c.ops)
        dt = time.perf_counter() - t0
        tr = complex(np.trace(rho))
        full[idx] = [tr.real, tr.imag] + [float(dm_oracle.expect_z(rho, m)) for m in masks]
        t, k = spent.get(c.n, (0.0, 0))
        spent[c.n] = (t + dt, k + len(c.ops))
    for n, (t, k) in spent.items():
        per_op[n] = t / k
    if full:
        parts.append(f"{len(full)} whole circuits of <= {full_max_n} qubits")
    for c in circuits:
        if c.n not in per_op:
            done, dt = oracle_prefix_time(c.n, c.ops, budget_per_n)
            per_op[c.n] = dt / done
            parts.append(f"{done} ops at n={c.n}")
    total = sum(per_op[c.n] * len(c.ops) for c in circuits)
    return total, ("oracle time per op measured per register size (" + ", ".join(parts)
                   + "), times the ops of every circuit"), full


def split_accuracy(tq, n=8, steps=30):
    """Error of the split path on the same ring TFIM at 8 qubits (30 Trotter
    steps), against the FP64 GPU path (held to the oracle by the parity
    tests): the largest <Z0 Z1> error over the steps, the trace drift before
    renormalisation, the largest entry difference of rho, and the most
    negative eigenvalue of both states."""
    import numpy as np
    from paper_2404_13184_gb300 import workloads
    c = workloads.tfim_ring(n, steps)
    out = {}
    for prec in ("fp64", "split"):
        st = tq.State(n, prec)
        zz = []
        for a, b in c.steps:
            st.run(c.ops[a:b], width=-1)
            zz.append(float(st.expect_z([ZZ_MASK])[0]))
        out[prec] = (zz, st.trace().real, st.rho())
        st.free()
    (z64, t64, r64), (z32, t32, r32) = out["fp64"], out["split"]

    def min_eig(r):
        return float(np.min(np.linalg.eigvalsh((r + r.conj().T) / 2)))
    return {"qubits": n, "steps": steps, "zz_max_abs_err_vs_fp64": max(abs(a - b) for a, b in zip(z32, z64)),
            "max_abs_rho_diff_vs_fp64": float(np.max(np.abs(r32 - r64))),
            "split_trace_drift": abs(t32 - 1.0), "fp64_trace_drift": abs(t64 - 1.0),
            "split_min_eigenvalue": min_eig(r32), "fp64_min_eigenvalue": min_eig(r64),
            "_zz64": z64, "_zz32": z32}


def oracle_tfim_zz(n=8, steps=30):
    """<Z0 Z1> after each Trotter step of the same ring TFIM on n qubits from
    the CPU oracle (the config's oracle comparison; run in the CPU-baseline
    leg only)."""
    from oracle import dm_oracle
    from paper_2404_13184_gb300 import workloads
    c = workloads.tfim_ring(n, steps)
    rho = dm_oracle.zero_state(n)
    zz = []
    for a, b in c.steps:
        for op in c.ops[a:b]:
            rho = dm_oracle.apply_op(rho, op)
        zz.append(float(dm_oracle.expect_z(rho, ZZ_MASK)))
    return zz


def autotune_cache():
    return os.path.join(ROOT, "paper_2404_13184_gb300", "autotune_cache.txt")


def run_sweep(tq, torch, precision, steps, warmup, count=1024, n_min=4, n_max=11, reference=None,
              with_cpu=False, oracle_results=None, engine="auto"):
    """Batched sweep: `count` independent noisy circuits (n ~ U{4..11}, depth
    ~ U{50..500}, {H, RZ, RX, CX}, per-circuit depolarising p) in one
    persistent launch per run (a CUDA graph replay), tile and fusion width per
    qubit count from the autotuner. Returns throughput, per-circuit readouts
    and their accuracy: the trace drift |Tr rho - 1| (the circuits are trace
    preserving) and, given the FP64 run's readouts as `reference`, the
    largest difference from them (the FP64 path is held to the oracle by the
    parity tests)."""
    from paper_2404_13184_gb300 import workloads
    circuits = workloads.sweep(count, n_min=n_min, n_max=n_max)
    t_tune = time.perf_counter()
    tuned = {n: tq.autotune(precision, n, autotune_cache(), engine=engine) for n in sorted({c.n for c in circuits})}
    t_tune = time.perf_counter() - t_tune
    b = tq.Batch(precision, engine=engine)
    for c in circuits:
        b.add(c.n, c.ops, width=tuned[c.n][1], masks=[1, 3])
    for n, (tile, _, _) in tuned.items():
        b.set_tile(n, tile)
    for _ in range(max(1, warmup)):
        b.run()
        b.wait()
    stream = torch.cuda.current_stream()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        b.run()
    e1.record(stream)
    b.wait()
    ms = e0.elapsed_time(e1) / steps
    results = [b.result(j) for j in range(len(circuits))]
    err = {"circuits": len(results), "max_trace_drift": max(abs(r[0] - 1.0) for r in results),
           "max_abs_imag_trace": max(abs(r[1]) for r in results)}
    if reference is not None:
        # split readouts are divided by the trace; FP64 ones are not (Tr = 1 to ~1e-13)
        err["max_abs_z_diff_vs_fp64"] = max(max(abs(r[2] - f[2]), abs(r[3] - f[3])) for r, f in zip(results, reference))
        err["max_abs_trace_diff_vs_fp64"] = max(abs(r[0] - f[0]) for r, f in zip(results, reference))
    info = b.info()
    work = b.work()
    tensor_jobs = b.tensor_jobs() if precision == "fp64" else 0
    b.free()
    # roofline of the whole run (graph replay incl. superoperator build, fusion
    # and readout): split, and FP64 whose tile jobs run on the tensor-core
    # pass (nearly all the bytes), against HBM bandwidth; FP64 on the DFMA
    # engine against the DFMA rate
    hbm_gbs, sm_max, src = peaks()
    if precision == "fp64" and tensor_jobs == 0:
        ach = work["flops"] / (ms / 1e3) / 1e12
        sms = device_sms()
        peak = fp64_peak_tflops(sm_max, sms)
        roof = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "flops_per_run": work["flops"],
                "peak_source": f"DFMA pipe, nominal: {sms} SMs x 4 FP64 flop/clk x {sm_max:.0f} MHz"}
        try:
            meas = measured_pipe(tq, "dfma")
            roof.update({"peak_measured_dfma": meas, "frac_of_measured_dfma": ach / meas})
        except Exception:
            pass
    else:
        ach = work["bytes"] / (ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm_gbs, "unit": "GB/s", "frac": ach / hbm_gbs,
                "bytes_per_run": work["bytes"], "peak_source": f"hbm_gbs ({src})"}
        if precision == "fp64":
            roof["tensor_core_jobs"] = tensor_jobs
            roof["flops_per_run"] = work["flops"]
    gates = sum(c.n_gates for c in circuits)
    cpu = None
    if with_cpu:
        est, sample, oracle_results = cpu_baseline_circuits(circuits)
        cpu = {"value": count / est, "unit": "circuits/s", "cores": 1, **host_cpu(), "kind": "oracle",
               "sample": sample}
    if oracle_results:
        # the oracle's whole-circuit sample from the CPU-baseline leg: trace and
        # <Z> of those circuits against the oracle
        err["oracle_sample_circuits"] = len(oracle_results)
        err["max_abs_z_err_vs_oracle_sample"] = max(max(abs(results[i][2] - o[2]), abs(results[i][3] - o[3]))
                                                    for i, o in oracle_results.items())
        err["max_abs_trace_err_vs_oracle_sample"] = max(abs(results[i][0] - o[0]) for i, o in oracle_results.items())
    return {"ms_per_run": ms, "circuits_per_s": count / (ms / 1e3), "gates_per_s": gates / (ms / 1e3),
            "cpu_baseline": cpu, "oracle_results": oracle_results,
            "circuits": count, "noisy_gates": gates, "items": info["items"], "rho_bytes": info["rho_bytes"],
            "autotune": {str(n): {"tile_log2": t, "width": w, "ms": round(m, 3)} for n, (t, w, m) in tuned.items()},
            "autotune_s": t_tune, "accuracy": err, "roofline": roof, "results": results}


def run_serve(tq, precision, rate, duration, drain, seed=SEED_SERVE, rho_budget=150 << 30, max_live=64,
              keep_small=0):
    """Poisson arrivals (`rate` per second for `duration` s) of random noisy
    circuits (n ~ U{5..15}, depth ~ U{50..2000}, 30% CX, depolarising and
    amplitude damping per request) served by the continuous-batching loop,
    fused by the library's cost model (widths <= 2). The FIFO queue is kept in arrival order; a request is materialised and
    handed to the server when it reaches the head (a lookahead of 8; at most
    one per tick), and its latency is measured from its arrival time to the
    tick that collects its result. Ticks are pipelined (tq_server_step_async):
    the client's work overlaps the GPU, and gpu_busy_frac is the GPU time of
    the ticks (CUDA events) over the wall time. Requests unfinished when the
    drain window ends are censored. The returned dict carries, under
    "_completed", the (n, depth) of every completed request and, for the
    first `keep_small` completed requests of at most 6 qubits, their ops and
    results under "_small" (both popped before printing)."""
    import numpy as np
    from paper_2404_13184_gb300 import workloads
    arrivals = workloads.poisson_arrivals(rate, duration, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    srv = tq.Server(precision, rho_budget=rho_budget, table_budget=8 << 30, max_live=max_live)
    t0 = time.perf_counter()
    nxt = 0
    inflight = {}            # rid -> (arrival time, n, depth, ops or None)
    lat, done_n, completed, small = [], [], [], []
    queued_in_server = 0
    while True:
        now = time.perf_counter() - t0
        if now > duration + drain:
            break
        # at most one submission per tick, so planning a request overlaps the
        # tick running on the GPU
        if nxt < len(arrivals) and arrivals[nxt] <= now and queued_in_server < 8:
            c = workloads.served_request(rng)
            rid = srv.submit(c.n, c.ops, width=-1, masks=[1])
            inflight[rid] = (arrivals[nxt], c.n, c.n_gates, c.ops if c.n <= 6 else None)
            nxt += 1
            queued_in_server += 1
        if not inflight:
            if nxt >= len(arrivals):
                break
            time.sleep(max(0.0, min(arrivals[nxt] - now, 0.01)))
            continue
        # pipelined ticks: this call collects the previous tick and launches
        # the next, so building and submitting requests overlaps the GPU
        live, queued_in_server, fin = srv.step_async()
        if fin:
            tdone = time.perf_counter() - t0
            for rid in list(inflight):
                st, res = srv.poll(rid)
                if st == 2:
                    arr, n, d, ops = inflight.pop(rid)
                    lat.append(tdone - arr)
                    done_n.append(n)
                    completed.append((n, d))
                    if ops is not None and len(small) < keep_small:
                        small.append((n, ops, [float(v) for v in res]))
    wall = time.perf_counter() - t0
    end = wall
    censored = [end - a for a, _, _, _ in inflight.values()] + [end - a for a in arrivals[nxt:] if a <= end]
    info = srv.info()
    busy = srv.gpu_ms() / 1e3      # GPU time of the collected ticks (CUDA events)
    srv.free()
    lat_sorted = sorted(lat)

    def pct(v, q):
        return v[min(len(v) - 1, int(q * len(v)))] if v else None
    return {"precision": precision, "rate_per_s": rate, "arrival_window_s": duration, "drain_s": drain,
            "arrived": sum(1 for a in arrivals if a <= end), "completed": len(lat), "wall_s": wall,
            "circuits_per_s": len(lat) / wall, "p50_latency_s": pct(lat_sorted, 0.5),
            "p99_latency_s": pct(lat_sorted, 0.99), "censored": len(censored),
            "censored_min_latency_s": min(censored) if censored else None,
            "completed_qubit_counts": {str(k): done_n.count(k) for k in sorted(set(done_n))},
            "gpu_busy_frac": busy / wall, "ticks": info["ticks"], "blocks_applied": info["blocks_applied"],
            "sustainable_rate_per_s": len(lat) / max(busy, 1e-9), "_completed": completed, "_small": small}


def gate_slices(ops):
    """Split a served request's ops into per-gate lists (a gate and the
    channels attached after it)."""
    out = []
    for op in ops:
        if op[0] in ("depol", "ad", "pd", "thermal") and out:
            out[-1].append(op)
        else:
            out.append([op])
    return out


def plain_fp64_ms_per_gate(tq, torch, seed=SEED_SERVE, n_range=(5, 15), budget_s=2.0):
    """The plain FP64 path (tq_run_circuit with no fusion: every gate and
    every channel its own pass) on the served request distribution: per
    register size n, the first request of that size in the stream's own
    request sequence runs from |0><0|. Its first 10 gates (with their
    channels) run as one tq_run_circuit call plus a synchronising <Z_0>
    readout to estimate the rate; the next G gates, G chosen to take about
    `budget_s` seconds (at most the rest of the request), run the same way
    and are timed. Returns {n: (ms per noisy gate, gates timed)}: a request's
    plain time is its depth x that rate (each gate's cost depends only on
    its kind and n, and the kinds are drawn i.i.d.)."""
    import numpy as np
    from paper_2404_13184_gb300 import workloads
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    first = {}
    guard = 0
    while len(first) < n_range[1] - n_range[0] + 1 and guard < 100000:
        c = workloads.served_request(rng)
        first.setdefault(c.n, c)
        guard += 1
    out = {}
    for n in sorted(first):
        gates = gate_slices(first[n].ops)
        st = tq.State(n, "fp64")
        t0 = time.perf_counter()
        st.run([op for g in gates[:10] for op in g], width=0)
        st.expect_z([1])
        est = (time.perf_counter() - t0) / 10
        G = int(max(10, min(len(gates) - 10, budget_s / max(est, 1e-9))))
        ops = [op for g in gates[10:10 + G] for op in g]
        prog = tq.Program(ops)
        t0 = time.perf_counter()
        st.run(prog, width=0)
        st.expect_z([1])
        dt = time.perf_counter() - t0
        st.free()
        out[n] = (dt * 1e3 / G, G)
    torch.cuda.synchronize()
    return out


def served_vs_plain(serve: dict, plain: dict) -> dict:
    """The plain FP64 path's time for exactly the requests the server
    completed (depth x the measured ms per gate at their n), against the
    served run's wall time."""
    completed = serve["_completed"]
    t_plain = sum(d * plain[n][0] / 1e3 for n, d in completed)
    return {"plain_fp64_s_for_completed": t_plain, "plain_fp64_circuits_per_s": len(completed) / max(t_plain, 1e-9),
            "speedup_vs_plain_fp64": t_plain / serve["wall_s"]}


def run_plain6(tq, torch, steps, warmup, with_cpu=True):
    """6 qubits, 200 random noisy gates, FP64, no fusion (every gate and
    every channel is its own pass): the single-state device program (one
    launch per pass) and the batch engine (one resident CTA for the whole
    circuit, one persistent launch), per circuit run, with the difference of
    their <Z_i>."""
    from paper_2404_13184_gb300 import workloads
    c = workloads.plain_6q()
    out = {"noisy_gates": c.n_gates, "ops": len(c.ops)}
    st = tq.State(c.n, "fp64")
    prog = tq.DeviceProgram(c.n, c.ops, 0, "fp64")
    stream = torch.cuda.current_stream()
    for _ in range(max(1, warmup)):
        st.reset()
        st.run_program(prog)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(steps):
        st.reset()
        st.run_program(prog)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    z_gpu = list(st.expect_z([1 << q for q in range(c.n)]))
    out["program"] = {"ms_per_circuit": ms, "gates_per_s": c.n_gates / (ms / 1e3), "passes": prog.n_blocks}
    st.free()
    b = tq.Batch("fp64")
    b.add(c.n, c.ops, width=0, masks=[1 << q for q in range(c.n)])
    for _ in range(max(1, warmup)):
        b.run()
        b.wait()
    e0.record(stream)
    for _ in range(steps):
        b.run()
    e1.record(stream)
    b.wait()
    ms = e0.elapsed_time(e1) / steps
    z_b = list(b.result(0)[2:])
    b.free()
    out["batch_engine"] = {"ms_per_circuit": ms, "gates_per_s": c.n_gates / (ms / 1e3)}
    # the two GPU paths (different kernels, both held to the oracle by the tests)
    out["accuracy"] = {"max_abs_z_diff_program_vs_batch": max(abs(a - b) for a, b in zip(z_gpu, z_b))}
    if with_cpu:
        from oracle import dm_oracle
        reps, t0 = 0, time.perf_counter()
        while reps < 3 or time.perf_counter() - t0 < 2.0:
            dm_oracle.run_circuit(c.n, c.ops)
            reps += 1
        dt = (time.perf_counter() - t0) / reps
        out["cpu_baseline"] = {"value": c.n_gates / dt, "unit": "noisy gates/s", "ms_per_circuit": dt * 1e3,
                               "cores": 1, **host_cpu(), "kind": "oracle", "sample": f"the whole circuit, {reps} runs"}
    return out


def run_teleport(tq, precision):
    """Teleportation channel tomography (Sec. 5, Case Study-1) for the
    noiseless, device-like and 0.1-gate-error settings."""
    from paper_2404_13184_gb300 import case_studies as C
    names = ["noiseless", "device", "device_gate_error_0.1"]
    chis, _, ms = C.teleport_chi(tq, [C.NOISELESS, C.DEVICE, C.DEVICE_WORSE], precision)
    return {"batch_ms": ms, "jobs": 36, "settings": {
        nm: {"process_fidelity": C.process_fidelity(chi),
             "chi_re": [[round(float(v), 6) for v in row] for row in chi.real],
             "chi_im": [[round(float(v), 6) for v in row] for row in chi.imag]} for nm, chi in zip(names, chis)}}


def run_purify(tq, precision):
    """Two rounds of nested purification (Sec. 5, Case Study-2): output
    fidelity against input Werner fidelity for several CX error rates, and
    the band of inputs that purification improves."""
    from paper_2404_13184_gb300 import case_studies as C
    Fs = [round(0.5 + 0.025 * i, 3) for i in range(21)]
    ps = [0.0, 0.01, 0.03, 0.05, 0.07, 0.1]
    curves, ms = C.purification_curves(tq, Fs, ps, 2, precision)
    out = {"batch_ms": ms, "jobs": len(Fs) * len(ps), "qubits": 8, "curves": {}}
    for p in ps:
        better = [F for F, f, _ in curves[p] if f > F + 1e-12]
        out["curves"][str(p)] = {"F_out": [round(f, 6) for _, f, _ in curves[p]],
                                 "P_success": [round(s_, 6) for _, _, s_ in curves[p]],
                                 "improves_for_F_in": [min(better), max(better)] if better else None}
    out["F_in"] = Fs
    return out


def run_layered(tq, torch, precision, widths=(0, 1, 2, 3, 4), n=12, with_cpu=False, cpu_budget_s=20.0):
    """Layered thermal-relaxation workload (n = 12: 2^24 entries, 2000 gates):
    time of the whole circuit per fusion width (0 = unfused plain path) and
    the max-abs difference of <Z_i> and sampled vec(rho) entries to the
    unfused FP64 result."""
    import numpy as np
    from paper_2404_13184_gb300 import workloads
    c = workloads.layered_thermal(n=n)
    masks = [1 << q for q in range(n)]
    ref_z, ref_v, out = None, None, {}
    idx = np.random.default_rng(0).integers(0, 1 << (2 * n), 4096)
    for w in widths:
        prog = tq.DeviceProgram(n, c.ops, width=w, precision=precision)
        st = tq.State(n, precision)
        st.run_program(prog)                      # warm-up
        st.reset()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st.run_program(prog)
        z = st.expect_z(masks)
        dt = time.perf_counter() - t0
        v = st.vec()[idx]
        if ref_z is None:
            ref_z, ref_v = z, v
        out[str(w)] = {"blocks": prog.n_blocks, "ms": dt * 1e3, "gates_per_s": c.n_gates / dt,
                       "max_abs_z_diff_vs_unfused": float(np.max(np.abs(z - ref_z))),
                       "max_abs_rho_diff_vs_unfused": float(np.max(np.abs(v - ref_v)))}
        st.free()
        prog.free()
    base = out[str(widths[0])]["ms"]
    for w in out:
        out[w]["speedup_vs_unfused"] = base / out[w]["ms"]
    line = {"n_qubits": n, "noisy_gates": c.n_gates, "widths": out}
    if with_cpu:
        done, dt = oracle_prefix_time(n, c.ops, cpu_budget_s)
        est = dt * len(c.ops) / done
        line["cpu_baseline"] = {"value": c.n_gates / est, "unit": "noisy gates/s", "ms_per_circuit": est * 1e3,
                                "cores": 1, **host_cpu(), "kind": "oracle",
                                "sample": f"first {done} of the circuit's {len(c.ops)} ops (gates and channels), "
                                          f"{dt:.1f} s, time scaled by {len(c.ops)}/{done}"}
    return line


def extras(tq, torch, args, with_cpu):
    """The other configurations, at their stated sizes, as objects of the
    benchmark line: plain 6-qubit circuit (unfused FP64), layered 12-qubit
    thermal circuit (fusion widths 0-4, FP64 and split), the 1024-circuit
    sweep (FP64 and split) and the served Poisson stream (FP64 and split,
    with its speedup over the plain FP64 path and latency below saturation)."""
    import numpy as np
    out = {}
    out["plain6"] = run_plain6(tq, torch, max(args.steps, 20), args.warmup, with_cpu=with_cpu)
    out["layered12"] = {"n_qubits": 12, "fp64": run_layered(tq, torch, "fp64", with_cpu=with_cpu, cpu_budget_s=10.0),
                        "split": run_layered(tq, torch, "split")}
    sw = {}
    ref, oracle_results = None, None
    for prec in ("fp64", "split"):
        r = run_sweep(tq, torch, prec, 3, 1, reference=ref, with_cpu=with_cpu and prec == "fp64",
                      oracle_results=oracle_results)
        res = r.pop("results")
        oracle_results = r.pop("oracle_results")
        if prec == "fp64":
            ref = res
        sw[prec] = r
    out["sweep"] = {"circuits": 1024, "n_qubits": "4-11", "depth": "50-500", **sw}
    if args.serve_window > 0:
        sv = {}
        plain = plain_fp64_ms_per_gate(tq, torch)
        for prec in ("fp64", "split"):
            r = run_serve(tq, prec, args.serve_rate, args.serve_window, args.serve_drain_in_line,
                          keep_small=6 if with_cpu else 0)
            r.update(served_vs_plain(r, plain))
            small = r.pop("_small")
            r.pop("_completed")
            if with_cpu and small:
                # CPU-baseline leg: the oracle on a sample of the completed
                # small requests, for correctness only
                from oracle import dm_oracle
                errz, errt = 0.0, 0.0
                for n, ops, res in small:
                    rho = dm_oracle.run_circuit(n, ops)
                    errt = max(errt, abs(res[0] - float(np.trace(rho).real)))
                    errz = max(errz, abs(res[2] - float(dm_oracle.expect_z(rho, 1))))
                r["oracle_sample"] = {"requests": len(small), "max_abs_z_err": errz, "max_abs_trace_err": errt}
            sv[prec] = r
        sub = []
        for prec in ("fp64", "split"):
            cap = sv[prec]["sustainable_rate_per_s"]
            for f in (0.5, 0.8):
                r = run_serve(tq, prec, f * cap, 15.0, 15.0)
                for k in ("_small", "_completed"):
                    r.pop(k)
                sub.append({"precision": prec, "fraction_of_sustainable": f, **{k: r[k] for k in (
                    "rate_per_s", "arrived", "completed", "censored", "p50_latency_s", "p99_latency_s",
                    "circuits_per_s", "gpu_busy_frac")}})
        sv["sub_saturation"] = sub
        sv["plain_fp64_ms_per_gate"] = {str(n): {"ms_per_gate": v[0], "gates_timed": v[1]} for n, v in plain.items()}
        sv["speedup_vs_plain_fp64"] = {p_: sv[p_]["speedup_vs_plain_fp64"] for p_ in ("fp64", "split")}
        out["serve"] = sv
    return out


def reference_arm(args, world, rank):
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        cpu_sample_rate(1)
    total_gates, total_s = 0, 0.0
    for _ in range(args.steps):
        _, raw, dt = cpu_sample_rate(1)
        total_gates += 2
        total_s += dt
    raw = total_gates / total_s
    value = raw * 4.0 ** (-(N_QUBITS - SAMPLE_QUBITS))
    sample = (f"per step: RZZ+2q depolarising and RX+1q depolarising of the ring TFIM on a {SAMPLE_QUBITS}-qubit "
              f"register, rate scaled by 4^-{N_QUBITS - SAMPLE_QUBITS} to 15 qubits (oracle cost per op ~ 4^n)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "tfim-ring-15q", "n_qubits": N_QUBITS},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, **host_cpu(), "kind": "oracle",
                             "sample": sample, "raw_value_at_sample_size": raw},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="tanq", choices=["tanq", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-split", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=None, help="timed steps of the FP64 leg (default --steps)")
    ap.add_argument("--n-qubits", type=int, default=15, help="register size (15 for the benchmark; smaller "
                    "registers for profiling captures)")
    ap.add_argument("--workload", default="tfim15",
                    choices=["tfim15", "sweep", "serve", "layered12", "plain6", "teleport", "purify"],
                    help="tfim15: the benchmark line; sweep / serve: the batched-sweep and served-stream workloads")
    ap.add_argument("--precision", default="both", choices=["fp64", "split", "both"], help="sweep / serve modes")
    ap.add_argument("--sweep-count", type=int, default=1024)
    ap.add_argument("--sweep-qubits", type=str, default="4-11", help="qubit range of the sweep, e.g. 4-11")
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-duration", type=float, default=60.0)
    ap.add_argument("--serve-drain", type=float, default=60.0)
    ap.add_argument("--serve-window", type=float, default=60.0,
                    help="arrival window (s) of the served streams added to the tfim15 line (0: none)")
    ap.add_argument("--serve-drain-in-line", type=float, default=20.0,
                    help="drain window (s) after the in-line served streams' arrivals stop")
    ap.add_argument("--fp64-engine", default="auto", choices=["auto", "dfma", "tensor"],
                    help="products of the FP64 apply passes (tq_set_fp64_engine; the sweep mode's batch: "
                         "tq_batch_set_fp64_engine)")
    ap.add_argument("--no-dfma-leg", action="store_true",
                    help="leave out the DFMA-engine comparison when the FP64 leg runs on the tensor cores")
    ap.add_argument("--no-extras", action="store_true",
                    help="tfim15 line only: leave out the plain6, layered12, sweep and serve objects")
    args = ap.parse_args()
    global N_QUBITS
    N_QUBITS = args.n_qubits
    if args.warmup < 3 and args.impl != "reference":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return reference_arm(args, world, rank)

    import torch
    import torch.distributed as dist
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2404_13184_gb300 import binding as tq
    tq.load()
    hbm_gbs, sm_max_cfg, peak_src = peaks()
    gpu_index = local
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis and vis.split(",")[0].strip().isdigit():
        gpu_index = int(vis.split(",")[local].strip())

    if args.workload == "layered12":
        precs = ["fp64", "split"] if args.precision == "both" else [args.precision]
        for i, prec in enumerate(precs):
            r = run_layered(tq, torch, prec, with_cpu=i == 0 and rank == 0 and not args.no_cpu_baseline)
            if rank == 0:
                print(json.dumps({"metric": "layered thermal circuit: time per fusion width", "workload":
                                  "layered-thermal-12q-2000g", "dtype": "f64" if prec == "fp64" else "f32", **r}),
                      flush=True)
        return 0
    if args.workload == "plain6":
        r = run_plain6(tq, torch, max(args.steps, 20), args.warmup, with_cpu=rank == 0 and not args.no_cpu_baseline)
        if rank == 0:
            print(json.dumps({"metric": "plain 6-qubit circuit, unfused: noisy gates/s", "workload":
                              "plain-6q-200g (FP64, no fusion)", "dtype": "f64", **r}), flush=True)
        return 0
    if args.workload in ("teleport", "purify"):
        precs = ["fp64", "split"] if args.precision == "both" else [args.precision]
        for prec in precs:
            r = run_teleport(tq, prec) if args.workload == "teleport" else run_purify(tq, prec)
            if rank == 0:
                print(json.dumps({"metric": f"case study: {args.workload}", "dtype": "f64" if prec == "fp64" else "f32",
                                  **r}), flush=True)
        return 0
    if args.workload in ("sweep", "serve"):
        precs = ["fp64", "split"] if args.precision == "both" else [args.precision]
        fp64_results = None
        for prec in precs:
            if args.workload == "sweep":
                lo, hi = (int(v) for v in args.sweep_qubits.split("-"))
                r = run_sweep(tq, torch, prec, args.steps, args.warmup, count=args.sweep_count, n_min=lo, n_max=hi,
                              reference=fp64_results if prec == "split" else None,
                              with_cpu=prec == precs[0] and rank == 0 and not args.no_cpu_baseline,
                              engine=args.fp64_engine)
                res = r.pop("results")
                r.pop("oracle_results")
                if prec == "fp64":
                    fp64_results = res
                line = {"metric": "batched sweep circuits/s",
                        "workload": f"sweep-{args.sweep_count} (n {lo}-{hi}, depth 50-500)",
                        "dtype": "f64" if prec == "fp64" else "f32", **r}
            else:
                r = run_serve(tq, prec, args.serve_rate, args.serve_duration, args.serve_drain)
                for k in ("_small", "_completed"):
                    r.pop(k)
                line = {"metric": "served circuits/s + p99 latency", "workload": "poisson-served (n 5-15, depth "
                        "50-2000)", "dtype": "f64" if prec == "fp64" else "f32", **r}
            if rank == 0:
                print(json.dumps(line), flush=True)
        return 0

    K, W = args.steps, args.warmup
    K64 = args.fp64_steps or K
    gates_per_step = 2 * N_QUBITS
    # pipe rates first, on a GPU that has not been loaded yet, with the clocks
    # sampled while the probes run
    clk_p = Clocks(gpu_index)
    clk_p.start()
    pipes = {p_: measured_pipe(tq, p_) for p_ in ("dfma", "dmma", "ffma", "cvt_f64_s64", "cvt_f64_f32")}
    pipes_clk = clk_p.stop()
    fp64 = run_device_leg(tq, torch, "fp64", K64, W, world, Clocks(gpu_index), engine=args.fp64_engine)
    split = None if args.no_split else run_device_leg(tq, torch, "split", K, W, world)
    e2e_ms = None if args.no_e2e else run_e2e_leg(tq, torch, "fp64", K64, W, world, engine=args.fp64_engine)

    ms64 = max_over_ranks(fp64["ms"], world)
    value = job_throughput(K64 * gates_per_step, ms64, world)
    clk = fp64["clocks"] or {}
    sm_mhz = clk.get("sm_mhz") or sm_max_cfg
    sms = device_sms()
    name64, st64 = dominant(fp64["stats"])
    roof = fp64_roofline(name64, st64, pipes, sm_max_cfg, sm_mhz, sms, hbm_gbs, peak_src)
    dfma_leg = None
    if fp64["on_tensor"] and not args.no_dfma_leg:
        # the same step on the DFMA engine (tq_run_circuit, planned for it):
        # its apply passes beside the tensor-core ones
        k_d = max(3, K64 // 4)
        ms_d, st_d, zz_d = run_e2e_leg(tq, torch, "fp64", k_d, W, world, engine="dfma", profile=True)
        nd, sd = dominant(st_d)
        # both legs start from |0..0> and run W untimed steps first: timed
        # step i of this leg is step W + i of the device leg
        ref_zz = fp64["zz"][W:]
        n_cmp = min(len(zz_d), len(ref_zz))
        dfma_leg = {"value": job_throughput(k_d * gates_per_step, max_over_ranks(ms_d, world), world), "unit": UNIT,
                    "ms_per_step": ms_d / k_d, "steps": k_d, "api": "tq_run_circuit (host tables)",
                    "zz_max_abs_diff_vs_tensor_engine": max(abs(a - b) for a, b in zip(zz_d[:n_cmp], ref_zz[:n_cmp])),
                    "roofline": fp64_roofline(nd, sd, pipes, sm_max_cfg, sm_mhz, sms, hbm_gbs, peak_src),
                    "kernels": {k: {"launches": v["launches"], "avg_ms": round(v["total_ms"] / v["launches"], 4)}
                                for k, v in st_d.items() if k.startswith("apply")}}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K64, "warmup": W,
            "ms_per_step": ms64 / K64, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"tfim-ring-{N_QUBITS}q: per step {N_QUBITS} x (RZZ(0.2) + 2q depolarising 5e-4) "
                                   f"on the ring and {N_QUBITS} x (RX(0.1) + 1q depolarising 5e-4), <Z0 Z1> after "
                                   "each step",
                       "n_qubits": N_QUBITS, "rho_bytes": 16 << (2 * N_QUBITS), "fusion": "auto",
                       "precision": "fp64 (split path in the 'split' object)",
                       "fp64_blocks_per_step": fp64["blocks"], "fp64_max_width": fp64["max_width"],
                       "l2": "inputs larger than L2 (16 GiB rho), no flush", "parallelism": "replicas"
                       if world > 1 else "single"},
            "roofline": roof, "gpu_launches": fp64["launches"],
            "fp64_engine": "tensor (tcgen05, fixed-point digit slicing)" if fp64["on_tensor"] else "dfma",
            "pipes_measured": {"dfma_tflops": pipes["dfma"], "dmma_tflops": pipes["dmma"], "ffma_tflops": pipes["ffma"],
                               "cvt_f64_s64_tops": pipes["cvt_f64_s64"], "cvt_f64_f32_tops": pipes["cvt_f64_f32"],
                               "how": "tq_pipe_rate: 8 independent chains per thread, 4 x 256 threads per SM on "
                                      "every SM, best of 3 launches (CUDA events)", "clocks": pipes_clk},
            "clocks": {"sm_mhz": clk.get("sm_mhz"), "sm_max_mhz": clk.get("sm_max_mhz"),
                       "reasons": clk.get("reasons", []), "samples": clk.get("samples")},
            "kernels": {k: {"launches": v["launches"], "total_ms": round(v["total_ms"], 3)}
                        for k, v in fp64["stats"].items()}}
    if dfma_leg is not None:
        line["fp64_dfma"] = dfma_leg
    if e2e_ms is not None:
        e2e_ms = max_over_ranks(e2e_ms, world)
        line["e2e"] = {"value": job_throughput(K64 * gates_per_step, e2e_ms, world), "unit": UNIT,
                       "h2d_bytes_per_step": fp64["table_bytes"] + 8, "d2h_bytes_per_step": 3 * 8,
                       "ms_per_step": e2e_ms / K64}
    if split is not None:
        mss = max_over_ranks(split["ms"], world)
        vs = job_throughput(K * gates_per_step, mss, world)
        ns, ss = dominant(split["stats"])
        ach = ss["bytes"] * ss["launches"] / (ss["total_ms"] / 1e3) / 1e9
        n_cmp = min(len(split["zz"]), len(fp64["zz"]))
        err = max(abs(a - b) for a, b in zip(split["zz"][:n_cmp], fp64["zz"][:n_cmp]))
        line["split"] = {"value": vs, "unit": UNIT, "ms_per_step": mss / K, "steps": K, "dtype": "f32",
                         "speedup_vs_fp64": vs / value, "blocks_per_step": split["blocks"],
                         "max_width": split["max_width"], "zz_max_abs_err_vs_fp64": err,
                         "accuracy_8q": split_accuracy(tq),
                         "roofline": {"kernel": ns, "bound": "hbm", "achieved": ach, "peak": hbm_gbs, "unit": "GB/s",
                                      "frac": ach / hbm_gbs, "traffic": traffic_from_profile(ns),
                                      "algorithmic_bytes_per_launch": ss["bytes"], "launches": ss["launches"],
                                      "avg_launch_ms": ss["total_ms"] / ss["launches"],
                                      "peak_source": f"{peak_src} HBM copy bandwidth"},
                         "gpu_launches": split["launches"]}
    with_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    if split is not None:
        acc = line["split"]["accuracy_8q"]
        z64, z32 = acc.pop("_zz64"), acc.pop("_zz32")
        if with_cpu:
            zo = oracle_tfim_zz(acc["qubits"], acc["steps"])
            acc["fp64_zz_max_abs_err_vs_oracle"] = max(abs(a - b) for a, b in zip(z64, zo))
            acc["split_zz_max_abs_err_vs_oracle"] = max(abs(a - b) for a, b in zip(z32, zo))
    if world == 1 and not args.no_extras:
        line.update(extras(tq, torch, args, with_cpu))
    if with_cpu:
        scaled, raw, dt = cpu_sample_rate(2)
        line["cpu_baseline"] = {"value": scaled, "unit": UNIT, "cores": 1, **host_cpu(), "kind": "oracle",
                                "sample": f"2 x (RZZ+2q depolarising, RX+1q depolarising) of the ring TFIM on a "
                                          f"{SAMPLE_QUBITS}-qubit register ({dt:.1f} s, {raw:.3g} gates/s), scaled by "
                                          f"4^-{N_QUBITS - SAMPLE_QUBITS} to 15 qubits (oracle cost per op ~ 4^n)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
