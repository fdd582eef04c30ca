#!/usr/bin/env python
"""Benchmark of stage 2 of the two-stage Hessenberg-triangular reduction on GB300.

Metric: stage-2 GFLOP/s, FP64-equivalent with the paper's operation count for stage 2
(10 n^3 including Q and Z), plus the backward error, on one n = 8192, r = 16 pencil.

One step = one full stage-2 reduction (all sweeps, all kernels) of a seeded synthetic
r-Hessenberg-triangular pencil (A with 16 subdiagonals, B the R factor of a Gaussian matrix),
with Q and Z accumulated.  The inputs (1 GiB for A and B) are larger than L2, and each step
restores A and B from pristine device copies before the timed call.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--mode emu|fp64]

``--mode`` selects the arithmetic of the delayed updates: ``emu`` (default) forms each block's
reflector product and applies it in FP64 emulated on the BF16 tensor cores, ``fp64`` applies
the reflectors one at a time in native FP64; the chase is native FP64 in both.
``--impl reference`` times the CPU oracle (Alg. 2 in plain C, OpenMP) on the host cores:
each step is a bounded sample (the first sweeps) of the same workload.
``--workload reduce|batch`` time the full reduction and the many-pencil case (supplementary
lines); ``--workload probe`` runs two untimed stage-2 calls for profiler captures.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "stage-2 GFLOP/s (FP64-equiv) + backward error at n=8192,r=16 on 1 GB300"
UNIT = "GFLOP/s"
N_DEFAULT, R_DEFAULT, SEED = 8192, 16, 4
MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
# the sources a kernel's DRAM figure depends on (besides hts_internal.cuh)
KERNEL_SOURCES = {"k_s2_generate": ("chase.cu", "schedule.cuh"), "k_s2_chase16": ("chase16.cu", "schedule.cuh"),
                  "k_s2_apply_right": ("stage2.cu",), "k_s2_apply_left": ("stage2.cu",),
                  "k_s2_emu_apply_right": ("emu.cu",), "k_s2_emu_apply_left": ("emu.cu",),
                  "k_s2_emu_apply_qz": ("emu.cu",), "k_s2_form_u": ("emu.cu",),
                  "k_s2_update": ("emu_tc.cu", "schedule.cuh", "emu_arith.cuh", "right_window.cuh")}


def paper_flops(n):
    """Paper's stage-2 operation count with Q and Z: 10 n^3 (Section "Unblocked stage two")."""
    return 10.0 * float(n) ** 3


def chase_critical_steps(n, r, q):
    """Steps on the chase's critical path, summed over the groups, under the kernel's waits:
    step (k, j) follows step (k-1, j), and sweep j-1's block k+2 (or its last block).  With
    unit steps, fin_j(k) = k + 1 + max_{i <= k} (fin_{j-1}(min(i+2, K_{j-1}-1)) - i), where
    K_j = 2 + (n-j-1) // r are the blocks sweep j walks (Alg. 3)."""
    total = 0
    for j1 in range(1, n - 1, q):
        qg = min(q, n - 2 - j1 + 1)
        prev = None
        for s in range(qg):
            K = 2 + (n - (j1 + s) - 1) // r
            k = np.arange(K)
            if prev is None:
                fin = k + 1
            else:
                dep = prev[np.minimum(k + 2, len(prev) - 1)]
                fin = k + 1 + np.maximum.accumulate(dep - k)
            prev = fin
        total += int(prev[-1])
    return total


def chase_floor_ms(n, r, q, mhz):
    """Latency floor of the chase: the steps on each group's critical path
    (chase_critical_steps) times the dependent chain of one step.  Per step (r = 16 kernel):
    r - 1 rows of the pivoted elimination at 332 cycles each, the measured latencies of a
    row's chain on this GPU (a DMUL and a DFMA, 64 each; the integer pivot search, 112; a
    shared load, 29; a shuffle, 37; the barrier, 26), and 105 dependent FP64 instructions of
    64 cycles: 24 each for Q^ and Z^, 18 for the band update and 39 for the last sweep's
    aggregated lazy updates."""
    chain = (r - 1) * 332 + (2 * 24 + 18 + 39) * 64
    return chase_critical_steps(n, r, q) * chain / (mhz * 1e3)


def sweep_work(n, r):
    """Direct flop count of each sweep of Alg. 2 (4 flops per element and reflector), used to
    scale a bounded oracle sample to its share of the whole stage."""
    w = np.zeros(n + 1)
    for j in range(1, n - 1):
        nb = 1 + (n - j - 2) // r
        k = np.arange(nb)
        jb = j + np.maximum(0, (k - 1) * r + 1)
        i1 = j + k * r + 1
        i2 = np.minimum(j + (k + 1) * r, n)
        i3 = np.minimum(j + (k + 2) * r, n)
        m = i2 - i1 + 1
        w[j] = float(np.sum(4 * m * ((n - jb) + (n - i1 + 1) + n + i3 + i2 + n)))
    return w


# ---------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(self.NAMES, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------------------
def log(msg):
    sys.stderr.write("[bench] %s\n" % msg)
    sys.stderr.flush()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# The profiling recipe's fallback denominators, used only while MEASURED_PEAKS.json is absent:
# a copy at 6.8 TB/s and cuBLAS BF16 at 1.9 PFLOP/s (burst) / 1.7 PFLOP/s (sustained), one
# earlier measurement on a GB300.
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "source": "fallback"}


def measured_peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            d = json.load(f)
        d.setdefault("source", "measured")
        return d
    except (OSError, ValueError):
        return dict(FALLBACK_PEAKS)


def source_digest(fnames):
    csrc = os.path.join(ROOT, "paper_2301_07964_gb300", "csrc")
    h = hashlib.sha256()
    for p in sorted(os.path.join(csrc, f) for f in tuple(fnames) + ("hts_internal.cuh",)):
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload):
    """DRAM bytes per launch from the committed ncu summary, or None when the summary is
    missing or was taken on a different version of the kernel's source."""
    try:
        lines = open(TRAFFIC_FILE).read().splitlines()
    except OSError:
        return None
    digest = source_digest(KERNEL_SOURCES.get(kernel, ("stage2.cu",)))
    for ln in lines:
        parts = ln.split()
        if len(parts) >= 4 and not ln.startswith("#") and parts[0] == kernel and parts[1] == workload:
            if parts[3] == digest:
                return float(parts[2])
    return None


def cpu_sample(A, B, r, budget_s):
    """Time the oracle on the first sweeps of stage 2 (bounded sample).  Returns
    (GFLOP/s in the paper's convention, seconds, sweeps, share of the stage, threads)."""
    import oracle
    n = A.shape[0]
    w = sweep_work(n, r)
    total = w.sum()
    hs_of = lambda s: int(sum(2 * (1 + (n - j - 2) // r) for j in range(1, s + 1)))
    t0 = time.perf_counter()
    oracle.stage2(A, B, r, max_half_steps=hs_of(2))
    t_cal = max(time.perf_counter() - t0, 1e-3)
    s = int(max(2, min(n - 2, 2 * budget_s / t_cal)))
    t0 = time.perf_counter()
    oracle.stage2(A, B, r, max_half_steps=hs_of(s))
    t = time.perf_counter() - t0
    share = float(w[1:s + 1].sum() / total)
    return paper_flops(n) * share / t / 1e9, t, s, share, oracle.threads()


# ---------------------------------------------------------------------------------------
# reference arm: the CPU oracle
# ---------------------------------------------------------------------------------------
def run_reference(args, n, r):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2301_07964_gb300.inputs import random_rht_pencil
    oracle.build()
    A, B = random_rht_pencil(n, r, SEED)
    w = sweep_work(n, r)
    total = w.sum()
    s = int(args.ref_sweeps)
    hs = int(sum(2 * (1 + (n - j - 2) // r) for j in range(1, s + 1)))
    share = float(w[1:s + 1].sum() / total)
    for _ in range(args.warmup):
        oracle.stage2(A, B, r, max_half_steps=hs)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.stage2(A, B, r, max_half_steps=hs)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    value = paper_flops(n) * share / t / 1e9
    sample = ("first %d of %d sweeps of the n=%d r=%d pencil (%.2f%% of stage-2 work), Q and Z "
              "accumulated, scaled by that share" % (s, n - 2, n, r, 100 * share))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "stage 2, n=%d r=%d, seeded r-HT pencil, Q and Z accumulated" % (n, r),
                   "n": n, "r": r},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------
def chase_floor(prof, n, r, q, clk, steps):
    """The chase's time against its dependent-FP64-chain floor (chase_floor_ms)."""
    name = "k_s2_chase16" if r <= 16 else "k_s2_generate"
    if name not in prof or r > 16:
        return None
    mhz = (clk or {}).get("sm_mhz") or 2070.0
    floor = chase_floor_ms(n, r, q, mhz)
    ms = prof[name]["ms"] / steps
    return {"kernel": name, "floor_ms": floor, "measured_ms": ms, "frac": floor / ms, "sm_mhz": mhz,
            "model": "critical-path steps x the measured latency of one step's dependent chain"}


def run_ours(args, n, r):
    import torch
    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_2301_07964_gb300 import binding as b
    from paper_2301_07964_gb300 import build
    from paper_2301_07964_gb300.device import Reducer, colmajor_empty, to_device
    from paper_2301_07964_gb300.inputs import random_rht_pencil
    if rank == 0 or not os.path.exists(build.LIB_PATH):
        build.build()
    if dist is not None:
        dist.barrier()
    b.load()

    mode = b.HTS_GEMM_FP64 if args.mode == "fp64" else b.HTS_GEMM_EMU_BF16
    sched_flags = b.HTS_FLAG_SERIAL_UPDATES if args.serial else 0
    red = Reducer(local)
    tile_m = args.tile_m
    tile_source = "given on the command line" if tile_m else "the library's default (64-line tcgen05 tiles)"
    if args.q:
        q, q_source = args.q, "given on the command line"
    elif args.tune:
        from paper_2301_07964_gb300 import tune
        path = os.path.join(tempfile.mkdtemp(), "tune.json")
        tuned = tune.tuned_stage2(red, n, r, mode, seed=SEED + 1, cache_path=path, reps=1, retune=True)
        q = tuned["q"]
        if not args.tile_m:
            tile_m = tuned["tile_m"]
            tile_source = "measured by tune.tuned_stage2"
        q_source = "measured by tune.tuned_stage2 on another seeded pencil of this size (ms per call: %s)" % (
            json.dumps(tuned["ms"]))
    else:
        q, q_source = r, "the library's default q = r (tune.tuned_q measured it fastest at n = 8192, r = 16)"
    A, B = random_rht_pencil(n, r, SEED)
    dA0, dB0 = to_device(A), to_device(B)
    dA, dB = colmajor_empty(n), colmajor_empty(n)
    dQ, dZ = colmajor_empty(n), colmajor_empty(n)
    stream = torch.cuda.current_stream()
    fp64_peak = b.hts_probe_fp64_peak(stream)

    def one_step(m=mode):
        dA.copy_(dA0)
        dB.copy_(dB0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        red.stage2(dA, dB, r, dQ, dZ, compq=b.HTS_COMP_INIT, compz=b.HTS_COMP_INIT, q=q, mode=m,
                   flags=sched_flags, stream=stream, tile_m=tile_m)
        e1.record(stream)
        return e0, e1

    for i in range(args.warmup):
        e0, e1 = one_step()
        torch.cuda.synchronize()
        log("warm-up step %d: %.1f ms" % (i, e0.elapsed_time(e1)))
    torch.cuda.synchronize()
    st, info = red.sync_status()
    if st != b.HTS_OK:
        raise SystemExit("device error during warm-up: %s %s" % (b.status_string(st), info))

    launches_per_step = (6 if args.mode == "emu" else 4) * ((n - 2 + q - 1) // q) + 4
    b.hts_profile_begin(red.ctx, launches_per_step * args.steps + 16)
    clocks = ClockSampler(local)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    events = [one_step() for _ in range(args.steps)]
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    prof, dropped = b.hts_profile_end(red.ctx)
    if r <= 16 and "k_s2_generate" in prof:   # the chase kernel for r <= 16
        prof["k_s2_chase16"] = prof.pop("k_s2_generate")
    st, info = red.sync_status()
    if st != b.HTS_OK:
        raise SystemExit("device error during timed steps: %s %s" % (b.status_string(st), info))
    step_ms = [e0.elapsed_time(e1) for e0, e1 in events]
    ms = sum(step_ms) / len(step_ms)
    log("timed steps (ms): %s; profile: %s" % (step_ms, json.dumps(prof)))
    if dist is not None:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())

    # end to end through the public API with host buffers, right after the timed steps (before
    # the backward-error products and the native steps, whose FP64 load would leave the GPU
    # hotter for these samples), with its own clock record
    e2e = None
    if not args.no_e2e:
        hA = torch.from_numpy(np.ascontiguousarray(A.T)).pin_memory()   # row-major of A^T = col-major A
        hB = torch.from_numpy(np.ascontiguousarray(B.T)).pin_memory()
        outs = [torch.empty((n, n), dtype=torch.float64).pin_memory() for _ in range(4)]
        e2e_ms = []
        e2e_clocks = ClockSampler(local)
        e2e_clocks.start()
        for _ in range(max(1, args.e2e_steps)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dA.t().copy_(hA, non_blocking=True)
            dB.t().copy_(hB, non_blocking=True)
            red.stage2(dA, dB, r, dQ, dZ, compq=b.HTS_COMP_INIT, compz=b.HTS_COMP_INIT, q=q, mode=mode,
                       flags=sched_flags, stream=stream, tile_m=tile_m)
            for o, d in zip(outs, (dA, dB, dQ, dZ)):
                o.copy_(d.t(), non_blocking=True)
            torch.cuda.synchronize()
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
        e2e_clk = e2e_clocks.stop()
        st, info = red.sync_status()
        if st != b.HTS_OK:
            raise SystemExit("device error during e2e steps: %s %s" % (b.status_string(st), info))
        e2e_t = sum(e2e_ms) / len(e2e_ms)
        if dist is not None:
            t = torch.tensor([e2e_t], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            e2e_t = float(t.item())
        e2e = {"value": ws * paper_flops(n) / (e2e_t / 1e3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 2 * 8 * n * n, "d2h_bytes_per_step": 4 * 8 * n * n,
               "ms_per_step": e2e_t, "samples": len(e2e_ms), "sample_ms": e2e_ms, "clocks": e2e_clk}

    # backward error of the last step (outside the timed region; residuals by cuBLAS DGEMM)
    def backward_error():
        H, T, Qm, Zm = dA, dB, dQ, dZ
        I = torch.eye(n, dtype=torch.float64, device="cuda")
        be = {
            "A": float(torch.linalg.norm(Qm @ H @ Zm.T - dA0) / torch.linalg.norm(dA0)),
            "B": float(torch.linalg.norm(Qm @ T @ Zm.T - dB0) / torch.linalg.norm(dB0)),
            "orth_Q": float(torch.linalg.norm(Qm.T @ Qm - I) / n ** 0.5),
            "orth_Z": float(torch.linalg.norm(Zm.T @ Zm - I) / n ** 0.5),
            "H_below_subdiag_max": float(torch.tril(H, -2).abs().max()),
            "T_below_diag_max": float(torch.tril(T, -1).abs().max()),
        }
        del I
        return be

    bwd = backward_error()

    # the same step with native FP64 delayed updates (the precision comparison of the
    # metric's configuration 4), outside the timed region of the line's value
    fp64_record = None
    if args.mode == "emu" and args.fp64_steps > 0 and ws == 1:
        one_step(b.HTS_GEMM_FP64)
        torch.cuda.synchronize()
        ev = [one_step(b.HTS_GEMM_FP64) for _ in range(args.fp64_steps)]
        torch.cuda.synchronize()
        st, info = red.sync_status()
        if st != b.HTS_OK:
            raise SystemExit("device error during FP64 steps: %s %s" % (b.status_string(st), info))
        f_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
        fm = sum(f_ms) / len(f_ms)
        fp64_record = {"mode": "fp64", "steps": args.fp64_steps, "warmup": 1, "ms_per_step": fm,
                       "value": paper_flops(n) / (fm / 1e3) / 1e9, "unit": UNIT, "step_ms": f_ms,
                       "backward_error": backward_error()}

    # roofline of the dominant kernel: FP64 kernels against the live FP64 peak, the emulated
    # kernels (BF16 tensor-core work) against the measured sustained BF16 peak
    peaks = measured_peaks()
    dom = max(prof.items(), key=lambda kv: kv[1]["ms"])
    kname, kp = dom
    workload = "n%d_r%d_q%d_%s" % (n, r, q, args.mode)
    traffic = ncu_traffic(kname, workload)
    if kp.get("mma_flops", 0.0) > 0.0:
        bf16 = peaks["bf16_tflops_sustained"]
        achieved = kp["mma_flops"] / (kp["ms"] / 1e3) / 1e12
        roofline = {"kernel": kname, "bound": "tensor", "achieved": achieved, "peak": bf16, "unit": "TFLOP/s",
                    "frac": achieved / bf16, "traffic": traffic,
                    "peak_source": "bf16_tflops_sustained (of %s)" % peaks["source"],
                    "algorithmic_flops_per_launch": kp["mma_flops"] / kp["launches"],
                    "algorithmic_bytes_per_launch": kp["bytes"] / kp["launches"],
                    "avg_launch_ms": kp["ms"] / kp["launches"]}
    else:
        achieved = kp["flops"] / (kp["ms"] / 1e3) / 1e12
        roofline = {"kernel": kname, "bound": "alu", "achieved": achieved, "peak": fp64_peak,
                    "unit": "TFLOP/s", "frac": achieved / fp64_peak,
                    "traffic": traffic,
                    "peak_source": "FP64 FMA throughput measured live by hts_probe_fp64_peak (of measured)",
                    "algorithmic_flops_per_launch": kp["flops"] / kp["launches"],
                    "algorithmic_bytes_per_launch": kp["bytes"] / kp["launches"],
                    "avg_launch_ms": kp["ms"] / kp["launches"]}
    # the delayed-update launches (tensor cores in emu mode) against the measured BF16 peak
    roofline_update = None
    ku = prof.get("k_s2_update")
    if ku and ku.get("mma_flops", 0.0) > 0.0:
        bf16 = peaks["bf16_tflops_sustained"]
        au = ku["mma_flops"] / (ku["ms"] / 1e3) / 1e12
        roofline_update = {"kernel": "k_s2_update", "bound": "tensor", "achieved": au, "peak": bf16,
                           "unit": "TFLOP/s", "frac": au / bf16, "traffic": ncu_traffic("k_s2_update", workload),
                           "peak_source": "bf16_tflops_sustained (of %s)" % peaks["source"],
                           "algorithmic_flops_per_launch": ku["mma_flops"] / ku["launches"],
                           "algorithmic_bytes_per_launch": ku["bytes"] / ku["launches"],
                           "avg_launch_ms": ku["ms"] / ku["launches"],
                           "hbm_frac": (ku["bytes"] / (ku["ms"] / 1e3) / 1e9) / peaks["hbm_gbs"]
                           if peaks.get("hbm_gbs") else None}
    kernels = {k: {"launches": v["launches"], "ms_per_step": v["ms"] / args.steps,
                   "share": v["ms"] / max(1e-9, sum(x["ms"] for x in prof.values())),
                   "tflops": v["flops"] / max(1e-9, v["ms"] / 1e3) / 1e12,
                   "mma_tflops": v.get("mma_flops", 0.0) / max(1e-9, v["ms"] / 1e3) / 1e12,
                   "gbs": v["bytes"] / max(1e-9, v["ms"] / 1e3) / 1e9}
               for k, v in prof.items()}

    line = {
        "metric": METRIC, "value": ws * paper_flops(n) / (ms / 1e3) / 1e9, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "stage 2, n=%d r=%d q=%d, seeded r-HT pencil (A band iid N(0,1), B = R of "
                               "a Gaussian), Q and Z accumulated, delayed updates %s" % (n, r, q, args.mode),
                   "n": n, "r": r, "q": q, "mode": args.mode, "parallelism": "replicas" if ws > 1 else "single",
                   "q_source": q_source,
                   "schedule": "serial" if args.serial else "look-ahead",
                   "update_tiles": tile_m or "library default", "update_tiles_source": tile_source,
                   "l2": "inputs (A, B: %.1f GiB) larger than L2" % (2 * 8 * n * n / 2 ** 30)},
        "backward_error": bwd,
        "fp64_updates": fp64_record,
        "direct_gflops": ws * 8.0 * n ** 3 / (ms / 1e3) / 1e9,
        "clocks": clk,
        "e2e": e2e,
        "gpu_launches": int(sum(v["launches"] for v in prof.values())),
        "profile_dropped": dropped,
        "roofline": roofline,
        "roofline_update": roofline_update,
        "chase_floor": chase_floor(prof, n, r, q, clk, args.steps),
        "kernels": kernels,
        "hbm_peak_gbs": peaks.get("hbm_gbs"),
        "peaks_source": peaks["source"],
        "wall_s_timed": t_wall,
    }
    log(json.dumps(line))
    if ws == 1 and rank == 0 and not args.no_cpu:
        v, t, s, share, cores = cpu_sample(A, B, r, args.cpu_seconds)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": "first %d of %d sweeps of the same pencil (%.2f%% of stage-2 work) "
                                          "in %.1f s, Q and Z accumulated, scaled by that share" %
                                          (s, n - 2, 100 * share, t)}
    if rank == 0:
        print(json.dumps(line))
    red.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------------------
# supplementary workloads (not the metric line): full reduction and the batch configuration
# ---------------------------------------------------------------------------------------
def run_reduce(args, n, r):
    """Full reduction (QR of B, stage 1, stage 2) of a dense pencil: A, B iid N(0, 1), B
    ill-conditioned (--ill), or the saddle-point pencil with a quarter of the eigenvalues
    infinite (--saddle)."""
    import torch
    from paper_2301_07964_gb300 import binding as b
    from paper_2301_07964_gb300 import build
    from paper_2301_07964_gb300.device import Reducer, colmajor_empty, to_device
    from paper_2301_07964_gb300.inputs import ill_conditioned_pencil, random_pencil, saddle_point_pencil
    build.build()
    b.load()
    seed = args.seed if args.seed is not None else 2
    if args.ill:
        A, B = ill_conditioned_pencil(n, seed)
    elif args.saddle:
        A, B = saddle_point_pencil(n, seed)
    else:
        A, B = random_pencil(n, seed)
    dA0, dB0 = to_device(A), to_device(B)
    dA, dB, dQ, dZ = (colmajor_empty(n) for _ in range(4))
    red = Reducer(0)
    stream = torch.cuda.current_stream()
    mode = b.HTS_GEMM_FP64 if args.mode == "fp64" else b.HTS_GEMM_EMU_BF16
    p, p_source = args.p, ("given on the command line" if args.p else "the library's default min(8, 128 / r)")
    if args.tune and not args.p:
        from paper_2301_07964_gb300 import tune
        path = os.path.join(tempfile.mkdtemp(), "tune.json")
        p = tune.tuned_stage1_p(red, n, r, mode, seed=seed + 1, cache_path=path, retune=True)
        p_source = "measured by tune.tuned_stage1_p on another seeded pencil of this size (ms per call: %s)" % (
            json.dumps(next(iter(tune.load_cache(path).values()))["ms"]))

    def step():
        dA.copy_(dA0)
        dB.copy_(dB0)
        red.reduce(dA, dB, r, dQ, dZ, compq=b.HTS_COMP_INIT, compz=b.HTS_COMP_INIT, q=args.q, p=p, stream=stream,
                   mode=mode)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    b.hts_profile_begin(red.ctx, 8 * n + 64)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    prof, _ = b.hts_profile_end(red.ctx)
    st, info = red.sync_status()
    assert st == b.HTS_OK, info
    ms = e0.elapsed_time(e1) / args.steps
    I = torch.eye(n, dtype=torch.float64, device="cuda")
    bwd = {"A": float(torch.linalg.norm(dQ @ dA @ dZ.T - dA0) / torch.linalg.norm(dA0)),
           "B": float(torch.linalg.norm(dQ @ dB @ dZ.T - dB0) / torch.linalg.norm(dB0)),
           "orth_Q": float(torch.linalg.norm(dQ.T @ dQ - I) / n ** 0.5),
           "orth_Z": float(torch.linalg.norm(dZ.T @ dZ - I) / n ** 0.5)}
    s01 = prof.get("stage1", {}).get("ms", 0.0) / args.steps
    if args.saddle:
        # T = Q^T B Z is triangular with the rank m = n - n/8 of B: n/8 vanishing diagonal entries
        dT = torch.sort(torch.diagonal(dB).abs()).values
        bwd["T_diag_zeros_at_least"] = n // 8
        bwd["T_diag_below_1e-12n"] = int((dT < 1e-12 * n).sum())
    kind = " ill-conditioned B" if args.ill else (" saddle point (n/4 infinite eigenvalues)" if args.saddle else "")
    print(json.dumps({"workload": "full reduction n=%d r=%d%s, delayed updates %s" % (n, r, kind, args.mode), "p": p,
                      "p_source": p_source,
                      "ms_per_step": ms, "stage01_ms": s01, "stage2_ms": ms - s01,
                      "gflops_two_stage_21.33n3": 21.33 * n ** 3 / (ms / 1e3) / 1e9,
                      "gflops_stage2_10n3": paper_flops(n) / ((ms - s01) / 1e3) / 1e9,
                      "backward_error": bwd, "steps": args.steps,
                      "kernels": {k: {"ms_per_step": v["ms"] / args.steps, "launches": v["launches"] // args.steps}
                                  for k, v in prof.items()}}))
    red.close()
    return 0


def run_probe(args, n, r):
    """Two untimed stage-2 calls on the metric's pencil family at size n, for profiler
    captures of single launches (no timing, no output besides a status line)."""
    import torch
    from paper_2301_07964_gb300 import binding as b
    from paper_2301_07964_gb300 import build
    from paper_2301_07964_gb300.device import Reducer, colmajor_empty, to_device
    from paper_2301_07964_gb300.inputs import random_rht_pencil
    build.build()
    b.load()
    q = args.q or r
    mode = b.HTS_GEMM_FP64 if args.mode == "fp64" else b.HTS_GEMM_EMU_BF16
    A, B = random_rht_pencil(n, r, SEED)
    red = Reducer(0)
    for _ in range(2):
        dA, dB = to_device(A), to_device(B)
        dQ, dZ = colmajor_empty(n), colmajor_empty(n)
        red.stage2(dA, dB, r, dQ, dZ, compq=b.HTS_COMP_INIT, compz=b.HTS_COMP_INIT, q=q, mode=mode,
                   flags=b.HTS_FLAG_SERIAL_UPDATES if args.serial else 0, tile_m=args.tile_m)
        st, info = red.sync_status()
        if st != b.HTS_OK:
            raise SystemExit("device error: %s %s" % (b.status_string(st), info))
    torch.cuda.synchronize()
    red.close()
    print(json.dumps({"workload": "probe", "n": n, "r": r, "q": q, "mode": args.mode, "status": "ok"}))
    return 0


def run_batch(args):
    """4096 pencils, n uniform in [32, 512], r = min(8, n // 8), A, B iid N(0, 1), full
    reduction with Q and Z in one hts_reduce_batched launch."""
    import torch
    from paper_2301_07964_gb300 import binding as b
    from paper_2301_07964_gb300 import build
    from paper_2301_07964_gb300.device import Reducer, colmajor_empty
    from paper_2301_07964_gb300.inputs import batch_sizes
    build.build()
    b.load()
    count = args.count
    ns, rs = batch_sizes(count, 5)
    ns, rs = [int(x) for x in ns], [int(x) for x in rs]
    gen = torch.Generator(device="cuda")
    gen.manual_seed(5)
    A0 = [torch.randn(n, n, dtype=torch.float64, device="cuda", generator=gen).t() for n in ns]
    B0 = [torch.randn(n, n, dtype=torch.float64, device="cuda", generator=gen).t() for n in ns]
    dA = [colmajor_empty(n) for n in ns]
    dB = [colmajor_empty(n) for n in ns]
    dQ = [colmajor_empty(n) for n in ns]
    dZ = [colmajor_empty(n) for n in ns]
    red = Reducer(0)
    nbytes = b.hts_workspace_size_batched(ns, rs)
    work = torch.empty(max(256, nbytes), dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def restore():
        for x, y in zip(dA, A0):
            x.copy_(y)
        for x, y in zip(dB, B0):
            x.copy_(y)

    params, shape_source = None, "the library's defaults (p = min(8, 64 / r_i), as many blocks per SM as fit)"
    if args.tune:
        from paper_2301_07964_gb300 import tune
        path = os.path.join(tempfile.mkdtemp(), "tune.json")
        tuned = tune.tuned_batch(red, ns, rs, seed=6, cache_path=path, reps=1, retune=True)
        params = {"p": tuned["p"], "tile_n": tuned["tile_n"]}
        shape_source = "measured by tune.tuned_batch on another seeded batch of these sizes (ms per call: %s)" % (
            json.dumps(tuned["ms"]))
    # the batch is planned once (descriptors and order into the workspace); every step is one
    # planned launch, and the same launch is also timed as a CUDA graph replay
    st = b.hts_plan_batched(red.ctx, ns, rs, dA, ns, dB, ns, b.HTS_COMP_INIT, dQ, ns, b.HTS_COMP_INIT, dZ, ns,
                            b.HTS_GEMM_FP64, params, work, work.numel(), stream)
    assert st == b.HTS_OK, b.status_string(st)

    def timed(launch):
        times = []
        for it in range(args.warmup + args.steps):
            restore()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            launch()
            e1.record(stream)
            torch.cuda.synchronize()
            if it >= args.warmup:
                times.append(e0.elapsed_time(e1))
        st, info = red.sync_status()
        assert st == b.HTS_OK, info
        return sum(times) / len(times)

    def planned():
        assert b.hts_reduce_batched_planned(red.ctx, count, work, work.numel(), stream) == b.HTS_OK

    ms = timed(planned)
    graph = torch.cuda.CUDAGraph()
    torch.cuda.synchronize()
    with torch.cuda.graph(graph):
        assert b.hts_reduce_batched_planned(red.ctx, count, work, work.numel(), torch.cuda.current_stream()) == b.HTS_OK
    ms_graph = timed(graph.replay)
    flops = sum(21.33 * n ** 3 for n in ns)
    print(json.dumps({"workload": "batch of %d pencils, n uniform in [32, 512], r = min(8, n // 8), full "
                                  "reduction with Q, Z, one persistent launch (planned once)" % count,
                      "ms_per_batch": ms, "pencils_per_s": count / (ms / 1e3),
                      "gflops_two_stage_21.33n3": flops / (ms / 1e3) / 1e9,
                      "graph_replay_ms_per_batch": ms_graph, "steps": args.steps,
                      "launch": params or "library defaults", "launch_source": shape_source}))
    red.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--mode", choices=["fp64", "emu"], default="emu")
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--r", type=int, default=R_DEFAULT)
    ap.add_argument("--q", type=int, default=0)
    ap.add_argument("--serial", action="store_true",
                    help="stage 2: each group's delayed updates after its chase (no look-ahead)")
    ap.add_argument("--tile-m", type=int, default=0, choices=[0, 32, 64],
                    help="emulated update tiles: 64 lines (tcgen05), 32 (mma.sync), 0 the library's choice")
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=2,
                    help="emu mode: also time this many steps with native FP64 updates (0: skip)")
    ap.add_argument("--tune", action="store_true",
                    help="measure the launch parameters before timing: q and the update tiles (stage 2), "
                         "stage 1's p (--workload reduce), p and blocks per SM (--workload batch)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-sweeps", type=int, default=24)
    ap.add_argument("--workload", choices=["stage2", "reduce", "batch", "probe"], default="stage2")
    ap.add_argument("--ill", action="store_true", help="reduce: ill-conditioned B")
    ap.add_argument("--saddle", action="store_true", help="reduce: saddle-point pencil")
    ap.add_argument("--p", type=int, default=0, help="reduce: stage 1's blocks per panel step (0: the default)")
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--count", type=int, default=4096)
    args = ap.parse_args()
    if args.workload == "reduce":
        return run_reduce(args, args.n, args.r)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "probe":
        return run_probe(args, args.n, args.r)
    if args.impl == "reference":
        return run_reference(args, args.n, args.r)
    return run_ours(args, args.n, args.r)


if __name__ == "__main__":
    sys.exit(main())
