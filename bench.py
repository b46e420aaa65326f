#!/usr/bin/env python
"""Benchmark: FP64-accuracy dense product C = A*B at M = N = K = 8192 on GB300.

One step = one FP64-accuracy product through the library (exponent scan,
slicing of both operands, tcgen05 slice products and exact recombination) on
inputs resident in HBM: A with entries uniform[-1,1)*2^e (e uniform on
[-20, 20] per row), B likewise per column. Inputs are 2 x 512 MiB, larger
than the 129 MB L2, so no flush is needed between steps.

Reported beside the headline value (all measured in this run): the plain FP64
kernel and the FP32-accuracy mode on the same inputs, the FP64 pipe peak, the
end-to-end figure through the host-buffer entry point, the dominant kernel's
roofline, SM clocks sampled during the timed region, and the CPU oracle on a
bounded row sample (which also gives the measured error of the sampled rows).

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]
Under torchrun each rank runs its own replica of the product (replicas only:
the single product is not sharded across GPUs); value = all ranks' flops over
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_DEFAULT = 8192
METRIC = "FP64-accuracy GEMM TFLOP/s, emulated vs plain FP64, N=8192; serve p50/p99 ms"
WORKLOAD = "split-precision FP64-accuracy GEMM M=N=K=8192, A uniform[-1,1)*2^e per row, B per column, e in [-20,20]"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons while running."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []          # csv lines, each stamped by nvidia-smi (wall clock of this host)
        self.window = None       # (t0, t1) of the timed region

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "50", "-i", str(self.idx)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def mark(self, t0: float, t1: float):
        self.window = (t0, t1)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        import datetime

        def stamp(ln):
            try:
                ts = ln.split(",")[0].strip()
                return datetime.datetime.strptime(ts, "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                return None

        lines = self.lines
        scope = "all samples"
        if self.window is not None:
            inside = [ln for ln in lines if (stamp(ln) or -1.0) >= self.window[0] and (stamp(ln) or -1.0) <= self.window[1]]
            if inside:
                lines, scope = inside, "timed region"
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")][1:]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm), "scope": scope,
                "power_w_median": statistics.median(power) if power else None}


# ---------------------------------------------------------------- helpers
def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


SLICE_GEMM_SOURCES = ("slice_gemm_kernel.cuh", "slice_gemm.cu", "slice_gemm_fold.cu", "slice_gemm_carry.cu",
                      "slice_gemm_crt.cu")


def code_of(text: str) -> str:
    """C++ source without comments, trailing spaces and blank lines (what the
    compiler sees), so a comment edit leaves the code hash unchanged."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
    return "\n".join(ln for ln in lines if ln)


def slice_gemm_source_hash() -> str:
    """sha256[:16] over the code of the slice GEMM's kernel header and sources,
    in order, comments removed."""
    h = hashlib.sha256()
    for name in SLICE_GEMM_SOURCES:
        with open(os.path.join(ROOT, "paper_2408_15384_gb300", "csrc", name)) as f:
            h.update(code_of(f.read()).encode())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the slice GEMM from the committed ncu summary,
    if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "slice_gemm_fp64emu_traffic.md")
    if not os.path.exists(path):
        return None, None
    txt = open(path).read()
    src_hash = slice_gemm_source_hash()
    m_hash = re.search(r"source sha256\[:16\]:\s*`?([0-9a-f]{16})", txt)
    m_bytes = re.search(r"bytes per launch at N=8192:\s*`?([0-9.eE+]+)", txt)
    if not m_hash or not m_bytes or m_hash.group(1) != src_hash:
        return None, src_hash
    return float(m_bytes.group(1)), src_hash


def workload_config(N: int, ws: int) -> dict:
    """The workload both arms report (the oracle arm runs a row sample of it)."""
    return {"workload": WORKLOAD, "m": N, "n": N, "k": N, "accuracy": "fp64",
            "l2": "inputs 2 x 512 MiB > 129 MB L2 (no flush)", "parallelism": f"replicas x{ws}"}


def slowest_rank_ms(t_ms: float, dist, dev) -> float:
    """The timed region's length on the slowest rank (every rank gets it)."""
    if dist is None:
        return t_ms
    import torch
    tt = torch.tensor([t_ms], dtype=torch.float64, device=dev)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_tflops(world_size: int, flop_per_product: float, steps: int, t_ms: float) -> float:
    """Every rank runs its own replica of the product (replicas only): the job's
    throughput is all ranks' flops over the slowest rank's time."""
    return world_size * flop_per_product * steps / (t_ms * 1e-3) / 1e12


def median_ci(xs, conf: float = 0.95):
    """(median, lo, hi): the sample median and the distribution-free interval of
    order statistics [x_(j), x_(n+1-j)] that covers the population median with
    probability >= conf (binomial(n, 1/2) counts), the widest j reaching it."""
    xs = sorted(xs)
    n = len(xs)
    if n == 0:
        return None, None, None
    med = statistics.median(xs)
    lo, hi = xs[0], xs[-1]
    for j in range(1, n // 2 + 1):
        cover = sum(math.comb(n, i) for i in range(j, n + 1 - j)) / 2.0 ** n
        if cover < conf:
            break
        lo, hi = xs[j - 1], xs[n - j]
    return med, lo, hi


def event_times(stream, reps, fn):
    """Device time (ms) of each of `reps` calls of fn(), CUDA events on `stream`."""
    import torch
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
    ev[0].record(stream)
    for i in range(reps):
        fn()
        ev[i + 1].record(stream)
    ev[-1].synchronize()
    return [ev[i].elapsed_time(ev[i + 1]) for i in range(reps)]


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- CPU oracle leg
def cpu_oracle_rows(A, B, seconds: float, max_rows: int):
    """Time the oracle's OpenMP triple loop (the paper's threaded scheme) on a
    bounded number of rows of the product; returns (rows, C_rows, seconds, threads)."""
    import oracle
    oracle.build()
    # one row per thread first, to size the sample
    _, used = oracle.gemm_omp_rows(A, B, 0, 1)
    t0 = time.perf_counter()
    _, used = oracle.gemm_omp_rows(A, B, 0, used)
    t1 = time.perf_counter() - t0
    reps = int(max(1, min(max_rows // used, seconds / max(t1, 1e-6))))
    rows = reps * used
    t0 = time.perf_counter()
    Cr, used = oracle.gemm_omp_rows(A, B, 0, rows)
    dt = time.perf_counter() - t0
    return rows, Cr, dt, used


def reference_arm(args):
    """The oracle (test infrastructure) timed as it stands on the host cores."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    from paper_2408_15384_gb300 import inputs
    import oracle
    oracle.build()
    N = args.n
    A = inputs.row_scaled(N, N, 3)
    B = inputs.col_scaled(N, N, 3)
    per_step = max(2.0, 150.0 / max(1, args.steps + args.warmup))
    rows, _, _, used = cpu_oracle_rows(A, B, per_step, 512)
    for _ in range(args.warmup):
        oracle.gemm_omp_rows(A, B, 0, rows)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.gemm_omp_rows(A, B, 0, rows)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    tflops = 2.0 * rows * N * N / t / 1e12
    line = {
        "impl": "reference", "metric": METRIC, "value": tflops, "unit": "TFLOP/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(N, ws),
        "cpu_baseline": {"value": tflops, "unit": "TFLOP/s", "cores": used, "kind": "oracle",
                         "sample": f"{rows} rows of the {N}^3 product per step (2*{rows}*{N}*{N} flop), "
                                   f"OpenMP triple loop on {used} host threads"},
        "e2e": {"value": tflops, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU arm
def ours(args):
    import numpy as np
    import torch
    import paper_2408_15384_gb300 as mm
    from paper_2408_15384_gb300 import inputs

    ws, rank, local = dist_env()
    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    N = args.n
    h = mm.Handle(local, budget_bytes=40 << 30)
    stream = torch.cuda.current_stream(dev)

    seed = 3 + 1000 * rank
    A = torch.empty((N, N), dtype=torch.float64, device=dev)
    B = torch.empty_like(A)
    C = torch.empty_like(A)
    mm.fill_uniform(A, seed, inputs.STREAM_A, 1, inputs.STREAM_EXP_A)
    mm.fill_uniform(B, seed, inputs.STREAM_B, 2, inputs.STREAM_EXP_B)
    # the form the device decides for these inputs: the modular form (one
    # residue product per modulus) or the digit form (s(s+1)/2 digit pairs)
    _, code, bits, _, _, _ = h.debug_fp64_product(A, B, C, residues=False)
    if code > mm.CRT_BASE:
        s, pairs = None, code - mm.CRT_BASE
        form = {"form": "modular (Chinese remainder)", "moduli": pairs, "bits": bits, "products": pairs}
    else:
        s = code
        pairs = s * (s + 1) // 2
        form = {"form": "digits", "slices": s, "products": pairs}
    flop = 2.0 * N ** 3

    def barrier():
        if dist is not None:
            dist.barrier()

    # ---------------- timed region: FP64-accuracy products
    for _ in range(max(args.warmup, 3)):
        h.gemm(A, B, C, precision=mm.FP64_EMU)
    torch.cuda.synchronize(dev)
    h.set_option(mm.OPT_PROFILE, 1)
    for kcls in (mm.KERNEL_SLICE_GEMM, mm.KERNEL_SPLIT, mm.KERNEL_REBUILD):
        h.profile_read(kcls, reset=True)
    launches0 = h.stats()
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(local)
    sampler = ClockSampler(gpu_id)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    tw0 = time.time()
    ev[0].record(stream)
    for i in range(args.steps):
        h.gemm(A, B, C, precision=mm.FP64_EMU, stream=stream)
        ev[i + 1].record(stream)
    torch.cuda.synchronize(dev)
    tw1 = time.time()
    barrier()
    sampler.mark(tw0, tw1)
    clocks = sampler.stop()
    t_ms = ev[0].elapsed_time(ev[-1])
    step_ms = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    med, lo, hi = median_ci(step_ms)
    launches = h.stats() - launches0
    status = h.sync()
    gemm_ms, gemm_n = h.profile_read(mm.KERNEL_SLICE_GEMM, reset=True)
    split_ms, split_n = h.profile_read(mm.KERNEL_SPLIT, reset=True)
    rebuild_ms, _ = h.profile_read(mm.KERNEL_REBUILD, reset=True)
    h.set_option(mm.OPT_PROFILE, 0)
    t_ms = slowest_rank_ms(t_ms, dist, dev)
    ms_step = t_ms / args.steps
    value = whole_job_tflops(ws, flop, args.steps, t_ms)

    # ---------------- dominant kernel roofline (tensor pipe, bf16)
    peaks = measured_peaks()
    # slice-GEMM device time per product: the launch that ran plus the launches
    # for the other candidate counts, which return at once
    kernel_ms = gemm_ms / max(args.steps, 1)
    slice_flop = flop * pairs
    achieved = slice_flop / (kernel_ms * 1e-3) / 1e12
    # the kernel runs at full clock in a sub-second region: the burst peak
    if "bf16_tflops" in peaks:
        peak, peak_note = peaks["bf16_tflops"], "of measured (bf16 burst)"
    else:
        peak, peak_note = 1900.0, "of fallback (bf16 burst)"
    traffic, src_hash = profiled_traffic()

    extra = {}
    if rank == 0 and not args.quick:
        # ---------------- the other modes on the same inputs (outside the timed region)
        def time_mode(prec, reps):
            h.gemm(A, B, C, precision=prec)
            torch.cuda.synchronize(dev)
            ts = event_times(stream, reps, lambda: h.gemm(A, B, C, precision=prec, stream=stream))
            m_, l_, u_ = median_ci(ts)
            return m_, {"median": m_, "lo": l_, "hi": u_, "n": reps}

        fp32_ms, fp32_ci = time_mode(mm.FP32_EMU, 15)
        fp64_ms, fp64_ci = time_mode(mm.FP64, 15)
        # the digit form on the same inputs, for comparison
        h.set_option(mm.OPT_FP64_SCHEME, 1)
        try:
            dig_ms, dig_ci = time_mode(mm.FP64_EMU, 15)
            dig_s = h.debug_slice_count(A, B)[0]
        finally:
            h.set_option(mm.OPT_FP64_SCHEME, 0)
        # the INT8 digit form on the legacy integer tensor path, for comparison
        h.set_option(mm.OPT_INT8_SLICES, 1)
        try:
            int8_ms, int8_ci = time_mode(mm.FP64_EMU, 3)
        finally:
            h.set_option(mm.OPT_INT8_SLICES, 0)
        dfma, dmma = h.peak_fp64()
        fp64_peak = max(dfma, dmma)
        extra["modes"] = {
            "fp64_emu_tflops": flop / (ms_step * 1e-3) / 1e12,
            "fp32_emu_tflops": flop / (fp32_ms * 1e-3) / 1e12,
            "plain_fp64_tflops": flop / (fp64_ms * 1e-3) / 1e12,
            "fp32_emu_ms_median_ci95": fp32_ci, "plain_fp64_ms_median_ci95": fp64_ci,
            "fp64_emu_int8_mma_sync_tflops": flop / (int8_ms * 1e-3) / 1e12, "fp64_emu_int8_ms_median_ci95": int8_ci,
            "emu_over_plain": fp64_ms / ms_step,
            "fp64_peak_tflops_measured": {"dfma": dfma, "dmma": dmma},
            "plain_fp64_frac_of_fp64_peak": (flop / (fp64_ms * 1e-3) / 1e12) / fp64_peak,
            "fp64_form": form,
            "fp64_emu_digit_form_tflops": flop / (dig_ms * 1e-3) / 1e12, "fp64_emu_digit_form_ms_median_ci95": dig_ci,
            "digit_form_slices": dig_s, "digit_form_pairs": dig_s * (dig_s + 1) // 2,
        }
        # ---------------- the configurations' other sizes: plain FP64 sweep and the
        # split-precision product at 4096, median and interval of 15 reps each
        extra["config_sweep"] = config_sweep_leg(h, args, mm, inputs, torch, dev, stream)
        # ---------------- end to end through the host-buffer entry point
        Ah = torch.empty((N, N), dtype=torch.float64, pin_memory=True)
        Bh = torch.empty_like(Ah, pin_memory=True)
        Ch = torch.empty_like(Ah, pin_memory=True)
        Ah.copy_(A.cpu())
        Bh.copy_(B.cpu())
        An, Bn, Cn = Ah.numpy(), Bh.numpy(), Ch.numpy()
        h.gemm_host(An, Bn, Cn, precision=mm.FP64_EMU)
        reps = max(1, min(3, args.steps))
        t0 = time.perf_counter()
        for _ in range(reps):
            h.gemm_host(An, Bn, Cn, precision=mm.FP64_EMU)
        e2e_s = (time.perf_counter() - t0) / reps
        # the copies alone on this machine, for context (a pinned buffer of their
        # own: the product's result in Ch is checked against the oracle below)
        Ad2 = torch.empty_like(A)
        Xh = torch.empty_like(Ah, pin_memory=True)
        torch.cuda.synchronize(dev)
        c0 = time.perf_counter()
        Ad2.copy_(Ah, non_blocking=True)
        torch.cuda.synchronize(dev)
        c1 = time.perf_counter()
        Xh.copy_(Ad2, non_blocking=True)
        torch.cuda.synchronize(dev)
        c2 = time.perf_counter()
        del Ad2, Xh
        extra["e2e"] = {"value": flop / e2e_s / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": 16 * N * N,
                        "d2h_bytes_per_step": 8 * N * N,
                        "ms_per_step": e2e_s * 1e3,
                        "copy_gbs": {"h2d": 8 * N * N / (c1 - c0) / 1e9, "d2h": 8 * N * N / (c2 - c1) / 1e9,
                                     "note": "one 512 MiB pinned copy each way"}}
        # ---------------- the paper's own sizes and inputs (Sec. IV), every mode
        if not args.no_paper_sweep:
            extra["paper_sweep"] = paper_sweep_leg(h, args, mm, inputs, torch, dev, stream)
        # ---------------- grouped: 512 products, dims log-uniform on [32, 1024], one graph replay each
        if not args.no_grouped:
            extra["grouped"] = grouped_leg(h, args, mm, inputs, torch, dev, stream, fp64_peak)
        # ---------------- serving: capacity (closed loop), then Poisson arrivals at 80 % of it
        if not args.no_serve:
            extra["serve"] = serve_leg(h, args, mm, inputs)
        # ---------------- CPU oracle on a bounded sample, and the measured error of those rows
        if not args.no_cpu_baseline:
            rows, Cr, dt, used = cpu_oracle_rows(An, Bn, args.cpu_seconds, 2048)
            import oracle
            from oracle import emulation as em
            D = oracle.absprod_rows_par(An, Bn, list(range(min(rows, 8))))
            got = Cn[:min(rows, 8)]
            ref = Cr[:min(rows, 8)]
            ratio = float(np.max(np.abs(got - ref) / (em.gamma(N, "fp64") * D)))
            # every mode's result at N on 64 sampled rows and 64 sampled columns
            def sample64(seed):
                picked = {0, N - 1}
                for v in inputs.int_uniform(0, N - 1, 256, seed, inputs.STREAM_DIMS):
                    if len(picked) >= 64:
                        break
                    picked.add(int(v))
                return sorted(picked)
            srows, scols = sample64(31), sample64(32)
            r_ref, r_D = oracle.gemm_rows_par(An, Bn, srows), oracle.absprod_rows_par(An, Bn, srows)
            Bc = np.ascontiguousarray(Bn[:, scols])
            c_ref = oracle.gemm_rows_par(An, Bc, list(range(N)))
            c_D = oracle.absprod_rows_par(An, Bc, list(range(N)))
            errs = {}
            for prec, name in ((mm.FP64_EMU, "fp64_emu"), (mm.FP32_EMU, "fp32_emu"), (mm.FP64, "plain_fp64")):
                errs[name] = sampled_error(h, mm, torch, A, B, C, prec, stream, srows, r_ref, r_D, scols, c_ref, c_D)
            extra["modes"]["max_err_over_bound"] = errs
            extra["modes"]["err_sample"] = f"{len(srows)} rows and {len(scols)} columns of each {N}^3 product vs the oracle"
            extra["cpu_baseline"] = {"value": 2.0 * rows * N * N / dt / 1e12, "unit": "TFLOP/s", "cores": used,
                                     "kind": "oracle",
                                     "sample": f"{rows} rows of the {N}^3 product by the OpenMP triple loop "
                                               f"({dt:.1f} s, {os.cpu_count()} host cores)"}
            # the paper's two CPU optimisations of the loop (Sec. III), on a smaller row sample
            variants = {}
            rv = max(used, rows // 4)
            for name, fn in (("column_prefetch", oracle.gemm_colprefetch_rows), ("cache_tiled", oracle.gemm_tiled_rows)):
                t0 = time.perf_counter()
                Cv, uv = fn(An, Bn, 0, rv)
                dv = time.perf_counter() - t0
                variants[name] = {"value": 2.0 * rv * N * N / dv / 1e12, "unit": "TFLOP/s", "cores": uv,
                                  "rows": rv, "same_bits_as_oracle": bool(np.array_equal(Cv[:min(rv, rows)],
                                                                                         Cr[:min(rv, rows)]))}
            extra["cpu_variants"] = variants
            extra["max_abs_err"] = float(np.max(np.abs(got - ref)))
            extra["max_err_over_bound"] = ratio
            extra["err_sample"] = f"{min(rows, 8)} rows x {N} columns vs the FP64 triple-loop oracle"

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "bf16", "data": "synthetic",
            "config": workload_config(N, ws),
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic, "peak_note": peak_note,
                         "kernel": ("slice_gemm (tcgen05 bf16 residue products; the epilogue stores the sums "
                                    "modulo each modulus, C is rebuilt by a pass of its own)" if s is None else
                                    "slice_gemm (tcgen05 bf16 slice products, FP64-accuracy epilogue)"),
                         "kernel_ms": kernel_ms, "algorithmic": f"2*N^3*{pairs} slice flop per launch",
                         "fp64_form": form},
            "step_ms_median_ci95": {"median": med, "lo": lo, "hi": hi, "n": args.steps,
                                    "tflops_at_median": flop / (med * 1e-3) / 1e12 if med else None,
                                    "method": "order-statistic interval of the per-step device times (CUDA events)"},
            "split_kernels_ms_per_step": split_ms / max(args.steps, 1),
            "rebuild_kernel_ms_per_step": rebuild_ms / max(args.steps, 1),
            "clocks": clocks, "gpu_launches": launches, "device_status": status,
        }
        line.update(extra)
        if "e2e" not in line:
            line["e2e"] = None
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


# The paper's best serial times (GCC -O3, Sec. VI table, Cirrus Xeon E5-2695
# at 2.1 GHz, mean of 15 runs): context for the sweep below, not a target.
PAPER_SERIAL_GCC_O3_S = {32: 0.00003, 64: 0.00026, 128: 0.00228, 256: 0.02028, 512: 0.17037, 1024: 1.69891}


def paper_sweep_leg(h, args, mm, inputs, torch, dev, stream):
    """The paper's sizes (32 .. 1024, Sec. IV) with its Box-Muller normal
    entries, through every mode: median device time of 15 products (the paper
    averages 15 runs) and, with the CPU leg on, the error of every output
    against the oracle."""
    import numpy as np
    out = {"inputs": "Box-Muller normal deviates from two seeded unit draws (Sec. IV)", "sizes": {},
           "slice_count": "automatic (decided on the device from the rows' and columns' spread)"}
    names = {mm.FP64: "fp64", mm.FP64_EMU: "fp64_emu", mm.FP32_EMU: "fp32_emu"}
    for N in sorted(PAPER_SERIAL_GCC_O3_S):
        A = inputs.box_muller(N, N, 7 + N, inputs.STREAM_A)
        B = inputs.box_muller(N, N, 7 + N, inputs.STREAM_B)
        Ad, Bd = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
        Cd = torch.empty((N, N), dtype=torch.float64, device=dev)
        row = {"paper_serial_gcc_O3_s": PAPER_SERIAL_GCC_O3_S[N]}
        ref = D = None
        if not args.no_cpu_baseline:
            import oracle
            ref, D = oracle.gemm(A, B), oracle.absprod(A, B)
        for prec, name in names.items():
            h.gemm(Ad, Bd, Cd, precision=prec, stream=stream)
            torch.cuda.synchronize(dev)
            ts = []
            for _ in range(15):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                h.gemm(Ad, Bd, Cd, precision=prec, stream=stream)
                e1.record(stream)
                e1.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            row[name + "_s"] = ms * 1e-3
            row[name + "_gflops"] = 2.0 * N ** 3 / (ms * 1e-3) / 1e9
            if ref is not None:
                from oracle import emulation as em
                row[name + "_max_err_over_bound"] = float(np.max(np.abs(Cd.cpu().numpy() - ref) / (em.gamma(N, name) * D)))
        row["fp64_emu_slices"] = h.debug_slice_count(Ad, Bd)[0]
        out["sizes"][str(N)] = row
    return out


def sampled_error(h, mm, torch, A, B, C, prec, stream, rows, ref_rows, D_rows, cols=None, ref_cols=None, D_cols=None):
    """max |C - C_oracle| / (gamma |A||B|) over the sampled rows (and columns) of one mode's product."""
    import numpy as np
    from oracle import emulation as em
    h.gemm(A, B, C, precision=prec, stream=stream)
    torch.cuda.synchronize()
    mode = {mm.FP64: "fp64", mm.FP64_EMU: "fp64_emu", mm.FP32_EMU: "fp32_emu"}[prec]
    g = em.gamma(A.shape[1], mode)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = float(np.nanmax(np.abs(C[rows].cpu().numpy() - ref_rows) / (g * D_rows)))
        if cols is not None:
            r = max(r, float(np.nanmax(np.abs(C[:, cols].cpu().numpy() - ref_cols) / (g * D_cols))))
    return r


def config_sweep_leg(h, args, mm, inputs, torch, dev, stream):
    """The configurations' sizes besides the headline: plain FP64 at 1024, 2048
    and 4096 on uniform[-1,1) entries, and the split-precision workload at 4096
    in all three modes; each the median and 95 % interval of 15 timed products
    (the paper's 15 repetitions, Sec. V) and, with the CPU leg on, the measured
    error of 16 sampled rows against the oracle."""
    out = {}
    cases = [("plain_fp64", n, False, mm.FP64) for n in (1024, 2048, 4096)]
    cases += [("split_" + nm, 4096, True, p) for nm, p in (("fp64_emu", mm.FP64_EMU), ("fp32_emu", mm.FP32_EMU),
                                                          ("plain_fp64", mm.FP64))]
    cache = {}
    for name, N, scaled, prec in cases:
        key = (N, scaled)
        if key not in cache:
            seed = 3 if scaled else 2 + int(math.log2(N))
            A = torch.empty((N, N), dtype=torch.float64, device=dev)
            B = torch.empty_like(A)
            if scaled:
                mm.fill_uniform(A, seed, inputs.STREAM_A, 1, inputs.STREAM_EXP_A)
                mm.fill_uniform(B, seed, inputs.STREAM_B, 2, inputs.STREAM_EXP_B)
            else:
                mm.fill_uniform(A, seed, inputs.STREAM_A)
                mm.fill_uniform(B, seed, inputs.STREAM_B)
            ref = None
            if not args.no_cpu_baseline:
                import oracle
                An, Bn = A.cpu().numpy(), B.cpu().numpy()
                rows = sorted({int(r) for r in inputs.int_uniform(0, N - 1, 14, seed, inputs.STREAM_DIMS)} | {0, N - 1})
                ref = (rows, oracle.gemm_rows_par(An, Bn, rows), oracle.absprod_rows_par(An, Bn, rows))
            cache = {key: (A, B, torch.empty_like(A), ref)}
        A, B, C, ref = cache[key]
        h.gemm(A, B, C, precision=prec, stream=stream)
        torch.cuda.synchronize(dev)
        ts = event_times(stream, 15, lambda: h.gemm(A, B, C, precision=prec, stream=stream))
        med, lo, hi = median_ci(ts)
        row = {"n": N, "ms_median": med, "ms_ci95": [lo, hi], "reps": 15,
               "tflops_at_median": 2.0 * N ** 3 / (med * 1e-3) / 1e12,
               "inputs": "uniform[-1,1)*2^e per row/column" if scaled else "uniform[-1,1)"}
        if ref is not None:
            row["max_err_over_bound"] = sampled_error(h, mm, torch, A, B, C, prec, stream, ref[0], ref[1], ref[2])
            row["err_sample"] = f"{len(ref[0])} rows x {N} columns"
        out[f"{name}_{N}"] = row
    return out


def grouped_leg(h, args, mm, inputs, torch, dev, stream, fp64_peak=None):
    """The grouped workload: 512 independent products with M, N, K each
    log-uniform on [32, 1024], entries uniform[-1,1), in one grouped call
    (persistent kernels replayed from a CUDA graph). TFLOP/s = sum 2mnk over
    the group / device time of a call, per mode, with the default tiles and
    with autotuned tiles; the emulated modes also as slice-product TFLOP/s
    (each problem's pairs) against the bf16 peak (measured burst; the whole
    call's time, split stages included), the plain mode against the FP64 peak;
    sampled rows of a few problems are checked against the oracle."""
    import numpy as np
    dims = inputs.problem_set(512, 32, 1024, 4)
    probs, flop = [], 0.0
    for i, (m, n, k) in enumerate(dims):
        m, n, k = int(m), int(n), int(k)
        A = torch.empty((m, k), dtype=torch.float64, device=dev)
        B = torch.empty((k, n), dtype=torch.float64, device=dev)
        C = torch.empty((m, n), dtype=torch.float64, device=dev)
        mm.fill_uniform(A, 4000 + i, inputs.STREAM_A)
        mm.fill_uniform(B, 4000 + i, inputs.STREAM_B)
        probs.append((A, B, C))
        flop += 2.0 * m * n * k
    arr = mm.Handle.problem_array(probs)
    torch.cuda.synchronize(dev)

    def timed(prec, reps=10):
        for _ in range(3):
            h.grouped(arr, precision=prec, stream=stream)
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            h.grouped(arr, precision=prec, stream=stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps

    out = {"problems": 512, "dims": "log-uniform [32, 1024]", "flop_per_call": flop}
    # slice products per call: each problem's automatic count (FP64-accuracy), 6 pairs (FP32-accuracy)
    slice_flop = {mm.FP64_EMU: 0.0, mm.FP32_EMU: 6.0 * flop}
    counts = {}
    for (A, B, _), (m, n, k) in zip(probs, dims):
        sc = h.debug_slice_count(A, B)[0] if int(k) > 4 else 0
        counts[sc] = counts.get(sc, 0) + 1
        if 3 <= sc <= 7:
            slice_flop[mm.FP64_EMU] += 2.0 * int(m) * int(n) * int(k) * sc * (sc + 1) // 2
    out["fp64_emu_slice_counts"] = {str(c): v for c, v in sorted(counts.items())}
    peaks = measured_peaks()
    bf16 = peaks.get("bf16_tflops", 1900.0)
    names = {mm.FP64: "fp64", mm.FP64_EMU: "fp64_emu", mm.FP32_EMU: "fp32_emu"}
    for prec, name in names.items():
        ms = timed(prec)
        out[name + "_tflops"] = flop / (ms * 1e-3) / 1e12
        out[name + "_ms"] = ms
        if prec in slice_flop:
            rate = slice_flop[prec] / (ms * 1e-3) / 1e12
            out[name + "_slice_tflops"] = rate
            out[name + "_frac_of_bf16"] = rate / bf16
        elif fp64_peak:
            out[name + "_frac_of_fp64_peak"] = out[name + "_tflops"] / fp64_peak
    h.set_option(mm.OPT_AUTOTUNE, 1)
    for prec, name in names.items():
        ms = timed(prec)
        out[name + "_tuned_tflops"] = flop / (ms * 1e-3) / 1e12
        d = np.mean([np.cbrt(a * b * c) for a, b, c in dims])
        out[name + "_tuned_cfg"] = h.tune_lookup(prec, 512, int(round(d)), grouped=True)
    h.set_option(mm.OPT_AUTOTUNE, 0)
    if not args.no_cpu_baseline:
        import oracle
        from oracle import emulation as em
        worst = 0.0
        for prec, name in names.items():
            h.grouped(arr, precision=prec, stream=stream)
            torch.cuda.synchronize(dev)
            for i in range(0, 512, 128):
                A, B, C = probs[i]
                Ah, Bh = A.cpu().numpy(), B.cpu().numpy()
                rows = [0, Ah.shape[0] - 1]
                D = oracle.absprod_rows(Ah, Bh, rows)
                ref = oracle.gemm_rows(Ah, Bh, rows)
                worst = max(worst, float(np.max(np.abs(C[rows].cpu().numpy() - ref) /
                                                (em.gamma(Ah.shape[1], name) * D))))
        out["sampled_max_err_over_bound"] = worst
    return out


def serve_leg(h, args, mm, inputs):
    """The serving workload: M, N, K each log-uniform on [64, 4096], accuracy
    class FP64/FP32 50:50, entries uniform[-1,1), admission under 40 GB.
    Capacity = closed-loop completion rate; then args.serve_requests requests
    arrive as a Poisson process at 80 % of it. Latency = scheduled arrival ->
    completion. A few sampled outputs are checked against the CPU oracle
    (their first two rows) when the CPU-baseline leg is on."""
    cap_res, _ = h.serve_bench(10000, 64, 4096, 0.5, 0.0, seed=5, slots=64)
    capacity = cap_res["req_per_s"]
    rate = 0.8 * capacity
    res, smp = h.serve_bench(args.serve_requests, 64, 4096, 0.5, rate, seed=6, slots=64,
                             sample_every=max(1, args.serve_requests // 16), max_samples=16, sample_cap=1 << 26)
    out = {"requests": args.serve_requests, "load": 0.8, "capacity_req_per_s": capacity,
           "offered_req_per_s": rate, "achieved_req_per_s": res["req_per_s"],
           "p50_ms": res["p50_ms"], "p90_ms": res["p90_ms"], "p99_ms": res["p99_ms"], "max_ms": res["max_ms"],
           "fp64_class_p99_ms": res["fp64_p99_ms"], "fp32_class_p99_ms": res["fp32_p99_ms"],
           "tflops": res["tflops"], "completed": res["completed"], "failed": res["failed"],
           "budget_gb": 40, "dims": "log-uniform [64, 4096]", "classes": "fp64/fp32 50:50"}
    if not args.no_cpu_baseline and smp:
        import numpy as np
        import oracle
        from oracle import emulation as em
        worst = 0.0
        for sm in smp[:6]:
            sd = 6 * 1000003 + sm["slot"]
            A2 = inputs.slot_block(sd, 1, 4096, 2, sm["k"])
            B = inputs.slot_block(sd, 2, 4096, sm["k"], sm["n"])
            mode = "fp64_emu" if sm["precision"] == 1 else "fp32_emu"
            D = oracle.absprod(A2, B)
            worst = max(worst, float(np.max(np.abs(sm["C"][:2] - oracle.gemm(A2, B)) / (em.gamma(sm["k"], mode) * D))))
        out["sampled_max_err_over_bound"] = worst
        out["err_sample"] = f"first 2 rows of {min(len(smp), 6)} sampled requests vs the FP64 triple-loop oracle"
    return out


def profile_case(args):
    """One workload alone, for profiler captures (prints a short status line,
    not a benchmark line): a single product of size --n in one mode on the
    benchmark's inputs, or the 512-problem grouped call in one mode; --warmup
    untimed calls, then --steps calls."""
    import torch
    import paper_2408_15384_gb300 as mm
    from paper_2408_15384_gb300 import inputs
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    h = mm.Handle(0, budget_bytes=40 << 30)
    stream = torch.cuda.current_stream(dev)
    kind, mode = args.profile_case.split(":")
    prec = {"fp64": mm.FP64, "fp64_emu": mm.FP64_EMU, "fp32_emu": mm.FP32_EMU}[mode]
    if kind == "single":
        N = args.n
        A = torch.empty((N, N), dtype=torch.float64, device=dev)
        B = torch.empty_like(A)
        C = torch.empty_like(A)
        mm.fill_uniform(A, 3, inputs.STREAM_A, 1, inputs.STREAM_EXP_A)
        mm.fill_uniform(B, 3, inputs.STREAM_B, 2, inputs.STREAM_EXP_B)
        run = lambda: h.gemm(A, B, C, precision=prec, stream=stream)   # noqa: E731
    else:
        probs = []
        for i, (m, n, k) in enumerate(inputs.problem_set(512, 32, 1024, 4)):
            A = torch.empty((int(m), int(k)), dtype=torch.float64, device=dev)
            B = torch.empty((int(k), int(n)), dtype=torch.float64, device=dev)
            mm.fill_uniform(A, 4000 + i, inputs.STREAM_A)
            mm.fill_uniform(B, 4000 + i, inputs.STREAM_B)
            probs.append((A, B, torch.empty((int(m), int(n)), dtype=torch.float64, device=dev)))
        arr = mm.Handle.problem_array(probs)
        run = lambda: h.grouped(arr, precision=prec, stream=stream)   # noqa: E731
    for _ in range(args.warmup):
        run()
    torch.cuda.synchronize(dev)
    for _ in range(args.steps):
        run()
    torch.cuda.synchronize(dev)
    status = h.sync()
    h.close()
    print(json.dumps({"profile_case": args.profile_case, "n": args.n, "status": status}), flush=True)
    if status != 0:
        sys.exit(1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true", help="headline line only")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-grouped", action="store_true", help="skip the grouped leg")
    ap.add_argument("--no-paper-sweep", action="store_true", help="skip the paper-size sweep")
    ap.add_argument("--serve-requests", type=int, default=100000)
    ap.add_argument("--profile-case", default=None,
                    help="single:MODE or grouped:MODE (MODE fp64, fp64_emu, fp32_emu): run only that workload")
    args = ap.parse_args()
    if args.profile_case:
        from paper_2408_15384_gb300 import build
        build.build()
        profile_case(args)
    elif args.impl == "reference":
        reference_arm(args)
    else:
        from paper_2408_15384_gb300 import build
        build.build()
        ours(args)


if __name__ == "__main__":
    main()
