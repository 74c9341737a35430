#!/usr/bin/env python3
"""Benchmark: bilinear biquaternion GEMM C = A B on one GB300 per rank.

Default workload (the precision configuration): m = n = k = 8192, both
operands Fock-like (N(0,1) exp(-|i-j|/200) per component) with per-row scales
10^U(-6,0), full biquaternions, op N/N, split-precision mode at tolerance
1e-12.  One step = one hmat_bq_gemm call (all stages of the path).  Metric:
TFLOP/s counted as 64 real GEMMs (64 * 2 n^3 / step time), the error checked
on sampled output rows against the CPU oracle, and the plain FP64 mode timed on
the same inputs for comparison.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on a
bounded row sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "biquaternion GEMM TFLOP/s (64-GEMM-equiv.) vs plain FP64 at n=8192, err≤1e-12"


FLAG_PAIRS = {"BQxBQ": (0xFF, 0xFF), "TRSxTRA": (0x0F, 0xF0), "TRSxTRS": (0x0F, 0x0F), "CxBQ": (0x11, 0xFF),
              "RxBQ": (0x01, 0xFF), "TRSxBQ": (0x0F, 0xFF), "BQxTRA": (0xFF, 0xF0), "CxC": (0x11, 0x11)}
FLAG_WORDS = {"BQxBQ": "full biquaternions x full biquaternions",
              "TRSxTRA": "real quaternions (TRS) x i*real quaternions (TRA)",
              "TRSxTRS": "real quaternions x real quaternions", "CxBQ": "complex x full biquaternions",
              "RxBQ": "real x full biquaternions", "TRSxBQ": "real quaternions x full biquaternions",
              "BQxTRA": "full biquaternions x i*real quaternions", "CxC": "complex x complex"}


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=8192, help="output columns (and m, k unless given)")
    ap.add_argument("--m", type=int, default=None, help="output rows (default: n)")
    ap.add_argument("--k", type=int, default=None, help="inner dimension (default: n)")
    ap.add_argument("--mode", choices=["split", "fp64", "mixed"], default="split",
                    help="mixed (grouped workload only): every fourth problem in FP64 mode, the rest in split "
                         "mode, in one hmat_bq_gemm_grouped_modes call")
    ap.add_argument("--tol", type=float, default=1e-12)
    ap.add_argument("--sample-rows", type=int, default=8)
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--e2e-budget-gb", type=float, default=100.0,
                    help="device budget of the end-to-end (host-resident operands) call")
    ap.add_argument("--seed", type=int, default=103)
    ap.add_argument("--workload", choices=["single", "grouped", "ops", "streamed", "fp64-peak"], default="single",
                    help="single: the n-sized product; grouped: 512 products with m,n,k log-uniform in [32,1024]; "
                         "ops: the element-wise and mapping operations at n x n; streamed: the product with "
                         "A, B, C in pinned host memory through a device budget (--budget-gb); fp64-peak: the "
                         "DFMA and DMMA probes that give the plain FP64 mode's roofline")
    ap.add_argument("--budget-gb", type=float, default=64.0, help="streamed: device budget in GB")
    ap.add_argument("--graph", action="store_true", help="grouped: replay a CUDA graph")
    ap.add_argument("--groups", type=int, default=512, help="grouped: the first G of the 512 problems")
    ap.add_argument("--complex-form", choices=["auto", "gauss", "four_m"], default="auto",
                    help="split mode, full biquaternions: complex products as Gauss's three real products, as two "
                         "over twice the inner dimension, or the library's default (four_m for k <= 512)")
    ap.add_argument("--tile-table", default=None,
                    help="tuned tables (tile width, FP64 split-k) JSON written by the autotuner")
    ap.add_argument("--results", default=None,
                    help="JSON-lines file: append each result with its configuration key; a configuration already "
                         "in the file is not run again (its stored line is printed)")
    ap.add_argument("--flags", choices=sorted(FLAG_PAIRS), default="BQxBQ",
                    help="subalgebra flags of A x B (single workload)")
    ap.add_argument("--opA", choices=["N", "T", "C", "H", "QC"], default="N", help="op(A) (single workload)")
    ap.add_argument("--no-row-scale", action="store_true",
                    help="banded Fock-like inputs without the per-row scales 10^U(-6,0)")
    ap.add_argument("--algo", choices=["bilinear", "standard", "isomorph"], default="bilinear",
                    help="product algorithm: the bilinear scheme, component-wise (HMAT-standard) "
                         "or the complex isomorph (CMAT)")
    args = ap.parse_args(argv)
    if args.mode == "mixed" and args.workload != "grouped":
        ap.error("--mode mixed applies to the grouped workload only")
    return args


def dims(args):
    """(m, n, k) of the single workload."""
    n = args.n
    return (getattr(args, "m", None) or n), n, (getattr(args, "k", None) or n)


def stored_shape(op, rows, cols):
    """Stored (rows, cols) of an operand whose op(X) is rows x cols."""
    return (cols, rows) if op in ("T", "H") else (rows, cols)


def workload_config(args):
    flags = getattr(args, "flags", "BQxBQ")
    opA = getattr(args, "opA", "N")
    scaled = not getattr(args, "no_row_scale", False)
    scale_txt = " with per-row scales 10^U(-6,0)" if scaled else ""
    m, n, k = dims(args)
    size = f"m=n=k={n}" if m == n == k else f"m={m} n={n} k={k}"
    return {"workload": f"bq_gemm {size} Fock-like N(0,1)*exp(-|i-j|/200){scale_txt}, "
                        f"{FLAG_WORDS[flags]}, op {opA},N, C=op(A)B",
            "m": m, "n": n, "k": k, "mode": args.mode, "tol": args.tol,
            "flags": flags, "opA": opA, "row_scale": scaled, "seed": args.seed,
            "algo": getattr(args, "algo", "bilinear"), "complex_form": getattr(args, "complex_form", "auto"),
            "l2": "inputs larger than L2 (8 x n^2 x 8 B per operand), no flush"}


# ----------------------------------------------------------------------------- distributed helpers
def dist_init(args):
    rank, world = int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples (200 ms) during the timed region."""

    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active," \
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown," \
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def recorded_traffic(kernel_file, workload_key, record="split_residue_gemm_traffic.json"):
    """DRAM bytes per launch from a committed ncu capture, if the kernel source is unchanged."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", record)
    src = os.path.join(ROOT, "paper_2609_02081_gb300", "csrc", kernel_file)
    if not (os.path.exists(prof) and os.path.exists(src)):
        return None
    with open(prof) as f:
        rec = json.load(f)
    with open(src, "rb") as f:
        digest = hashlib.sha256(f.read()).hexdigest()
    if rec.get("kernel_source_sha256") != digest or rec.get("workload") != workload_key:
        return None
    return rec.get("dram_bytes_per_launch")


def run_key(args):
    """The configuration a result line belongs to (for --results resume)."""
    keys = ["impl", "workload", "n", "mode", "tol", "flags", "opA", "algo", "seed", "gpus", "no_row_scale",
            "budget_gb", "graph", "tile_table", "complex_form"]
    return {k: getattr(args, k, None) for k in keys}


def emit(args, line):
    """Print the result line; with --results also append it (with its key) to that JSON-lines file."""
    print(json.dumps(line), flush=True)
    if getattr(args, "results", None):
        with open(args.results, "a") as f:
            f.write(json.dumps({"key": run_key(args), "line": line}) + "\n")


def completed(args):
    """The stored line of this configuration in --results, if any."""
    path = getattr(args, "results", None)
    if not path or not os.path.exists(path):
        return None
    key = run_key(args)
    with open(path) as f:
        for text in f:
            try:
                rec = json.loads(text)
            except ValueError:
                continue
            if rec.get("key") == key:
                return rec.get("line")
    return None


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def split_stage_work(hm, shapes, tol, opA="N", opB="N", fa=0xFF, fb=0xFF, algo="bilinear", complex_form="auto"):
    """Algorithmic work of one split-mode step per stage, summed over (m, n, k) shapes:
    bytes for the exponent, encode and CRT stages (what each stage must read and write:
    the present FP64 components, the encoded factor tiles of the plan's nlf / nrf factors
    per modulus, the int8 residue of every product and modulus, C) and BF16 flops for the
    residue GEMM (moduli x product terms x 2 m n k); "split_residue_gemm_bytes" is the least
    DRAM traffic of the residue GEMM (every encoded factor tile read once, every int8
    residue written once), its bound on products too small to reuse their tiles.  Full
    biquaternion products in the four-multiplication form (complex_form "four_m", or
    "auto" at k <= 512) count its 16 factors per side, 16 products and 32 terms."""
    def form(a):
        T, U, V, _, _ = hm.plan_info(opA, opB, fa, fb, algo=a)
        P = T // 2 if a == "four_m" else T
        return T, P, len({tuple(r) for r in U.tolist()}), len({tuple(r) for r in V.tolist()})
    gauss = form(algo)
    four = form("four_m") if algo == "bilinear" and fa == 0xFF and fb == 0xFF else gauss
    ca, cb = bin(fa).count("1"), bin(fb).count("1")
    w = {"split_exponents": 0.0, "split_encode": 0.0, "split_crt": 0.0, "split_residue_gemm": 0.0,
         "split_residue_gemm_bytes": 0.0}
    for m, n, k in shapes:
        T, P, nlf, nrf = four if complex_form == "four_m" or (complex_form == "auto" and k <= 512) else gauss
        L = len(hm.split_info(k, tol)[0])
        kp = -(-k // 64) * 64
        raw = 8.0 * (ca * m * k + cb * k * n)
        w["split_exponents"] += raw
        w["split_encode"] += raw + 2.0 * L * (nlf * m + nrf * n) * kp
        w["split_crt"] += L * P * m * n + 64.0 * m * n
        w["split_residue_gemm"] += 2.0 * L * T * m * n * k
        w["split_residue_gemm_bytes"] += 2.0 * L * (nlf * m + nrf * n) * kp + L * P * m * n
    return w


def stage_rates(stages, work, steps=1):
    """GB/s (HBM stages) and TFLOP/s (residue GEMM) of each timed stage from its summed event time."""
    for name, st in stages.items():
        ms = st.get("ms_total", st.get("ms"))
        if name not in work or not ms:
            continue
        if name == "split_residue_gemm":
            st["TFLOP_per_s"] = work[name] * steps / (ms * 1e-3) / 1e12
            if "split_residue_gemm_bytes" in work:
                st["GB_per_s"] = work["split_residue_gemm_bytes"] * steps / (ms * 1e-3) / 1e9
                st["algorithmic_bytes_per_step"] = work["split_residue_gemm_bytes"]
        else:
            st["GB_per_s"] = work[name] * steps / (ms * 1e-3) / 1e9
            st["algorithmic_bytes_per_step"] = work[name]
    return stages


def fp64_peaks(hm, iterations=1 << 16):
    """Measured FP64 throughput of this GPU (best of 3 launches per probe), TFLOP/s:
    {"dfma": ..., "dmma_m8n8k4": ..., "dmma_m16n8k4": ...}."""
    out = {}
    for kind in hm.FP64_PEAK_KINDS:
        hm.measure_fp64_peak(kind, 1 << 10)                      # warm-up
        out[kind] = max(hm.measure_fp64_peak(kind, iterations)[0] for _ in range(3))
    return out


def fp64_roofline(achieved, peaks, kernel="fp64_bilinear_kernel", **extra):
    """Roofline of an FP64-mode launch against the measured DFMA peak (the kernel's pipe),
    with its fraction of the best FP64 tensor-core (DMMA) probe beside it."""
    dmma = max(peaks["dmma_m8n8k4"], peaks["dmma_m16n8k4"])
    r = {"bound": "alu", "achieved": achieved, "peak": peaks["dfma"], "unit": "TFLOP/s",
         "frac": achieved / peaks["dfma"], "traffic": None, "kernel": kernel,
         "peak_source": "hmat_measure_fp64_peak DFMA probe, measured in this run (of measured)",
         "frac_of_dmma": achieved / dmma, "peaks_measured": peaks}
    r.update(extra)
    return r


def freivalds_host(A_cpu, B_cpu, C_cpu, opA, seed):
    """Whole-matrix check of C = op(A) B: ||C x - op(A) (B x)|| / (||C||_F ||x||) for a
    random biquaternion vector x, both sides by the CPU oracle (Freivalds 1977)."""
    import numpy as np
    import bq_inputs as bi
    import oracle
    x = bi.uniform(seed, C_cpu.shape[2], 1).numpy()
    y1 = oracle.bq_gemm(C_cpu, x)
    y2 = oracle.bq_gemm(A_cpu, oracle.bq_gemm(B_cpu, x), opA, "N")
    return float(np.linalg.norm(y1 - y2) / (np.linalg.norm(C_cpu) * np.linalg.norm(x)))


def fp64_peak_arm(args, rank, world, local):
    """The FP64 probes alone: DFMA and the two DMMA shapes, each timed with CUDA events."""
    import torch
    import paper_2609_02081_gb300 as hm
    dev = torch.device("cuda", local if torch.cuda.device_count() > local else 0)
    torch.cuda.set_device(dev)
    clocks = ClockSampler(dev.index)
    clocks.start()
    runs = {}
    for kind in hm.FP64_PEAK_KINDS:
        for _ in range(args.warmup):
            hm.measure_fp64_peak(kind, 1 << 12)
        vals = [hm.measure_fp64_peak(kind, 1 << 17) for _ in range(args.steps)]
        runs[kind] = {"tflops_best": max(v[0] for v in vals), "tflops_median": statistics.median(v[0] for v in vals),
                      "ms_median": statistics.median(v[1] for v in vals)}
    clk = clocks.stop()
    if rank == 0:
        best = runs["dfma"]["tflops_best"]
        line = {"metric": "FP64 throughput TFLOP/s (DFMA probe; DMMA probes beside it)", "value": best,
                "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": runs["dfma"]["ms_median"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": {"workload": "FP64 probe kernels: 8 blocks per SM, 8 independent chains per thread "
                                       "(DFMA) or per warp (mma.sync m8n8k4 / m16n8k4), 2^17 loop trips"},
                "probes": runs, "clocks": clk, "gpu_launches": args.steps * len(runs)}
        emit(args, line)


# ----------------------------------------------------------------------------- oracle sample
def oracle_rows(A_cpu, B_cpu, rows, opA="N"):
    """Selected output rows of op(A) B from the CPU oracle; returns (rows x, seconds, threads)."""
    import numpy as np
    import oracle
    if opA in ("T", "H"):                     # rows of op(A) are columns of the stored A
        Asub = np.ascontiguousarray(A_cpu[:, :, rows])
    else:
        Asub = np.ascontiguousarray(A_cpu[:, rows, :])
    t0 = time.perf_counter()
    out = oracle.bq_gemm(Asub, B_cpu, opA, "N")
    return out, time.perf_counter() - t0, oracle.max_threads()


def reference_arm(args, rank, world):
    """CPU oracle on a bounded row sample of the same workload (host cores)."""
    if rank != 0:
        return
    import numpy as np
    import torch
    import bq_inputs as bi
    import oracle
    m, n, k = dims(args)
    fa, fb = FLAG_PAIRS[args.flags]
    scaled = not args.no_row_scale
    A = bi.fock_like(args.seed, *stored_shape(args.opA, m, k), flags=fa, row_scale=scaled).numpy()
    B = bi.fock_like(args.seed + 1, k, n, flags=fb, row_scale=scaled).numpy()
    threads = oracle.max_threads()
    rows_per_step = max(1, min(threads, 16))
    times = []
    rng = np.random.default_rng(args.seed)
    for step in range(args.warmup + args.steps):
        rows = np.sort(rng.choice(m, size=rows_per_step, replace=False))
        _, dt, _ = oracle_rows(A, B, rows, args.opA)
        if step >= args.warmup:
            times.append(dt)
    t = statistics.mean(times)
    flops64 = 64 * 2.0 * rows_per_step * n * k
    value = flops64 / t / 1e12
    sample = f"{rows_per_step} of {m} output rows per step (all 8 components), oracle on {threads} threads"
    line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "impl": "reference", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args),
            "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    emit(args, line)


# ----------------------------------------------------------------------------- our arm
def ours(args, rank, world, local):
    import numpy as np
    import torch
    import bq_inputs as bi
    import paper_2609_02081_gb300 as hm

    dev = torch.device("cuda", local if torch.cuda.device_count() > local else 0)
    torch.cuda.set_device(dev)
    m, n, k = dims(args)
    fa, fb = FLAG_PAIRS[args.flags]
    scaled = not args.no_row_scale
    A = bi.fock_like(args.seed, *stored_shape(args.opA, m, k), flags=fa, row_scale=scaled, device=dev)
    B = bi.fock_like(args.seed + 1, k, n, flags=fb, row_scale=scaled, device=dev)
    C = torch.empty((8, m, n), dtype=torch.float64, device=dev)
    h = hm.Handle()
    h.set_algorithm(args.algo)
    h.set_complex_form(args.complex_form)
    if args.tile_table:
        from paper_2609_02081_gb300 import autotune
        h.set_tile_table(autotune.load(args.tile_table))
        fp = autotune.load_fp64(args.tile_table)
        if fp is not None:
            h.set_fp64_splitk_table(fp)
        for (ta, tb), t in autotune.load_flag_tables(args.tile_table).items():
            h.set_tile_table_flags(ta, tb, t)
    d = hm.make_desc(A, B, C, args.opA, "N", fa, fb)
    ws_bytes = hm.hmat_workspace_size(h, [d], args.mode, args.tol)
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(mode=args.mode):
        hm.hmat_bq_gemm(h, A, B, C, args.opA, "N", fa, fb, mode=mode, tol=args.tol, workspace=ws, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    h.set_profiling(True)
    h.reset_profile()
    clocks = ClockSampler(dev.index)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    ms_local = ev0.elapsed_time(ev1) / args.steps
    ms = max_over_ranks(ms_local, world)
    kernels = {k: h.profile(k) for k in hm.KERNEL_IDS}
    h.set_profiling(False)
    launches = sum(v[0] for v in kernels.values())
    flops64 = 64 * 2.0 * m * n * k
    value = world * flops64 / (ms * 1e-3) / 1e12

    # accuracy on sampled rows (rank 0)
    info = {}
    naive = bin(fa).count("1") * bin(fb).count("1")      # component-wise real products
    # the real products one step executes: plan products x their size relative to n^3
    if args.algo == "isomorph":
        P = hm.plan_info("N", "N", hm.HMAT_COMPLEX, hm.HMAT_COMPLEX)[0]
        size, kin = 8, 2 * k          # one complex product of 2m x 2n x 2k
    else:
        P = hm.plan_info(args.opA, "N", fa, fb, algo=args.algo)[0]
        size, kin = 1, k
        if (args.mode == "split" and args.algo == "bilinear" and fa == fb == 0xFF and
                (args.complex_form == "four_m" or (args.complex_form == "auto" and k <= 512))):
            P = hm.plan_info(args.opA, "N", fa, fb, algo="four_m")[0]   # product terms (two per product)
    mods, bits = hm.split_info(kin, args.tol)
    if rank == 0:
        rng = np.random.default_rng(args.seed + 7)
        rows = np.sort(rng.choice(m, size=args.sample_rows, replace=False))
        A_cpu = A.cpu().numpy()
        B_cpu = B.cpu().numpy()
        want, t_or, threads = oracle_rows(A_cpu, B_cpu, rows, args.opA)
        got = C[:, torch.as_tensor(rows, device=dev), :].cpu().numpy()
        err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
        info["rel_fro_err_sampled"] = err
        cpu_value = 64 * 2.0 * len(rows) * n * k / t_or / 1e12
        info["cpu_baseline"] = {"value": cpu_value, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
                                "sample": f"{len(rows)} of {m} output rows (all 8 components) of the same "
                                          f"product, C oracle on {threads} OpenMP threads, {t_or:.1f} s"}
        # plain FP64 mode on the same inputs (1 timed call)
        if not args.no_fp64_compare and args.mode == "split":
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step("fp64")
            e1.record(stream)
            torch.cuda.synchronize()
            fms = e0.elapsed_time(e1)
            got64 = C[:, torch.as_tensor(rows, device=dev), :].cpu().numpy()
            ex64 = P * size * 2.0 * m * n * k / (fms * 1e-3) / 1e12
            info["fp64_plain"] = {"ms": fms, "tflops_64equiv": flops64 / (fms * 1e-3) / 1e12,
                                  "tflops_executed": ex64,
                                  "rel_fro_err_sampled": float(np.linalg.norm(got64 - want) / np.linalg.norm(want)),
                                  "speedup_split_vs_fp64": fms / ms,
                                  "roofline": fp64_roofline(ex64, fp64_peaks(hm))}
            step()                          # C back to the timed mode's result for the checks below
            torch.cuda.synchronize()
        # whole-matrix accuracy of the timed mode's C (Freivalds, oracle matrix-vector products)
        t0 = time.perf_counter()
        info["freivalds_ratio"] = freivalds_host(A_cpu, B_cpu, C.cpu().numpy(), args.opA, args.seed + 11)
        info["freivalds_s"] = time.perf_counter() - t0

        # end to end with the operands in pinned host memory.  Serial form: copy A, B in, the product,
        # copy C out, one after another on the stream (bq_gemm_host).
        Ah = A.cpu().pin_memory()
        Bh = B.cpu().pin_memory()
        Ch = torch.empty((8, m, n), dtype=torch.float64).pin_memory()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        A.copy_(Ah, non_blocking=True)
        B.copy_(Bh, non_blocking=True)
        ev[1].record(stream)
        step()
        ev[2].record(stream)
        Ch.copy_(C, non_blocking=True)
        ev[3].record(stream)
        torch.cuda.synchronize()
        serial = {"h2d": ev[0].elapsed_time(ev[1]), "product": ev[1].elapsed_time(ev[2]),
                  "d2h": ev[2].elapsed_time(ev[3])}
        serial["total"] = sum(serial.values())
        # The public call for host-resident operands: hmat_bq_gemm_streamed copies blocks of A and B in and
        # blocks of C out behind the products, within a device budget; the bytes it copies per call come
        # from the library's plan (hmat_streamed_traffic).
        del ws
        torch.cuda.empty_cache()
        budget = int(args.e2e_budget_gb * (1 << 30))
        mb, nb, kb, _ = hm.streamed_plan(m, n, k, args.opA, "N", fa, fb, args.mode, args.tol, budget, handle=h)
        ws_e2e = torch.empty(budget, dtype=torch.uint8, device=dev)

        def e2e_step():
            hm.hmat_bq_gemm_streamed(h, Ah, Bh, Ch, args.opA, "N", fa, fb, mode=args.mode, tol=args.tol,
                                     workspace=ws_e2e, stream=stream)

        e2e_step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.e2e_steps):
            e2e_step()
        e1.record(stream)
        torch.cuda.synchronize()
        ems = e0.elapsed_time(e1) / args.e2e_steps
        got_e2e = Ch.numpy()[:, rows, :]
        h2d, d2h = hm.streamed_traffic(m, n, k, args.opA, "N", fa, fb, args.mode, args.tol, budget, handle=h)
        info["e2e"] = {"value": flops64 / (ems * 1e-3) / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "ms_per_step": ems,
                       "api": "hmat_bq_gemm_streamed (pinned host A, B, C)", "blocks": [mb, nb, kb],
                       "rel_fro_err_sampled": float(np.linalg.norm(got_e2e - want) / np.linalg.norm(want)),
                       "serial_ms": serial,
                       "serial_value": flops64 / (serial["total"] * 1e-3) / 1e12}
        del ws_e2e

    if rank == 0:
        peaks, src = measured_peaks()
        gl, gms = kernels["split_residue_gemm"] if args.mode == "split" else kernels["fp64_bilinear"]
        wl_key = ((f"n={n}" if m == n == k else f"m={m} n={n} k={k}") + f" split tol={args.tol}" +
                  ("" if args.algo == "bilinear" else f" algo={args.algo}"))
        if args.mode == "split":
            # BF16 tensor flops of the GEMM launches of one step, per launch
            alg = len(mods) * P * size * 2.0 * m * n * k * args.steps / max(gl, 1)
            avg = gms / max(gl, 1)
            ach = alg / (avg * 1e-3) / 1e12
            peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
            roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                    "traffic": recorded_traffic("split_gemm.cu", wl_key),
                    "kernel": "split_residue_gemm_kernel", "peak_source": f"bf16 sustained ({src})",
                    "algorithmic_flops_per_launch": alg, "avg_launch_ms": avg}
        else:
            alg = P * size * 2.0 * m * n * k * args.steps / max(gl, 1)   # a plan over 24 products takes passes
            avg = gms / max(gl, 1)
            ach = alg / (avg * 1e-3) / 1e12
            roof = fp64_roofline(ach, fp64_peaks(hm), algorithmic_flops_per_launch=alg, avg_launch_ms=avg)
        stages = {k: {"launches": v[0], "ms_total": v[1]} for k, v in kernels.items() if v[0] > 0}
        if args.mode == "split" and args.algo == "bilinear":
            stages = stage_rates(stages, split_stage_work(hm, [(m, n, k)], args.tol, args.opA, "N", fa, fb,
                                                          complex_form=args.complex_form), args.steps)
        line = {"metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16" if args.mode == "split" else "f64", "data": "synthetic",
                "config": dict(workload_config(args), parallelism=f"replicas x{world}",
                               moduli=len(mods), bits=bits, products=P),
                "roofline": roof, "cpu_baseline": info.get("cpu_baseline"), "e2e": info.get("e2e"),
                "gpu_launches": launches, "clocks": clk,
                "rel_fro_err_sampled": info.get("rel_fro_err_sampled"),
                "freivalds_ratio": info.get("freivalds_ratio"),
                "freivalds_note": "||C x - op(A)(B x)|| / (||C||_F ||x||) over the whole output, random "
                                  "biquaternion x, both sides in the CPU oracle; bound tol + 1e-14",
                "err_ok": (info.get("rel_fro_err_sampled") is not None and info["rel_fro_err_sampled"] <= 1e-12
                           and info.get("freivalds_ratio") is not None
                           and info["freivalds_ratio"] <= args.tol + 1e-14),
                "fp64_plain": info.get("fp64_plain"), "stages": stages,
                "executed_tflops": value * size * (len(mods) * P if args.mode == "split" else P) / 64.0,
                "naive_equiv_tflops": value * naive / 64.0,
                "naive_equiv_note": f"counted as {naive} component-wise real GEMMs of n^3"}
        emit(args, line)
    barrier(world)
    h.close()


def grouped(args, rank, world, local):
    """512 independent products of log-uniform shapes in one grouped call per step."""
    import numpy as np
    import torch
    import bq_inputs as bi
    import oracle
    import paper_2609_02081_gb300 as hm

    dev = torch.device("cuda", local if torch.cuda.device_count() > local else 0)
    torch.cuda.set_device(dev)
    shapes = bi.batch_shapes(104, 512)[:args.groups]
    mats, descs = [], []
    for i, (m, n, k) in enumerate(shapes):
        A = bi.uniform(10_000 + i, m, k, device=dev)
        B = bi.uniform(20_000 + i, k, n, device=dev)
        C = torch.empty((8, m, n), dtype=torch.float64, device=dev)
        mats.append((A, B, C))
        descs.append(hm.make_desc(A, B, C))
    h = hm.Handle()
    h.set_complex_form(args.complex_form)
    if args.tile_table:
        from paper_2609_02081_gb300 import autotune
        h.set_tile_table(autotune.load(args.tile_table))
        fp = autotune.load_fp64(args.tile_table)
        if fp is not None:
            h.set_fp64_splitk_table(fp)
        for (ta, tb), t in autotune.load_flag_tables(args.tile_table).items():
            h.set_tile_table_flags(ta, tb, t)
    modes = ["fp64" if i % 4 == 3 else "split" for i in range(len(descs))] if args.mode == "mixed" else None
    if modes:
        ws_bytes = hm.hmat_workspace_size_modes(h, descs, modes, args.tol)
    else:
        ws_bytes = hm.hmat_workspace_size(h, descs, args.mode, args.tol)
    ws = torch.empty(max(ws_bytes, 1), dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        if modes:
            hm.hmat_bq_gemm_grouped_modes(h, descs, modes, args.tol, workspace=ws, stream=stream,
                                          use_graph=args.graph)
        else:
            hm.hmat_bq_gemm_grouped(h, descs, args.mode, args.tol, workspace=ws, stream=stream,
                                    use_graph=args.graph)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev.index)
    barrier(world)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world)
    # per-stage kernel times (one extra eager step with event brackets)
    h.set_profiling(True)
    h.reset_profile()
    if modes:
        hm.hmat_bq_gemm_grouped_modes(h, descs, modes, args.tol, workspace=ws, stream=stream, use_graph=False)
    else:
        hm.hmat_bq_gemm_grouped(h, descs, args.mode, args.tol, workspace=ws, stream=stream, use_graph=False)
    torch.cuda.synchronize()
    stages = {k: {"launches": v[0], "ms": v[1]} for k, v in ((k, h.profile(k)) for k in hm.KERNEL_IDS) if v[0]}
    h.set_profiling(False)
    flops64 = sum(64 * 2.0 * m * n * k for m, n, k in shapes)
    value = world * flops64 / (ms * 1e-3) / 1e12
    launches_per_step = sum(v["launches"] for v in stages.values())
    split_shapes = [sh for i, sh in enumerate(shapes) if modes is None or modes[i] == "split"]
    if args.mode in ("split", "mixed"):
        gemm_flops = split_stage_work(hm, split_shapes, args.tol,
                                      complex_form=args.complex_form)["split_residue_gemm"]
        gst = stages.get("split_residue_gemm", {"launches": 1, "ms": float("nan")})
        ach = gemm_flops / (gst["ms"] / gst["launches"] * 1e-3) / 1e12
        peaks, src = measured_peaks()
        peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        roof = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "kernel": "split_residue_gemm_kernel",
                "peak_source": f"bf16 sustained ({src}); algorithmic flops exclude tile padding"}
    else:
        P = hm.plan_info("N", "N", hm.HMAT_BQ, hm.HMAT_BQ)[0]
        fst = stages.get("fp64_bilinear", {"launches": 1, "ms": float("nan")})
        ach = sum(P * 2.0 * m * n * k for m, n, k in shapes) / (fst["ms"] / fst["launches"] * 1e-3) / 1e12
        roof = fp64_roofline(ach, fp64_peaks(hm))
    if rank == 0:
        # accuracy: 16 sampled problems against the oracle
        rng = np.random.default_rng(5)
        errs = []
        small = [i for i, (m, n, k) in enumerate(shapes) if m * n * k <= (1 << 25)]
        t_or, f_or = 0.0, 0.0
        for i in rng.choice(small, size=min(16, len(small)), replace=False):
            A, B, C = mats[i]
            An, Bn = A.cpu().numpy(), B.cpu().numpy()
            t0 = time.perf_counter()
            want = oracle.bq_gemm(An, Bn)
            t_or += time.perf_counter() - t0
            m, n, k = shapes[i]
            f_or += 64 * 2.0 * m * n * k
            errs.append(float(np.linalg.norm(C.cpu().numpy() - want) / np.linalg.norm(want)))
        cpu_base = {"value": f_or / t_or / 1e12, "unit": "TFLOP/s", "cores": oracle.max_threads(), "kind": "oracle",
                    "sample": f"the 16 sampled problems of the batch (m n k <= 2^25), {t_or:.1f} s"}
        roof_hbm = None
        if args.mode in ("split", "mixed"):
            stages = stage_rates(stages, split_stage_work(hm, split_shapes, args.tol, complex_form=args.complex_form))
            g = stages.get("split_residue_gemm", {})
            if g.get("GB_per_s"):
                hbm = measured_peaks()[0].get("hbm_gbs")
                roof_hbm = {"bound": "hbm", "achieved": g["GB_per_s"], "peak": hbm, "unit": "GB/s",
                            "frac": g["GB_per_s"] / hbm if hbm else None, "kernel": "split_residue_gemm_kernel",
                            "note": "the residue GEMM against the copy bandwidth for its least DRAM traffic "
                                    "(encoded factor tiles read once, int8 residues written once): the bound "
                                    "of products whose tiles feed one to four output tiles"}
        line = {"metric": "grouped biquaternion GEMM TFLOP/s (64-GEMM-equiv.)", "value": value, "unit": "TFLOP/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"split": "bf16", "fp64": "f64", "mixed": "bf16+f64"}[args.mode], "data": "synthetic",
                "config": {"workload": f"{len(shapes)} products, m,n,k log-uniform in [32,1024] (seed 104), "
                                       f"iid U[-1,1], full biquaternions", "mode": args.mode, "graph": args.graph,
                           "tol": args.tol, "total_flops_64equiv": flops64,
                           "tile_table": args.tile_table, "complex_form": args.complex_form,
                           "workspace_bytes": ws_bytes},
                "max_rel_fro_err_16_sampled": max(errs), "clocks": clk, "stages_one_step": stages,
                "roofline": roof, "roofline_hbm": roof_hbm, "cpu_baseline": cpu_base,
                "gpu_launches": launches_per_step * args.steps}
        emit(args, line)
    barrier(world)
    h.close()


def ops_arm(args, rank, world, local):
    """The HBM-bound element-wise / mapping kernels on n x n full biquaternions:
    achieved GB/s (algorithmic bytes / CUDA-event time) against the measured copy bandwidth."""
    import torch
    import bq_inputs as bi
    import paper_2609_02081_gb300 as hm

    dev = torch.device("cuda", local if torch.cuda.device_count() > local else 0)
    torch.cuda.set_device(dev)
    n = args.n
    A = bi.fock_like(args.seed, n, n, device=dev)
    B = bi.fock_like(args.seed + 1, n, n, device=dev)
    Hj = bi.apply_flags(A.clone(), 0xCC)
    C = torch.empty_like(A)
    # a Hermitian matrix (A + A^dagger, formed by the library) and a pure-j Hermitian one
    Herm = torch.empty_like(A)
    hm_handle = hm.Handle()
    hm.hmat_bq_add(hm_handle, A, A, Herm, 1.0, 1.0, "N", "H")
    Pj = bi.apply_flags(Herm.clone(), 0x44)
    torch.cuda.synchronize()
    hm_handle.close()
    Z = torch.empty((2 * n, 2 * n), dtype=torch.complex128, device=dev)
    Zh = torch.empty((n, n), dtype=torch.complex128, device=dev)
    res = torch.empty(2, dtype=torch.float64, device=dev)
    h = hm.Handle()
    stream = torch.cuda.current_stream(dev)
    e = n * n
    # name -> (call, algorithmic bytes per launch)
    cases = {
        "add": (lambda: hm.hmat_bq_add(h, A, B, C, 1.0, 1.0, stream=stream), 3 * 64 * e),
        "add_complex_scalars": (lambda: hm.hmat_bq_add(h, A, B, C, 1 - 1j, 0.5, stream=stream), 3 * 64 * e),
        "add_opH": (lambda: hm.hmat_bq_add(h, A, B, C, 1.0, 1.0, "H", "N", stream=stream), 3 * 64 * e),
        "scale_real": (lambda: hm.hmat_bq_scale(h, A, C, 2.5, stream=stream), 2 * 64 * e),
        "scale_complex": (lambda: hm.hmat_bq_scale(h, A, C, 2 - 1j, stream=stream), 2 * 64 * e),
        "to_complex": (lambda: hm.hmat_bq_to_complex(h, A, Z, stream=stream), 2 * 64 * e),
        "to_complex_opT": (lambda: hm.hmat_bq_to_complex(h, A, Z, op="T", stream=stream), 2 * 64 * e),
        "from_complex": (lambda: hm.hmat_complex_to_bq(h, Z, C, stream=stream), 2 * 64 * e),
        "hermiticity": (lambda: hm.hmat_bq_hermiticity(h, A, out=res, stream=stream), 64 * e),
        "hermiticity_of_hermitian": (lambda: hm.hmat_bq_hermiticity(h, Herm, out=res, stream=stream), 64 * e),
        "hadamard": (lambda: hm.hmat_bq_hadamard_block(h, Hj, 1j, 0xCC, Z=Zh, stream=stream), (32 + 16) * e),
        "hadamard_pure_j": (lambda: hm.hmat_bq_hadamard_block(h, Pj, 1j, 0x44, Z=Zh, stream=stream),
                            (16 + 16) * e),
    }
    peaks, src = measured_peaks()
    peak = peaks["hbm_gbs"]
    out = {}
    clocks = ClockSampler(dev.index)
    clocks.start()
    for name, (call, nbytes) in cases.items():
        for _ in range(args.warmup):
            call()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            call()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        gbs = nbytes / (ms * 1e-3) / 1e9
        out[name] = {"ms": ms, "GB_per_s": gbs, "frac": gbs / peak, "bytes": nbytes}
    clk = clocks.stop()
    if rank == 0:
        top = out["add"]
        line = {"metric": "element-wise biquaternion ops, achieved HBM GB/s", "value": top["GB_per_s"],
                "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": top["ms"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": f"n={n} full biquaternions, Fock-like N(0,1)*exp(-|i-j|/200) (seed "
                                       f"{args.seed}); value = the paper's sum C = A + B",
                           "l2": "operands 8 x n^2 x 8 B, larger than L2, no flush"},
                "roofline": {"bound": "hbm", "achieved": top["GB_per_s"], "peak": peak, "unit": "GB/s",
                             "frac": top["GB_per_s"] / peak,
                             "traffic": recorded_traffic("elementwise.cu", f"ops n={n} add",
                                                         "elementwise_ops_traffic.json"),
                             "kernel": "axpby_rows_kernel<2>",
                             "peak_source": f"hbm copy ({src})"},
                "ops": out, "clocks": clk, "gpu_launches": args.steps * len(cases)}
        emit(args, line)
    h.close()


def streamed_arm(args, rank, world, local):
    """Split-mode product with every operand in pinned host memory, computed block by block within a device
    budget; the timed region covers all copies in and out."""
    import numpy as np
    import torch
    import bq_inputs as bi
    import paper_2609_02081_gb300 as hm

    dev = torch.device("cuda", local if torch.cuda.device_count() > local else 0)
    torch.cuda.set_device(dev)
    n = args.n
    A = bi.fock_like(args.seed, n, n, row_scale=True, device=dev).cpu().pin_memory()
    B = bi.fock_like(args.seed + 1, n, n, row_scale=True, device=dev).cpu().pin_memory()
    torch.cuda.empty_cache()
    C = torch.empty((8, n, n), dtype=torch.float64).pin_memory()
    budget = int(args.budget_gb * (1 << 30))
    mb, nb, kb, nbytes = hm.streamed_plan(n, n, n, mode=args.mode, tol=args.tol, budget=budget)
    h = hm.Handle()
    ws = torch.empty(budget, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step():
        hm.hmat_bq_gemm_streamed(h, A, B, C, mode=args.mode, tol=args.tol, workspace=ws, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    h.set_profiling(True)
    h.reset_profile()
    clocks = ClockSampler(dev.index)
    barrier(world)
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier(world)
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, world)
    kernels = {k: h.profile(k) for k in hm.KERNEL_IDS}
    h.set_profiling(False)
    flops64 = 64 * 2.0 * n ** 3
    value = world * flops64 / (ms * 1e-3) / 1e12
    if rank == 0:
        rng = np.random.default_rng(args.seed + 7)
        rows = np.sort(rng.choice(n, size=args.sample_rows, replace=False))
        want, t_or, threads = oracle_rows(A.numpy(), B.numpy(), rows)
        got = C.numpy()[:, rows, :]
        err = float(np.linalg.norm(got - want) / np.linalg.norm(want))
        h2d, d2h = hm.streamed_traffic(n, n, n, mode=args.mode, tol=args.tol, budget=budget, handle=h)
        mods, bits = hm.split_info(kb, args.tol)
        P = hm.plan_info("N", "N", hm.HMAT_BQ, hm.HMAT_BQ)[0]
        gl, gms = kernels["split_residue_gemm"]
        alg = len(mods) * P * 2.0 * mb * nb * kb     # per launch (full blocks)
        avg = gms / max(gl, 1)
        peaks, src = measured_peaks()
        peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
        line = {"metric": "biquaternion GEMM TFLOP/s (64-GEMM-equiv.), operands in host memory, streamed",
                "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "bf16" if args.mode == "split" else "f64", "data": "synthetic",
                "config": {"workload": f"bq_gemm m=n=k={n} Fock-like row-scaled, A, B, C in pinned host memory, "
                                       f"device budget {args.budget_gb:g} GB, blocks {mb} x {nb} x {kb}",
                           "mode": args.mode, "tol": args.tol, "blocks": [mb, nb, kb], "device_bytes": nbytes},
                "roofline": {"bound": "tensor", "achieved": alg / (avg * 1e-3) / 1e12, "peak": peak,
                             "unit": "TFLOP/s", "frac": alg / (avg * 1e-3) / 1e12 / peak, "traffic": None,
                             "kernel": "split_residue_gemm_kernel", "peak_source": f"bf16 sustained ({src})"},
                "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "rel_fro_err_sampled": err, "err_ok": err <= 1e-12,
                "cpu_baseline": {"value": 64 * 2.0 * len(rows) * n * n / t_or / 1e12, "unit": "TFLOP/s",
                                 "cores": threads, "kind": "oracle",
                                 "sample": f"{len(rows)} of {n} output rows, {t_or:.1f} s"},
                "stages": {k: {"launches": v[0], "ms_total": v[1]} for k, v in kernels.items() if v[0] > 0},
                "gpu_launches": sum(v[0] for v in kernels.values()), "clocks": clk}
        emit(args, line)
    h.close()


def main():
    args = parse()
    done = completed(args)
    if done is not None:
        if int(os.environ.get("RANK", 0)) == 0:
            print(json.dumps(done), flush=True)
        return
    rank, world, local = dist_init(args)
    try:
        if args.workload == "ops" and args.impl == "ours":
            ops_arm(args, rank, world, local)
        elif args.workload == "streamed" and args.impl == "ours":
            streamed_arm(args, rank, world, local)
        elif args.workload == "grouped" and args.impl == "ours":
            grouped(args, rank, world, local)
        elif args.workload == "fp64-peak" and args.impl == "ours":
            fp64_peak_arm(args, rank, world, local)
        elif args.impl == "reference":
            reference_arm(args, rank, world)
        else:
            ours(args, rank, world, local)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
