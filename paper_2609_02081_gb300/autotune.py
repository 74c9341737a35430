"""Autotuner for the split-mode output tile width (hmat_set_tile_table) and
the FP64 split-k slice count (hmat_set_fp64_splitk_table).

Tile width: for every (ceil(log2 m), ceil(log2 n)) bin that a set of problem
shapes touches, the tuner times one representative product of that bin on the
GPU with the built-in rule (the fewest tiles of at most 256 columns, each a
multiple of 32 wide) and with each fixed tile width (128 x 64, 128 x 128,
128 x 256), and keeps the fastest.  The result is a 16 x 16 table of codes (0 = built-in rule, 1/2/3 =
64/128/256 columns) that :meth:`Handle.set_tile_table` installs.

Split-k (--fp64): for every (ceil(log2 tiles), ceil(log2 k)) bin of the FP64
shapes, one representative product is timed in FP64 mode with its inner
dimension in 1, 2, 4 and 8 slices; the fastest code (1..4) goes into a second
16 x 16 table that :meth:`Handle.set_fp64_splitk_table` installs.

Grouped (--grouped): per-bin timing alone does not predict a grouped call,
whose residue-GEMM items of all products share the SMs; this mode times
every candidate table on one grouped call over all the shapes and walks the
bins greedily, largest share of the flops first, keeping a width only when
the whole call gets faster by more than --gain.

Per flag pair (--flags FA,FB): the tile widths are tuned on products with
those component flags and saved as that pair's table
("table_flags_AA_BB", installed by :meth:`Handle.set_tile_table_flags`),
which the library uses for products of exactly that pair.  All tables go into
one JSON file ("table", "fp64_splitk", "table_flags_AA_BB"), the format
HMAT_TUNE_TABLE reads.

    python -m paper_2609_02081_gb300.autotune --out tile_table.json          # the 512-shape batch
    python -m paper_2609_02081_gb300.autotune --shapes 256x256x256,1024x64x512
    python -m paper_2609_02081_gb300.autotune --fp64 256x256x256,128x128x2048 --out tuned.json
    python -m paper_2609_02081_gb300.autotune --flags 0x0f,0xff --shapes 4096x4096x4096 --out tuned.json
    python -m paper_2609_02081_gb300.autotune --grouped --out tuned_batch.json   # whole-batch timing
"""
from __future__ import annotations

import argparse
import json
import math
import os

import numpy as np

from . import Handle, hmat_bq_gemm, hmat_bq_gemm_grouped, hmat_workspace_size, make_desc

BINS = 16
CODES = {0: "rule", 1: 64, 2: 128, 3: 256}


def _bin(x: int) -> int:
    return min(BINS - 1, max(0, math.ceil(math.log2(max(x, 1)))))


def _time_call(h, A, B, C, ws, tol, reps, flags=(0xFF, 0xFF)):
    import torch
    stream = torch.cuda.current_stream()
    kw = dict(flagsA=flags[0], flagsB=flags[1], mode="split", tol=tol, workspace=ws, stream=stream)
    hmat_bq_gemm(h, A, B, C, **kw)   # warm
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        hmat_bq_gemm(h, A, B, C, **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune(shapes, tol: float = 1e-12, reps: int = 5, seed: int = 0, flags=(0xFF, 0xFF)):
    """Return (table, report) for the given (m, n, k) shapes of products with
    component flags `flags` = (flagsA, flagsB)."""
    import torch
    dev = torch.device("cuda")
    groups = {}
    for m, n, k in shapes:
        groups.setdefault((_bin(m), _bin(n)), []).append((m, n, k))
    table = np.zeros((BINS, BINS), dtype=np.int8)
    report = {}
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    with Handle() as h:
        for (bm, bn_), members in sorted(groups.items()):
            members.sort(key=lambda s: s[0] * s[1] * s[2])
            m, n, k = members[len(members) // 2]                    # median-work representative
            A = torch.rand((8, m, k), generator=g, device=dev, dtype=torch.float64) * 2 - 1
            B = torch.rand((8, k, n), generator=g, device=dev, dtype=torch.float64) * 2 - 1
            C = torch.empty((8, m, n), dtype=torch.float64, device=dev)
            times = {}
            for code, width in CODES.items():
                t = np.zeros((BINS, BINS), dtype=np.int8)
                t[bm, bn_] = code
                if flags == (0xFF, 0xFF):
                    h.set_tile_table(t)
                else:
                    h.set_tile_table_flags(flags[0], flags[1], t)
                nbytes = hmat_workspace_size(h, [make_desc(A, B, C, flagsA=flags[0], flagsB=flags[1])], "split", tol)
                ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
                times[width] = _time_call(h, A, B, C, ws, tol, reps, flags)
                del ws
            best = min(times, key=times.get)
            table[bm, bn_] = {"rule": 0, 64: 1, 128: 2, 256: 3}[best]
            report[f"{bm},{bn_}"] = {"shape": [m, n, k], "ms": times, "best": best, "members": len(members)}
    return table, report


def greedy_bins(order, timed, table=None, gain: float = 0.01):
    """Coordinate search over the tile-width table for one whole call.

    order: the bins (bm, bn) to visit, in that order; timed(table) -> ms of the
    call with that table installed.  Starting from `table` (default: all
    zeros, the built-in rule) each bin in turn takes the code among 0..3 whose
    table times fastest, but a change is kept only when it beats the bin's
    current code, re-timed next to the candidates, by more than the fraction
    `gain` (noise of a few tenths of a percent between timings otherwise
    moves codes back and forth).  Returns (table, report)."""
    t = np.zeros((BINS, BINS), dtype=np.int8) if table is None else np.array(table, dtype=np.int8)
    report = {}
    for b in order:
        cur = int(t[b])
        times = {}
        for code in CODES:
            trial = t.copy()
            trial[b] = code
            times[code] = timed(trial)
        best = min(times, key=times.get)
        if best != cur and times[best] < times[cur] * (1.0 - gain):
            t[b] = best
        report["%d,%d" % b] = {"ms": {CODES[c]: v for c, v in times.items()}, "kept": CODES[int(t[b])]}
    return t, report


def tune_grouped(shapes, tol: float = 1e-12, reps: int = 5, seed: int = 0, gain: float = 0.01,
                 flags=(0xFF, 0xFF)):
    """Tile widths for one grouped call over all `shapes` (m, n, k).

    Per-bin tuning (:func:`tune`) times each bin's representative alone, but
    in a grouped call the residue-GEMM items of all products share the SMs,
    so a width that is fastest alone need not be fastest in the batch.  Here
    every candidate table is timed on the whole grouped call, bins visited in
    order of their share of the flops, by :func:`greedy_bins`."""
    import torch
    dev = torch.device("cuda")
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    mats, descs, work = [], [], {}
    for m, n, k in shapes:
        A = torch.rand((8, m, k), generator=g, device=dev, dtype=torch.float64) * 2 - 1
        B = torch.rand((8, k, n), generator=g, device=dev, dtype=torch.float64) * 2 - 1
        C = torch.empty((8, m, n), dtype=torch.float64, device=dev)
        mats.append((A, B, C))
        descs.append(make_desc(A, B, C, flagsA=flags[0], flagsB=flags[1]))
        b = (_bin(m), _bin(n))
        work[b] = work.get(b, 0) + m * n * k
    order = sorted(work, key=lambda b: -work[b])
    stream = torch.cuda.current_stream()
    with Handle() as h:
        def install(t):
            if flags == (0xFF, 0xFF):
                h.set_tile_table(t)
            else:
                h.set_tile_table_flags(flags[0], flags[1], t)

        def timed(t):
            install(t)
            nbytes = hmat_workspace_size(h, descs, "split", tol)
            ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=dev)
            hmat_bq_gemm_grouped(h, descs, "split", tol, workspace=ws, stream=stream)   # warm
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                hmat_bq_gemm_grouped(h, descs, "split", tol, workspace=ws, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        rule_ms = timed(np.zeros((BINS, BINS), dtype=np.int8))
        table, report = greedy_bins(order, timed, gain=gain)
        final_ms = timed(table)
    return table, {"grouped": {"problems": len(shapes), "rule_ms": rule_ms, "tuned_ms": final_ms,
                               "gain": gain}, **report}


def _time_fp64(h, A, B, C, reps):
    import torch
    stream = torch.cuda.current_stream()
    nbytes = hmat_workspace_size(h, [make_desc(A, B, C)], "fp64")
    ws = torch.empty(max(nbytes, 1), dtype=torch.uint8, device=A.device)
    hmat_bq_gemm(h, A, B, C, mode="fp64", workspace=ws, stream=stream)   # warm
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        hmat_bq_gemm(h, A, B, C, mode="fp64", workspace=ws, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_fp64(shapes, reps: int = 5, seed: int = 0):
    """Return (split-k table, report) for FP64 products of the given (m, n, k) shapes."""
    import torch
    dev = torch.device("cuda")
    groups = {}
    for m, n, k in shapes:
        tiles = math.ceil(m / 32) * math.ceil(n / 32)
        groups.setdefault((_bin(tiles), _bin(k)), []).append((m, n, k))
    table = np.zeros((BINS, BINS), dtype=np.int8)
    report = {}
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    with Handle() as h:
        for (bt, bk), members in sorted(groups.items()):
            members.sort(key=lambda s: s[0] * s[1] * s[2])
            m, n, k = members[len(members) // 2]
            A = torch.rand((8, m, k), generator=g, device=dev, dtype=torch.float64) * 2 - 1
            B = torch.rand((8, k, n), generator=g, device=dev, dtype=torch.float64) * 2 - 1
            C = torch.empty((8, m, n), dtype=torch.float64, device=dev)
            times = {}
            for code in (1, 2, 3, 4):
                t = np.zeros((BINS, BINS), dtype=np.int8)
                t[bt, bk] = code
                h.set_fp64_splitk_table(t)
                times[1 << (code - 1)] = _time_fp64(h, A, B, C, reps)
            best = min(times, key=times.get)
            table[bt, bk] = int(math.log2(best)) + 1
            report[f"{bt},{bk}"] = {"shape": [m, n, k], "ms": times, "best_slices": best, "members": len(members)}
    return table, report


def save(table, report, path, fp64_table=None, fp64_report=None, flag_tables=None):
    """Write the tables as JSON; flag_tables: {(flagsA, flagsB): 16 x 16 codes}."""
    out = {"table": np.asarray(table).astype(int).tolist(), "report": report}
    if fp64_table is not None:
        out["fp64_splitk"] = np.asarray(fp64_table).astype(int).tolist()
        out["fp64_report"] = fp64_report
    for (fa, fb), t in (flag_tables or {}).items():
        out["table_flags_%02x_%02x" % (fa, fb)] = np.asarray(t).astype(int).tolist()
    with open(path, "w") as f:
        json.dump(out, f, indent=1)


def load(path):
    with open(path) as f:
        return np.asarray(json.load(f)["table"], dtype=np.int8)


def load_flag_tables(path):
    """The per flag pair tile tables of a tuned JSON file: {(flagsA, flagsB): table}."""
    with open(path) as f:
        data = json.load(f)
    out = {}
    for key, t in data.items():
        if key.startswith("table_flags_"):
            fa, fb = (int(x, 16) for x in key[len("table_flags_"):].split("_"))
            out[(fa, fb)] = np.asarray(t, dtype=np.int8)
    return out


def load_fp64(path):
    """The FP64 split-k table of a tuned JSON file, or None."""
    with open(path) as f:
        t = json.load(f).get("fp64_splitk")
    return None if t is None else np.asarray(t, dtype=np.int8)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--shapes", default="batch512",
                    help="'batch512' (512 log-uniform shapes in [32,1024], seed 104) or 'MxNxK,MxNxK,...'")
    ap.add_argument("--tol", type=float, default=1e-12)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--fp64", default=None, help="'MxNxK,...': also tune the FP64 split-k table on these shapes")
    ap.add_argument("--flags", default=None,
                    help="'FA,FB' (e.g. 0x0f,0xff): tune the tile widths of products with these component flags "
                         "and save them as that pair's table")
    ap.add_argument("--grouped", action="store_true",
                    help="time every candidate table on one grouped call over all the shapes "
                         "(greedy per bin) instead of each bin's representative alone")
    ap.add_argument("--gain", type=float, default=0.01,
                    help="--grouped: keep a width only when it is this fraction faster")
    ap.add_argument("--out", default="tile_table.json")
    args = ap.parse_args()
    if args.shapes == "batch512":
        import sys
        sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
        import bq_inputs
        shapes = bq_inputs.batch_shapes(104, 512)
    else:
        shapes = [tuple(int(x) for x in s.split("x")) for s in args.shapes.split(",")]
    flag_tables = None
    tuner = tune
    if args.grouped:
        def tuner(shapes, tol, reps, flags=(0xFF, 0xFF)):
            return tune_grouped(shapes, tol, reps, gain=args.gain, flags=flags)
    if args.flags:
        fa, fb = (int(x, 0) for x in args.flags.split(","))
        ftab, report = tuner(shapes, args.tol, args.reps, flags=(fa, fb))
        flag_tables = {(fa, fb): ftab}
        table = np.zeros((BINS, BINS), dtype=np.int8)      # other products keep the built-in rule
    else:
        table, report = tuner(shapes, args.tol, args.reps)
    ftable = freport = None
    if args.fp64:
        fshapes = [tuple(int(x) for x in s.split("x")) for s in args.fp64.split(",")]
        ftable, freport = tune_fp64(fshapes, args.reps)
    save(table, report, args.out, ftable, freport, flag_tables)
    print(json.dumps({"bins": len(report), "fp64_bins": len(freport or {}), "out": args.out}))


if __name__ == "__main__":
    main()
