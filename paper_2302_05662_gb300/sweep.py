"""Exhaustive search over the tuned space: format x kernel/launch parameters.

The paper labels each matrix with the configuration that measured best
(Section 5.4, Step 2: a dataset of diverse matrices run under many
configurations) and learns to predict it.  This module times every point of
the space on the GPU through the C ABI: CUDA-event timing on the launching
stream, the L2 flushed between repetitions, median of the repetitions.
Results go to a JSON-lines file, one record per (matrix, configuration);
a rerun skips records already present (checkpoint/resume).

The space (Section 4 knobs 1-4, plus threads per row and unroll):
  CSR  threads_per_row in {1,2,4,8,16,32} or the nnz-balanced split,
  ELL, COO, HYB, BSR (r in {2, 4}),
  each at threads_per_block in {32, 64, 128, 256, 512, 1024}.
The register cap, unroll and L1/shared carveout are refined on the winner.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import time

import numpy as np

from . import binding as B

TPB = (32, 64, 128, 256, 512, 1024)
CSR_TPR = (1, 2, 4, 8, 16, 32, B.TPR_SPLIT)


def label_space(tpb=TPB, include_sell: bool = False):
    """The selector's label space: (format, threads_per_block, threads_per_row)
    points, each a dict of spmv_config fields.  include_sell adds the six
    SELL points (the committed selector's 78 classes include them; its SELL
    timings come from a supplementary sweep)."""
    out = []
    if include_sell:
        out += [dict(format=B.FMT_SELL, threads_per_block=t) for t in tpb]
    for t in tpb:
        for tpr in CSR_TPR:
            out.append(dict(format=B.FMT_CSR, threads_per_block=t, threads_per_row=tpr))
        out.append(dict(format=B.FMT_ELL, threads_per_block=t))
        out.append(dict(format=B.FMT_COO, threads_per_block=t))
        out.append(dict(format=B.FMT_HYB, threads_per_block=t))
        for s in (1, 4):
            out.append(dict(format=B.FMT_BSR, threads_per_block=t, threads_per_row=s, bsr_block=4))
    return out


def refine_space(best: dict):
    """Register cap x unroll x carveout around a winning point (x SELL's
    column groups: column-major or groups of four; x split CSR's form: warp
    chunks, or staged tiles of 1024 or 4096 nonzeros; x vector CSR's load
    group of 4 or 8 entries)."""
    out = []
    ell_family = best.get("format", 0) in (B.FMT_ELL, B.FMT_HYB, B.FMT_SELL)
    if best.get("format", 0) == B.FMT_SELL:
        groups = [("bsr_block", 1), ("bsr_block", 4)]             # SELL column groups
    elif best.get("format", 0) == B.FMT_CSR and best.get("threads_per_row") == B.TPR_SPLIT:
        groups = [("hyb_ell_width", w) for w in (0, 1024, 4096)]  # split CSR form
    elif best.get("format", 0) == B.FMT_CSR and best.get("threads_per_row", 0) in (0, 1, 2):
        groups = [("bsr_block", 4), ("bsr_block", 8)]             # CSR load group (1-2 lanes per row)
    else:
        groups = [None]
    for rc in ((32, 48, 64) if ell_family else (32, 64)):
        for u in ((1, 2, 4, 8) if ell_family else (1, 2, 4)):
            for cv in (-1, 0, 100):
                for g in groups:
                    d = dict(best)
                    d.update(regcap=rc, unroll=u, carveout=cv)
                    if g is not None:
                        d[g[0]] = g[1]
                    out.append(d)
    return out


def config_key(d: dict) -> str:
    return ",".join(f"{k}={d[k]}" for k in sorted(d))


class Timer:
    """Times spmv_run on one handle with CUDA events, flushing L2 between
    repetitions with a buffer twice the L2 size.

    flush="write" zeroes the buffer between repetitions: the dirty lines it
    leaves are written back while the timed product runs, which slowed
    products of 2 to 30 million nonzeros by 4-19% against flush="read" (the
    buffer is read, leaving no dirty line) in the same session on GB300.  stat:
    "median" of the repetitions, or "trimmed" (the mean of the middle 60%):
    the event timer of this GPU ticks in steps of about 2.05 us, so the
    median of a 9 us product is always a whole number of ticks, while the
    mean of repetitions started at unrelated timer phases resolves it."""

    def __init__(self, l2_bytes: int = 129 * 2**20, flush: str = "write", stat: str = "median"):
        import torch
        self.torch = torch
        self.flush = flush
        self.stat = stat
        self.flush_buf = torch.zeros(2 * l2_bytes // 4, dtype=torch.int32, device="cuda")

    def _flush(self):
        if self.flush == "read":
            self.flush_buf.max()
        else:
            self.flush_buf.zero_()

    def time_us(self, h, x, y, reps: int = 7, warm: int = 1) -> float:
        torch = self.torch
        stream = torch.cuda.current_stream()
        for _ in range(warm):
            B.spmv_run(h, 1.0, x, 0.0, y, stream.cuda_stream)
        ts = []
        for _ in range(reps):
            self._flush()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            B.spmv_run(h, 1.0, x, 0.0, y, stream.cuda_stream)
            e1.record(stream)
            e1.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3)
        return summarize(ts, self.stat)


def summarize(ts, stat: str = "median") -> float:
    """Median, or mean of the middle 60% (stat="trimmed"), of timings."""
    if stat != "trimmed" or len(ts) < 5:
        return statistics.median(ts)
    v = sorted(ts)
    k = len(v) // 5
    return statistics.fmean(v[k:len(v) - k])


def device_matrix(coo, value_dtype="f64"):
    import torch
    from . import matgen
    rows = torch.from_numpy(coo.rows).cuda()
    cols = torch.from_numpy(coo.cols).cuda()
    if value_dtype == "bf16":
        bits = matgen.bf16_bits(matgen.round_to_bf16(coo.vals)).view(np.int16)
        vals = torch.from_numpy(bits).cuda().view(torch.bfloat16)
    else:
        vals = torch.from_numpy(coo.vals).cuda().to(torch.float64 if value_dtype == "f64" else torch.float32)
    return rows, cols, vals


def sweep_matrix(coo, space, timer: Timer, reps=7, value_dtype="f64", seed=0):
    """Time every configuration of `space` on one matrix.  Returns a list of
    (config dict, median microseconds or None when the format is refused)."""
    import torch
    rows, cols, vals = device_matrix(coo, value_dtype)
    xdt = torch.float64 if value_dtype == "f64" else torch.float32
    x = torch.from_numpy(np.random.default_rng(seed).uniform(-1, 1, coo.n)).to(xdt).cuda()
    y = torch.zeros(coo.m, dtype=xdt, device="cuda")
    h = B.spmv_create(coo.m, coo.n, rows, cols, vals)
    out = [None] * len(space)
    # visit configurations grouped by what must be re-packed, so a change of
    # launch parameters alone reuses the packed arrays
    def pack_key(i):
        c = space[i]
        return (c.get("format", 0), c.get("threads_per_row", 0), c.get("bsr_block", 4), c.get("unroll", 0),
                c.get("hyb_ell_width", 0))
    refused = set()
    try:
        for i in sorted(range(len(space)), key=pack_key):
            cfg = space[i]
            if pack_key(i) in refused:
                out[i] = (cfg, None)
                continue
            try:
                B.spmv_set_config(h, B.make_config(**cfg))
            except B.SpmvError as e:
                if e.status == -4:
                    refused.add(pack_key(i))
                out[i] = (cfg, None)
                continue
            out[i] = (cfg, timer.time_us(h, x, y, reps=reps))
    finally:
        B.spmv_destroy(h)
    return out


def matrix_features(coo):
    """Device-computed features (spmv_features) of a matrix."""
    rows, cols, vals = device_matrix(coo)
    h = B.spmv_create(coo.m, coo.n, rows, cols, vals)
    try:
        return B.spmv_features(h)
    finally:
        B.spmv_destroy(h)


def default_csr(coo) -> dict:
    """The 'default CSR' baseline: CSR with the library's default threads per
    row and 256 threads per block."""
    return dict(format=B.FMT_CSR, threads_per_block=256, threads_per_row=0)


def generate_dataset_matrix(idx: int, n_lo=1e3, n_hi=2.1e6):
    """Matrix idx of the selector dataset: family by index, n log-uniform in
    [n_lo, n_hi] from the matrix seed, family parameters jittered."""
    from . import matgen
    rng = np.random.default_rng(10_000 + idx)
    fam = matgen.FAMILIES[idx % len(matgen.FAMILIES)]
    n = int(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))))
    return fam, matgen.family_matrix(fam, n, seed=20_000 + idx, jitter=True)


def calibrate_pack(indices, out_path, reps: int = 3):
    """Conversion-cost calibration: for dataset matrices `indices`, the wall
    time of spmv_set_config from default CSR to each format (CSR as the
    split variant), median of `reps`.  Appends JSON lines {matrix, format,
    nnz, m, us}."""
    import torch
    with open(out_path, "a") as fh:
        for idx in indices:
            fam, coo = generate_dataset_matrix(idx)
            rows, cols, vals = device_matrix(coo)
            h = B.spmv_create(coo.m, coo.n, rows, cols, vals)
            del rows, cols, vals
            try:
                for f in range(6):
                    cfg = dict(format=f)
                    if f == B.FMT_CSR:
                        cfg["threads_per_row"] = B.TPR_SPLIT
                    ts = []
                    for _ in range(reps):
                        B.spmv_set_config(h, B.make_config(format=B.FMT_CSR))
                        torch.cuda.synchronize()
                        t0 = time.perf_counter()
                        try:
                            B.spmv_set_config(h, B.make_config(**cfg))
                        except B.SpmvError:
                            ts = None
                            break
                        ts.append((time.perf_counter() - t0) * 1e6)
                    us = statistics.median(ts) if ts else None
                    fh.write(json.dumps({"matrix": idx, "family": fam, "format": f, "nnz": coo.nnz, "m": coo.m,
                                         "us": us}) + "\n")
                fh.flush()
            finally:
                B.spmv_destroy(h)


def best_label(records_by_matrix: dict, idx: int):
    """The fastest label configuration of matrix idx over its sweep records
    (the main sweep and any supplementary format sweep), as a config dict."""
    best = None
    for rec in records_by_matrix.get(idx, []):
        for key, us in rec["times"]:
            if us is not None and (best is None or us < best[1]):
                best = (key, us)
    if best is None:
        return None
    return {kv.split("=")[0]: int(kv.split("=")[1]) for kv in best[0].split(",")}


def refine_sweep(args, timer):
    """Register cap x unroll x carveout (refine_space) around each matrix's
    best label configuration from earlier sweep records, timed in one
    session together with that configuration at the library defaults.
    Appends {matrix, family, best, best_us, refine: [[key, us], ...]}."""
    import gzip
    import ast
    by = {}
    for path in args.refine_from:
        with (gzip.open(path, "rt") if path.endswith(".gz") else open(path)) as fh:
            for line in fh:
                r = json.loads(line)
                t = r["times"]
                r["times"] = ast.literal_eval(t) if isinstance(t, str) else t
                by.setdefault(r["matrix"], []).append(r)
    done = set()
    if os.path.exists(args.out):
        with open(args.out) as fh:
            done = {json.loads(l)["matrix"] for l in fh if l.strip()}
    t0 = time.time()
    with open(args.out, "a") as fh:
        for idx in range(args.start, args.start + args.count):
            if idx in done or idx not in by:
                continue
            if time.time() - t0 > args.time_budget:
                break
            best = best_label(by, idx)
            if best is None:
                continue
            fam, coo = generate_dataset_matrix(idx, n_hi=args.n_hi)
            space = [dict(best)] + refine_space(best)
            res = sweep_matrix(coo, space, timer, reps=args.reps, value_dtype=args.dtype, seed=idx)
            fh.write(json.dumps({"matrix": idx, "family": fam, "dtype": args.dtype, "best": config_key(best),
                                 "best_us": res[0][1],
                                 "refine": [[config_key(c), t] for c, t in res[1:]]}) + "\n")
            fh.flush()


def _cfg_dict(cfg) -> dict:
    """spmv_config (ctypes) as a dict of its fields."""
    return {k: int(getattr(cfg, k)) for k in ("format", "threads_per_block", "threads_per_row", "unroll",
                                              "regcap", "carveout", "bsr_block", "hyb_ell_width")}


def label_key(cfg: dict) -> str:
    """Key of the label point a full configuration belongs to (format and
    threads per block; threads per row for CSR and BSR; BSR's block size)."""
    keep = {"format": cfg["format"], "threads_per_block": cfg["threads_per_block"]}
    if cfg["format"] in (B.FMT_CSR, B.FMT_BSR):
        keep["threads_per_row"] = cfg["threads_per_row"]
    if cfg["format"] == B.FMT_BSR:
        keep["bsr_block"] = cfg["bsr_block"]
    return config_key(keep)


def retime(coo, cfgs, timer: Timer, reps: int, value_dtype="f64", seed=0):
    """Microseconds of each configuration (the timer's statistic of `reps`
    repetitions), one handle per configuration, repetitions interleaved
    across the configurations (so a drift of the GPU's state during the
    session affects them alike)."""
    import torch
    rows, cols, vals = device_matrix(coo, value_dtype)
    xdt = torch.float64 if value_dtype == "f64" else torch.float32
    x = torch.from_numpy(np.random.default_rng(seed).uniform(-1, 1, coo.n)).to(xdt).cuda()
    y = torch.zeros(coo.m, dtype=xdt, device="cuda")
    hs = []
    try:
        for c in cfgs:
            hs.append(B.spmv_create(coo.m, coo.n, rows, cols, vals, B.make_config(**c)))
        ts = [[] for _ in cfgs]
        for _ in range(reps):
            for j, h in enumerate(hs):
                ts[j].append(timer.time_us(h, x, y, reps=1, warm=1))
        return [summarize(t, timer.stat) for t in ts]
    finally:
        for h in hs:
            B.spmv_destroy(h)


def heldout_eval(args):
    """The selector's evaluation on held-out matrices, in one session: the
    device selector's pick (spmv_select: features and MLP on the GPU), the
    exhaustive search over the label space, the register cap x unroll x
    carveout space around its winner, then the winner, the pick and default
    CSR timed again with interleaved repetitions, so that the slowdown of
    the pick is measured against the refined exhaustive best's own re-timed
    time rather than the minimum of many noisy timings.  Appends one JSON
    line per matrix."""
    from . import selector as S
    if args.blob:  # this blob for every value type
        S.load_default_selector(args.blob, lowp_path=None, bf16_path=None)
    else:
        S.load_default_selector()
    timer = Timer(flush=args.flush, stat=args.stat)
    table = {}
    if args.knob_table:
        with open(args.knob_table) as fh:
            table = json.load(fh).get("knob_table", {})
    space = label_space(include_sell=True)
    done = set()
    if os.path.exists(args.out):
        with open(args.out) as fh:
            done = {json.loads(l)["matrix"] for l in fh if l.strip()}
    t0 = time.time()
    with open(args.out, "a") as fh:
        for idx in range(args.start, args.start + args.count):
            if idx in done:
                continue
            if time.time() - t0 > args.time_budget:
                break
            fam, coo = generate_dataset_matrix(idx, n_hi=args.n_hi)
            rows, cols, vals = device_matrix(coo, args.dtype)
            h = B.spmv_create(coo.m, coo.n, rows, cols, vals)
            try:
                pick = _cfg_dict(B.spmv_select(h)[0])
            finally:
                B.spmv_destroy(h)
            del rows, cols, vals
            res = sweep_matrix(coo, space, timer, reps=args.reps, value_dtype=args.dtype, seed=idx)
            ok = [(c, t) for c, t in res if t is not None]
            cbest, tbest = min(ok, key=lambda ct: ct[1])
            ref = sweep_matrix(coo, refine_space(cbest), timer, reps=args.reps, value_dtype=args.dtype, seed=idx)
            okr = [(c, t) for c, t in ref if t is not None]
            winner = min(ok + okr, key=lambda ct: ct[1])[0]
            cands = {"winner": winner, "pick": pick, "default_csr": default_csr(coo)}
            pkey = label_key(pick)
            if pkey in table:
                cands["pick_knob_table"] = dict(pick, **table[pkey])
            names = list(cands)
            final = retime(coo, [cands[k] for k in names], timer, args.final_reps, args.dtype, seed=idx)
            fh.write(json.dumps({"matrix": idx, "family": fam, "m": coo.m, "nnz": coo.nnz, "dtype": args.dtype,
                                 "flush": args.flush, "pick": pkey, "winner": config_key(winner),
                                 "search_best_us": min(t for _, t in ok + okr),
                                 "labels": [[config_key(c), t] for c, t in res],
                                 "refine": [[config_key(c), t] for c, t in ref],
                                 "final": {k: round(v, 3) for k, v in zip(names, final)}}) + "\n")
            fh.flush()


def main():
    ap = argparse.ArgumentParser(description="exhaustive format/launch sweep")
    ap.add_argument("--start", type=int, default=0)
    ap.add_argument("--count", type=int, default=10)
    ap.add_argument("--out", required=True)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--n-hi", type=float, default=2.1e6)
    ap.add_argument("--time-budget", type=float, default=1e9, help="seconds; stop cleanly after")
    ap.add_argument("--calibrate-pack", action="store_true",
                    help="time format conversions of matrices start..start+count instead")
    ap.add_argument("--dtype", default="f64", choices=["f64", "f32", "bf16"],
                    help="value type of the swept matrices (labels for a per-precision selector)")
    ap.add_argument("--formats", default=None,
                    help="comma list (csr,ell,coo,hyb,bsr,sell): a supplementary sweep of these formats' "
                         "label points only, merged into earlier records by the selector trainer")
    ap.add_argument("--refine-from", nargs="*", default=None,
                    help="sweep records: time the register cap x unroll x carveout space around each "
                         "matrix's best label configuration instead")
    ap.add_argument("--heldout-eval", action="store_true",
                    help="evaluate the committed selector on matrices start..start+count: its device pick "
                         "against the refined exhaustive best, both re-timed in one session")
    ap.add_argument("--flush", default="write", choices=["write", "read"], help="L2 flush between repetitions")
    ap.add_argument("--stat", default="median", choices=["median", "trimmed"],
                    help="statistic of the repetitions (trimmed: mean of the middle 60%%)")
    ap.add_argument("--final-reps", type=int, default=21, help="interleaved repetitions of the final re-timing")
    ap.add_argument("--blob", default=None, help="selector blob evaluated by --heldout-eval (default: the committed "
                                                 "blobs for each value type)")
    ap.add_argument("--knob-table", default=None,
                    help="selector report JSON whose knob_table is also evaluated (heldout-eval)")
    args = ap.parse_args()
    from . import build
    build.build()
    B.load_library()
    if args.heldout_eval:
        heldout_eval(args)
        return
    if args.refine_from:
        refine_sweep(args, Timer(flush=args.flush, stat=args.stat))
        return
    if args.calibrate_pack:
        calibrate_pack(range(args.start, args.start + args.count), args.out)
        return
    done = set()
    if os.path.exists(args.out):
        with open(args.out) as fh:
            for line in fh:
                try:
                    done.add(json.loads(line)["matrix"])
                except Exception:
                    pass
    timer = Timer(flush=args.flush, stat=args.stat)
    space = label_space(include_sell=True)
    if args.formats is not None:
        names = {"csr": B.FMT_CSR, "ell": B.FMT_ELL, "coo": B.FMT_COO, "hyb": B.FMT_HYB, "bsr": B.FMT_BSR,
                 "sell": B.FMT_SELL}
        keep = {names[f] for f in args.formats.split(",")}
        space = [c for c in space if c["format"] in keep]
    t0 = time.time()
    with open(args.out, "a") as fh:
        for idx in range(args.start, args.start + args.count):
            if idx in done:
                continue
            if time.time() - t0 > args.time_budget:
                break
            fam, coo = generate_dataset_matrix(idx, n_hi=args.n_hi)
            res = sweep_matrix(coo, space + [default_csr(coo)], timer, reps=args.reps, value_dtype=args.dtype,
                               seed=idx)
            rec = {"matrix": idx, "family": fam, "m": coo.m, "n": coo.n, "nnz": coo.nnz, "dtype": args.dtype,
                   "default_us": res[-1][1], "times": [[config_key(c), t] for c, t in res[:-1]]}
            if args.formats is None:
                rec["features"] = [float(v) for v in matrix_features(coo)]
            else:
                rec["supplement"] = args.formats
            fh.write(json.dumps(rec) + "\n")
            fh.flush()


if __name__ == "__main__":
    main()
