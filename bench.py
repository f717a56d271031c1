"""Benchmark: the SpMV format sweep on one GB300 (or N independent replicas).

Workload: the format sweep over five synthetic matrices (27-point stencil
128^3, Poisson(16) random rows n = 2^20, R-MAT scale 20 edge factor 16,
banded n = 2^20 half-width 32, block-diagonal 4x4 n = 2^20), fp64 values and
vectors, int32 indices.  For each matrix the exhaustive sweep over format x
launch parameters is run first (what the selector is scored against; its per-format
best times are reported in format_sweep), then the trained selector picks a
configuration on the device (spmv_select).  One timed step = one product
y <- A x of every matrix in its selected configuration; value = 2 * (sum of
nnz) per step / step time, in GFLOP/s.  Every step streams ~2 GB, far more
than the 129 MB L2, and consecutive launches use different matrices.

Besides the timed step the JSON line carries: per_kernel (time, warm-cache
time, fraction of the measured HBM peak per matrix, and the time of a
device copy moving the same bytes in the same order: the size-matched
floor that launch and ramp costs put under small kernels), roofline (dominant
kernel, DRAM traffic from the committed ncu capture), e2e (x uploaded and y
downloaded every step, copies overlapping the products), selector (choice
vs exhaustive best, overheads, the run-time gate's predictions against
measurements), format_sweep (best time of every format per matrix, against
the format-independent byte model and the format's own bytes), batched (512
uneven fp32 matrices in one graph-captured launch), cg (conjugate gradients
on the 27-point Laplacian, default CSR vs the gate's choice), energy (NVML
energy counter, report-only), clocks, gpu_launches and cpu_baseline.

--impl reference times the fp64 CPU oracle instead (the timed baseline of
this method; there is no other reference implementation).  --traffic runs
one product per (matrix, format) in NVTX ranges for an ncu DRAM-bytes
capture and exits.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6800.0
THROTTLE_BITS = {0x1: "gpu_idle", 0x2: "applications_clocks_setting", 0x4: "sw_power_cap",
                 0x8: "hw_slowdown", 0x10: "sync_boost", 0x20: "sw_thermal_slowdown",
                 0x40: "hw_thermal_slowdown", 0x80: "hw_power_brake_slowdown",
                 0x100: "display_clock_setting"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--dtype", default="f64", choices=["f64", "f32", "bf16"])
    p.add_argument("--scale", default="full", choices=["full", "small"])
    p.add_argument("--e2e-steps", type=int, default=20)
    p.add_argument("--no-cg", action="store_true", help="skip the conjugate-gradient section")
    p.add_argument("--traffic", action="store_true",
                   help="profiling aid: one product per (matrix, format) in NVTX ranges under 'traffic', then exit")
    p.add_argument("--no-tune", action="store_true",
                   help="skip the exhaustive search (selector choice only; for launch-list captures)")
    p.add_argument("--no-energy", action="store_true", help="skip the energy report")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--only", default=None, help="comma-separated matrix names (profiling runs)")
    p.add_argument("--no-batched", action="store_true")
    p.add_argument("--batched-only", type=int, default=None, metavar="COUNT",
                   help="profiling runs: only the batched section, over COUNT matrices, then exit")
    p.add_argument("--halo", action="store_true",
                   help="--mode shard: each rank receives only the window of x its rows touch (one all-to-all)")
    p.add_argument("--mode", default="replicas", choices=["replicas", "shard"],
                   help="N > 1: independent replicas of the step (weak scaling), or every product sharded "
                        "by nnz-balanced row blocks with an all-gather of x (strong scaling)")
    p.add_argument("--fixed", default=None,
                   help="profiling runs: skip tuning and selection, run this kernel variant's default "
                        "configuration (csr, csr_split, csr_tiles, ell, coo, hyb, bsr, sell)")
    p.add_argument("--config", default=None,
                   help="profiling runs: like --fixed, with these spmv_config fields (a JSON object, "
                        "e.g. '{\"format\": 0, \"threads_per_row\": 2}')")
    return p.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def copy_floor_us(torch, stream, sizes, steps=100):
    """Size-matched floor: for each byte count, a device-to-device copy that
    reads half of it and writes the other half, in the step's order and
    timed like the step's kernels (CUDA events around each copy on the
    launching stream, each copy preceded by the previous one).  A small
    kernel pays the same launch and memory-pipeline ramp as a copy of its
    size, so kernel time against this floor separates that fixed cost from
    the kernel's own efficiency.  Returns the mean microseconds per copy."""
    bufs = [(torch.empty(max(16, b // 2), dtype=torch.uint8, device="cuda"),
             torch.empty(max(16, b // 2), dtype=torch.uint8, device="cuda")) for b in sizes]
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in sizes]
          for _ in range(steps)]
    with torch.cuda.stream(stream):
        for _ in range(3):
            for src, dst in bufs:
                dst.copy_(src)
        for s in range(steps):
            for i, (src, dst) in enumerate(bufs):
                ev[s][i][0].record(stream)
                dst.copy_(src)
                ev[s][i][1].record(stream)
    torch.cuda.synchronize()
    out = [sum(ev[s][i][0].elapsed_time(ev[s][i][1]) for s in range(steps)) * 1e3 / steps
           for i in range(len(sizes))]
    del bufs
    return out


def gather_floor_us(B, torch, stream, mats, steps=100):
    """Gather floor of every matrix (spmv_probe_gather_floor: the product's
    bytes with ideal streaming access and its x gathers, no floating-point
    instruction), launched in the step's order and timed like the step's
    kernels.  Returns the mean microseconds per launch."""
    sh = stream.cuda_stream
    for _ in range(3):
        for p in mats:
            B.spmv_probe_gather_floor(p["h"], p["x"], p["y"], sh)
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in mats]
          for _ in range(steps)]
    for s_ in range(steps):
        for i, p in enumerate(mats):
            ev[s_][i][0].record(stream)
            B.spmv_probe_gather_floor(p["h"], p["x"], p["y"], sh)
            ev[s_][i][1].record(stream)
    torch.cuda.synchronize()
    return [sum(ev[s_][i][0].elapsed_time(ev[s_][i][1]) for s_ in range(steps)) * 1e3 / steps
            for i in range(len(mats))]


def fp64_fma_peak(B, torch, stream, iterations=4096, reps=5):
    """Measured fp64 ceiling of this GPU: a full wave of independent fp64 FMA
    chains (spmv_probe_fp64_fma), best of `reps` launches after two warm-up
    launches, in TFLOP/s (2 flops per FMA)."""
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    sh = stream.cuda_stream
    for _ in range(2):
        B.spmv_probe_fp64_fma(iterations, sink, sh)
    best = None
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        count = B.spmv_probe_fp64_fma(iterations, sink, sh)
        e1.record(stream)
        torch.cuda.synchronize()
        t = e0.elapsed_time(e1) * 1e-3
        rate = 2.0 * count / t / 1e12
        best = rate if best is None else max(best, rate)
    return best


def byte_model(m, n, nnz, vt_size, vec_size, beta_nonzero=False):
    """Algorithmic bytes of one product: values + column indices of every
    nonzero, the m+1 row pointers, x once and y once (twice if beta != 0)."""
    b = nnz * (vt_size + 4) + 4 * (m + 1) + vec_size * n + vec_size * m
    if beta_nonzero:
        b += vec_size * m
    return b


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        cmd = ["nvidia-smi", "-i", str(self.gpu),
               "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active",
               "--format=csv,noheader,nounits", "-lms", "100"]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 4:
                continue
            try:
                s, m_ = float(parts[0]), float(parts[1])
                bits = int(parts[3], 16)
            except ValueError:
                continue
            if bits & 0x1:      # idle sample
                continue
            sm.append(s)
            mx.append(m_)
            for b, name in THROTTLE_BITS.items():
                if bits & b and name != "gpu_idle":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
def reference_arm(args, rank):
    """Time the fp64 CPU oracle on the same workload (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    from paper_2302_05662_gb300 import matgen
    oracle.build()
    mats = [(name, coo) for name, coo in matgen.workload_matrices(args.scale)]
    xs = {name: matgen.dense_vector(coo.n, 100 + k) for k, (name, coo) in enumerate(mats)}
    # each step: one oracle product of a bounded row sample of every matrix
    # (the first rows holding ~2M nonzeros of each), so that warmup + steps
    # stay within a few minutes
    budget = 2_000_000
    samples = []
    for name, coo in mats:
        cut = min(coo.nnz, budget)
        mrows = int(coo.rows[cut - 1]) + 1 if cut else 0
        k = int(np.searchsorted(coo.rows, mrows))
        samples.append((name, mrows, coo.n, coo.rows[:k], coo.cols[:k], coo.vals[:k], xs[name]))
    flops = sum(2 * s[3].size for s in samples)
    for _ in range(args.warmup):
        for _, mr, n, r, c, v, x in samples:
            oracle.spmv_coo(mr, n, r, c, v, x)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for _, mr, n, r, c, v, x in samples:
            oracle.spmv_coo(mr, n, r, c, v, x)
    dt = time.perf_counter() - t0
    value = flops * args.steps / dt / 1e9
    sample = (f"per step: first rows holding <= {budget} nonzeros of each of the five "
              f"matrices ({flops // 2} nonzeros), one fp64 oracle product each")
    line = {"impl": "reference", "metric": "SpMV GFLOP/s (selected format+config per matrix, 5 format-sweep matrices)",
            "value": round(value, 4), "unit": "GFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(dt / args.steps * 1e3, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(args),
            "cpu_baseline": {"value": round(value, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(value, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def workload_config(args):
    return {"workload": "format sweep over stencil27 128^3, poisson16 2^20, rmat s20 ef16, banded 2^20 w32, "
                        "blockdiag4 2^20 (CSR/ELL/COO/HYB/BSR/SELL x launch parameters); step = one product per "
                        "matrix in the configuration the selector picks",
            "scale": args.scale, "value_dtype": args.dtype, "index_dtype": "int32", "alpha": 1.0, "beta": 0.0,
            "l2": "inputs larger than L2: each step streams ~2 GB; consecutive launches use different matrices"}


def cpu_baseline(mats_host, seconds: float = 12.0):
    """The fp64 oracle as it stands, single thread: whole-matrix products of
    the five matrices, repeated in passes until about `seconds` of CPU work."""
    import oracle
    oracle.build()
    for name, coo, x in mats_host:                       # warm (page in, build)
        oracle.spmv_coo(coo.m, coo.n, coo.rows[:1], coo.cols[:1], coo.vals[:1], x)
    flops = 0
    passes = 0
    t0 = time.perf_counter()
    while True:
        for name, coo, x in mats_host:
            oracle.spmv_coo(coo.m, coo.n, coo.rows, coo.cols, coo.vals, x)
            flops += 2 * coo.nnz
        passes += 1
        t = time.perf_counter() - t0
        if t >= seconds:
            break
    return {"value": round(flops / t / 1e9, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
            "sample": f"{passes} passes of whole-matrix fp64 oracle products over the five matrices "
                      f"({t:.1f} s of one host core)"}


NAMES = ("stencil27_128^3", "poisson16_2^20", "rmat_s20_ef16", "banded_2^20_w32", "blockdiag4_2^20")

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# one ncu --set full capture of the kernel as it is now, per (kernel, matrix,
# value type); summaries and commands in profiles/.  A kernel missing here
# reports traffic null.
NCU_TRAFFIC = {
    ("sell", "banded_2^20_w32", "f64"): (835.5e6, "profiles/sell_banded_2p20_w32_f64.md"),
    ("csr", "stencil27_128^3", "f64"): (712.0e6, "profiles/csr_vector_stencil27_128_f64.md"),
    ("ell", "banded_2^20_w32", "f64"): (830.7e6, "profiles/ell_banded_2p20_w32_f64.md"),
    ("sell", "rmat_s20_ef16", "f64"): (224.96e6, "profiles/sell_rmat_s20_f64_colmajor_u1.md"),
    ("sell", "poisson16_2^20", "f64"): (218.24e6, "profiles/sell_poisson16_2p20_f64_colmajor_u1.md"),
}
FMT_KEYS = {0: "csr", 1: "ell", 2: "coo", 3: "hyb", 4: "bsr", 5: "sell"}


def fmt_name(cfg: dict) -> str:
    n = FMT_KEYS[cfg["format"]]
    if n == "csr" and cfg.get("threads_per_row") == -1:
        return "csr_tiles" if cfg.get("hyb_ell_width", 0) > 0 else "csr_split"
    return n


def format_bytes_of(B, h, cfg, m, n, xsz):
    """Bytes the configured kernel itself reads (its format arrays) plus x
    and y once: the format-actual counterpart of the byte model."""
    B.spmv_set_config(h, B.make_config(**cfg))
    return B.spmv_get_info(h).format_bytes + xsz * (n + m)


def tune_matrix(B, sweep, h, coo, x, y, timer, reps):
    """Exhaustive search on one handle: the label space, then register cap x
    unroll x carveout around the winner.  Returns (best cfg, best us,
    per-format best {name: (cfg, us)})."""
    space = sweep.label_space(include_sell=True)
    times = []
    for cfg in space:
        try:
            B.spmv_set_config(h, B.make_config(**cfg))
        except B.SpmvError:
            continue
        times.append((cfg, timer.time_us(h, x, y, reps=reps)))
    per_fmt = {}
    for cfg, t in times:
        k = fmt_name(cfg)
        if k not in per_fmt or t < per_fmt[k][1]:
            per_fmt[k] = (cfg, t)
    best_cfg, best_t = min(times, key=lambda ct: ct[1])
    for cfg in sweep.refine_space(best_cfg):
        try:
            B.spmv_set_config(h, B.make_config(**cfg))
        except B.SpmvError:
            continue
        t = timer.time_us(h, x, y, reps=reps)
        if t < best_t:
            best_cfg, best_t = cfg, t
    return best_cfg, best_t, per_fmt


def batched_section(B, matgen, torch, count=512, seed=7, steps=20, select=True):
    """512 uneven fp32 matrices: one graph-captured persistent launch (after
    the autotuner) against one spmv_run per matrix.  With `select`, every
    handle first takes the format the selector picks for it (the batch runs
    ELL and SELL matrices in their format, the others from CSR)."""
    hs, xs, ys, nnz, nbytes = [], [], [], 0, 0
    fmts = {}
    for i, coo in matgen.batched_workload(count, seed):
        r = torch.from_numpy(coo.rows).cuda()
        c = torch.from_numpy(coo.cols).cuda()
        v = torch.from_numpy(coo.vals).cuda().float()
        hs.append(B.spmv_create(coo.m, coo.n, r, c, v))
        if select:
            cfg, _ = B.spmv_select(hs[-1])
            B.spmv_set_config(hs[-1], cfg)
        f = FMT_KEYS[B.spmv_get_config(hs[-1]).format]
        fmts[f] = fmts.get(f, 0) + 1
        xs.append(torch.from_numpy(matgen.dense_vector(coo.n, 9000 + i)).float().cuda())
        ys.append(torch.zeros(coo.m, dtype=torch.float32, device="cuda"))
        nnz += coo.nnz
        nbytes += byte_model(coo.m, coo.n, coo.nnz, 4, 4)
    ones, zeros = np.ones(count), np.zeros(count)
    b = B.spmv_batch_create(hs, ones, xs, zeros, ys)
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    try:
        B.spmv_batch_tune(b)
        modes, items, tpb = B.spmv_batch_get_plan(b, count)

        def timed(fn):
            for _ in range(3):
                fn()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                fn()
            e1.record(stream)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / steps

        torch.cuda.nvtx.range_push("batched_graph")    # ncu --nvtx-include "batched_graph/"
        t_graph = timed(lambda: B.spmv_batch_launch(b, sh))
        torch.cuda.nvtx.range_pop()

        def separate():
            for k in range(count):
                B.spmv_run(hs[k], 1.0, xs[k], 0.0, ys[k], sh)
        t_sep = timed(separate)

        # the same 512 launches captured once into a CUDA graph: what one
        # kernel per matrix costs without the host's per-call overhead
        g = torch.cuda.CUDAGraph()
        separate()
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            cap = torch.cuda.current_stream().cuda_stream
            for k in range(count):
                B.spmv_run(hs[k], 1.0, xs[k], 0.0, ys[k], cap)
        t_sep_graph = timed(g.replay)
        del g
    finally:
        B.spmv_batch_destroy(b)
        for h in hs:
            B.spmv_destroy(h)
    peak, peak_kind = measured_peak()
    return {"matrices": count, "nnz": nnz, "value_dtype": "f32",
            "graph_ms": round(t_graph, 4), "graph_gflops": round(2 * nnz / (t_graph * 1e-3) / 1e9, 2),
            "algorithmic_bytes": nbytes, "gbs": round(nbytes / (t_graph * 1e-3) / 1e9, 1),
            "frac": round(nbytes / (t_graph * 1e-3) / 1e9 / peak, 4), "peak_source": peak_kind,
            "separate_launches_ms": round(t_sep, 4),
            "separate_gflops": round(2 * nnz / (t_sep * 1e-3) / 1e9, 2),
            "speedup": round(t_sep / t_graph, 3),
            "separate_launches_graph_ms": round(t_sep_graph, 4),
            "speedup_vs_graph_of_launches": round(t_sep_graph / t_graph, 3),
            "formats_selected": fmts,
            "plan": {"items": items, "threads_per_block": tpb,
                     "ell_matrices": int((modes == -1).sum()), "sell_matrices": int((modes == -5).sum()),
                     "coo_matrices": int((modes == -2).sum()), "bsr_matrices": int((modes == -4).sum()),
                     "csr_split_matrices": int((modes == 0).sum()),
                     "csr_vector_matrices": int((modes > 0).sum())}}


def cg_section(B, matgen, torch, S, have_v2, tol=1e-8, maxit=5000):
    """Conjugate gradients (spmv_cg) on the 27-point Laplacian 128^3 (centre
    26, neighbours -1), fp64, b ~ U[-1, 1]: default CSR against the
    configuration the run-time gate picks for the expected iteration count,
    with feature extraction, selection, conversion and the solver graph's
    construction counted as overhead (Section 7.5's iterative setting)."""
    coo = matgen.stencil_3d(128, 27, values="laplace")
    r = torch.from_numpy(coo.rows).cuda()
    c = torch.from_numpy(coo.cols).cuda()
    v = torch.from_numpy(coo.vals).cuda()
    h = B.spmv_create(coo.m, coo.n, r, c, v)
    del r, c, v
    b = torch.from_numpy(matgen.dense_vector(coo.m, 77)).cuda()
    x = torch.zeros(coo.m, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    vec_bytes = 11 * 8 * coo.m          # p.q 2 reads; x, r update 4 reads 2 writes; p update 2 reads 1 write
    spmv_bytes = byte_model(coo.m, coo.n, coo.nnz, 8, 8)

    def solve():
        x.zero_()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = B.spmv_cg(h, b, x, tol, maxit)
        e1.record(stream)
        torch.cuda.synchronize()
        return res, e0.elapsed_time(e1)

    def summary(res, ms):
        it = max(res.iterations, 1)
        return {"iterations": res.iterations, "converged": bool(res.converged),
                "rel_residual": float(np.sqrt(res.rho / res.bb)), "solve_ms": round(ms, 3),
                "ms_per_iteration": round(ms / it, 4),
                "gbs_per_iteration": round((spmv_bytes + vec_bytes) * it / (ms * 1e-3) / 1e9, 1)}

    try:
        t0 = time.perf_counter()
        solve()                                            # builds the default-CSR solver graph
        t_first = (time.perf_counter() - t0) * 1e3
        res_d, ms_d = solve()
        out = {"matrix": "stencil27_laplace_128^3", "nnz": coo.nnz, "tol": tol, "default_csr": summary(res_d, ms_d)}
        t0 = time.perf_counter()
        if have_v2:
            cfg, dec = B.spmv_select_runtime(h, res_d.iterations)
            out["gate"] = dec.as_dict()
            convert = bool(dec.convert)
        else:
            cfg, _ = B.spmv_select(h)
            convert = True
        t_select = (time.perf_counter() - t0) * 1e3
        t0 = time.perf_counter()
        if convert:
            B.spmv_set_config(h, cfg)
        torch.cuda.synchronize()
        t_convert = (time.perf_counter() - t0) * 1e3
        t0 = time.perf_counter()
        solve()                                            # builds the selected configuration's graph
        t_first_sel = (time.perf_counter() - t0) * 1e3
        res_s, ms_s = solve()
        applied = B.spmv_get_config(h)
        out["selected"] = dict(summary(res_s, ms_s), config=fmt_name(
            {k: getattr(applied, k) for k, _ in applied._fields_}))
        over = t_select + t_convert + max(0.0, t_first_sel - ms_s)
        out["overhead_ms"] = {"features_and_select": round(t_select, 3), "convert": round(t_convert, 3),
                              "solver_graph": round(max(0.0, t_first_sel - ms_s), 3),
                              "default_solver_graph": round(max(0.0, t_first - ms_d), 3)}
        gain_it = out["default_csr"]["ms_per_iteration"] - out["selected"]["ms_per_iteration"]
        out["break_even_iterations"] = round(over / gain_it, 1) if gain_it > 0 else None
        out["end_to_end_speedup"] = round(ms_d / (ms_s + over), 3)
    finally:
        B.spmv_destroy(h)
    return out


def energy_section(B, torch, mats, gpu_index, seconds=0.3):
    """Report-only energy objective (Section 6.3): for every matrix, the best
    configuration of each format (from the exhaustive search) replayed for
    `seconds` with the GPU's energy counter read around the loop.  Which
    format minimises energy is compared with the one that minimises time."""
    from paper_2302_05662_gb300 import energy
    try:
        nv = energy.Nvml(gpu_index)
    except (OSError, energy.NvmlError) as e:
        return {"unavailable": str(e)}
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream
    rows = []
    try:
        for p in mats:
            by = {}
            for fname, (cfg, t) in sorted(p["per_fmt"].items()):
                B.spmv_set_config(p["h"], B.make_config(**cfg))
                r = energy.measure(nv, lambda: B.spmv_run(p["h"], 1.0, p["x"], 0.0, p["y"], sh),
                                   torch.cuda.synchronize, 2.0 * p["nnz"], min_seconds=seconds)
                if r:
                    by[fname] = {"us": round(t, 2), "watts": r["watts"], "gflop_per_joule": r["gflop_per_joule"],
                                 "uj_per_product": round(r["joules_per_call"] * 1e6, 2)}
            B.spmv_set_config(p["h"], B.make_config(**p["cfg"]))
            if by:
                rows.append({"matrix": p["matrix"], "by_format": by,
                             "time_best": min(by, key=lambda f: by[f]["us"]),
                             "energy_best": max(by, key=lambda f: by[f]["gflop_per_joule"])})
    finally:
        nv.close()
    return {"per_matrix": rows, "same_choice": sum(r["time_best"] == r["energy_best"] for r in rows),
            "matrices": len(rows), "seconds_per_point": seconds,
            "note": "report-only: one GPU of a shared machine; NVML total-energy counter, read only"}


def ours(args, world, rank, local):
    import torch
    import torch.distributed as dist
    from paper_2302_05662_gb300 import binding as B
    from paper_2302_05662_gb300 import build as build_mod
    from paper_2302_05662_gb300 import matgen, replicas, sweep
    from paper_2302_05662_gb300 import selector as S

    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        build_mod.build()
    if world > 1:
        dist.barrier()
    B.load_library()
    vt = {"f64": B.SPMV_F64, "f32": B.SPMV_F32, "bf16": B.SPMV_BF16}[args.dtype]
    xdt = torch.float64 if vt == B.SPMV_F64 else torch.float32
    vsz = {"f64": 8, "f32": 4, "bf16": 2}[args.dtype]
    xsz = 8 if vt == B.SPMV_F64 else 4
    have_selector = os.path.exists(S.DEFAULT_BLOB)
    have_v2 = have_selector and S.default_is_v2()
    if have_selector:
        S.load_default_selector()
    if args.no_tune and not have_selector:
        raise SystemExit("--no-tune needs the trained selector")
    if args.batched_only:
        if rank == 0:
            print(json.dumps({"batched": batched_section(B, matgen, torch, count=args.batched_only)}), flush=True)
        return
    timer = sweep.Timer(flush="read", stat="trimmed")

    only = set(args.only.split(",")) if args.only else None
    mats = []          # per matrix: name, handle, x, y, nnz, bytes, chosen cfg
    mats_host = []
    format_sweep = []
    selector_rows = []
    for mname, coo in matgen.workload_matrices(args.scale, only=only):
        k = NAMES.index(mname) if mname in NAMES else len(mats)
        x_np = matgen.dense_vector(coo.n, 100 + k)
        mats_host.append((mname, coo, x_np))
        rows, cols, vals = sweep.device_matrix(coo, args.dtype)
        x = torch.from_numpy(x_np).to(xdt).cuda()
        y = torch.zeros(coo.m, dtype=xdt, device="cuda")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = B.spmv_create(coo.m, coo.n, rows, cols, vals)     # COO -> CSR on the device
        t_create = time.perf_counter() - t0
        del rows, cols, vals
        nnz = B.spmv_get_info(h).nnz
        t0 = time.perf_counter()
        B.spmv_features(h)
        t_feat = time.perf_counter() - t0
        nbytes = byte_model(coo.m, coo.n, nnz, vsz, xsz)
        if args.fixed or args.config:
            from paper_2302_05662_gb300.workload import SWEEP_VARIANTS
            fixed = json.loads(args.config) if args.config else dict(dict(SWEEP_VARIANTS)[args.fixed])
            B.spmv_set_config(h, B.make_config(**fixed))
            t = timer.time_us(h, x, y, reps=3)
            best_cfg, best_t, per_fmt = fixed, t, {fmt_name(fixed): (fixed, t)}
        elif args.no_tune:
            best_cfg, best_t, per_fmt = None, None, {}
        else:
            best_cfg, best_t, per_fmt = tune_matrix(B, sweep, h, coo, x, y, timer, reps=5)
        for fname, (cfg, t) in sorted(per_fmt.items()):
            gbs = nbytes / (t * 1e-6) / 1e9
            fb = format_bytes_of(B, h, cfg, coo.m, coo.n, xsz)
            format_sweep.append({"matrix": mname, "kernel": fname, "config": cfg, "us": round(t, 2),
                                 "gflops": round(2 * nnz / (t * 1e-6) / 1e9, 1), "gbs": round(gbs, 1),
                                 "format_gbs": round(fb / (t * 1e-6) / 1e9, 1)})
        chosen, source = best_cfg, ("fixed" if args.fixed or args.config else "exhaustive")
        t_sel = t_pack = None
        if have_selector and not (args.fixed or args.config):
            B.spmv_set_config(h, B.make_config(format=B.FMT_CSR))
            gate = None
            if have_v2:
                # run-time gate from default CSR: predictions against measurements
                t_def = timer.time_us(h, x, y, reps=5)
                _, d1 = B.spmv_select_runtime(h, 1)
                _, d1k = B.spmv_select_runtime(h, 1000)
                gate = {"default_csr_us": round(t_def, 2),
                        "predicted_default_csr_us": round(d1.predicted_us_current, 2),
                        "predicted_selected_us": round(d1.predicted_us_selected, 2),
                        "predicted_convert_ms": round(d1.predicted_pack_us / 1e3, 3),
                        "measured_select_ms": round(d1.measured_select_us / 1e3, 3),
                        "convert_at_1_run": int(d1.convert), "convert_at_1000_runs": int(d1k.convert)}
            t0 = time.perf_counter()
            sel_cfg, _ = B.spmv_select(h)
            t_select = time.perf_counter() - t0
            t0 = time.perf_counter()
            B.spmv_set_config(h, sel_cfg)
            t_pack = time.perf_counter() - t0
            t_sel = timer.time_us(h, x, y, reps=5)
            chosen = {kk: getattr(sel_cfg, kk) for kk, _ in sel_cfg._fields_}
            source = "selector"
            selector_rows.append({"matrix": mname, "selected": fmt_name(chosen), "selected_us": round(t_sel, 2),
                                  "best": fmt_name(best_cfg) if best_cfg else None,
                                  "best_us": round(best_t, 2) if best_t else None,
                                  "slowdown": round(t_sel / best_t, 4) if best_t else None,
                                  "overhead_ms": {"coo_to_csr": round(t_create * 1e3, 2),
                                                  "features": round(t_feat * 1e3, 3),
                                                  "select": round(t_select * 1e3, 3),
                                                  "pack_selected": round(t_pack * 1e3, 2)},
                                  "runtime_gate": gate})
        else:
            B.spmv_set_config(h, B.make_config(**best_cfg))
        info = B.spmv_get_info(h)
        mats.append({"matrix": mname, "h": h, "x": x, "y": y, "nnz": nnz, "bytes": nbytes, "cfg": chosen,
                     "source": source, "best_us": best_t, "per_fmt": per_fmt,
                     "launches": (2 if info.format == B.FMT_HYB and info.hyb_coo_nnz > 0 else 1)})
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    if args.traffic:
        # one product per (matrix, format variant) inside NVTX ranges, for
        # ncu --nvtx --nvtx-include "traffic/" with DRAM byte metrics
        from paper_2302_05662_gb300.workload import SWEEP_VARIANTS
        pairs = []
        torch.cuda.nvtx.range_push("traffic")
        for p in mats:
            for vname, kw in SWEEP_VARIANTS:
                try:
                    B.spmv_set_config(p["h"], B.make_config(**kw))
                except B.SpmvError:
                    continue
                B.spmv_run(p["h"], 1.0, p["x"], 0.0, p["y"], sh)      # warm (not in a pair range)
                torch.cuda.synchronize()
                torch.cuda.nvtx.range_push(f"{p['matrix']}|{vname}")
                B.spmv_run(p["h"], 1.0, p["x"], 0.0, p["y"], sh)
                torch.cuda.synchronize()
                torch.cuda.nvtx.range_pop()
                info = B.spmv_get_info(p["h"])
                pairs.append({"matrix": p["matrix"], "variant": vname, "bytes": p["bytes"],
                              "format_bytes": info.format_bytes + xsz * (info.m + info.n)})
        torch.cuda.nvtx.range_pop()
        if rank == 0:
            print(json.dumps({"traffic_pairs": pairs}), flush=True)
        for p in mats:
            B.spmv_destroy(p["h"])
        return

    def step(events=None):
        for i, p in enumerate(mats):
            if events is not None:
                events[i][0].record(stream)
            B.spmv_run(p["h"], 1.0, p["x"], 0.0, p["y"], sh)
            if events is not None:
                events[i][1].record(stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in mats]
          for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    gpu_index = int(vis.split(",")[local]) if vis.replace(",", "").isdigit() else local
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_index) as clk:
        torch.cuda.nvtx.range_push("timed_step")    # ncu --nvtx-include "timed_step/"
        t_start.record(stream)
        for s_ in range(args.steps):
            step(ev[s_])
        t_end.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
    if world > 1:
        dist.barrier()
    elapsed_ms = t_start.elapsed_time(t_end)
    per_ms = [statistics.mean(ev[s_][i][0].elapsed_time(ev[s_][i][1]) for s_ in range(args.steps))
              for i in range(len(mats))]
    elapsed_ms = replicas.max_over_ranks(elapsed_ms, device="cuda")
    flops_step = sum(2 * p["nnz"] for p in mats)
    value = replicas.whole_job_rate(flops_step, args.steps, world, elapsed_ms) / 1e9

    # end to end through the C ABI: x from pinned host memory, y back to it
    xs_host = [p["x"].cpu().pin_memory() for p in mats]
    ys_host = [torch.empty(p["y"].numel(), dtype=xdt).pin_memory() for p in mats]
    h2d = sum(t.numel() * t.element_size() for t in xs_host)
    d2h = sum(t.numel() * t.element_size() for t in ys_host)

    # copies overlap the products: x of matrix i+1 goes up and y of matrix
    # i-1 comes down while matrix i multiplies.  Per matrix, the upload waits
    # for the previous step's product (it overwrites x), the product for its
    # upload and for the previous step's download of y (it overwrites y).
    up, down = torch.cuda.Stream(), torch.cuda.Stream()
    ev = lambda: torch.cuda.Event()
    in_done, k_done, out_done = ([ev() for _ in mats] for _ in range(3))

    def e2e_step():
        for i, p in enumerate(mats):
            up.wait_event(k_done[i])
            with torch.cuda.stream(up):
                p["x"].copy_(xs_host[i], non_blocking=True)
            in_done[i].record(up)
        for i, p in enumerate(mats):
            stream.wait_event(in_done[i])
            stream.wait_event(out_done[i])
            B.spmv_run(p["h"], 1.0, p["x"], 0.0, p["y"], sh)
            k_done[i].record(stream)
            down.wait_event(k_done[i])
            with torch.cuda.stream(down):
                ys_host[i].copy_(p["y"], non_blocking=True)
            out_done[i].record(down)

    e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    up.wait_event(e0)
    for _ in range(args.e2e_steps):
        e2e_step()
    for d in out_done:
        stream.wait_event(d)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    for i, p in enumerate(mats):        # the downloaded results are the products
        if not torch.equal(ys_host[i], p["y"].cpu()):
            raise SystemExit(f"e2e: downloaded y of {p['matrix']} differs from the device result")
    e2e_ms = replicas.max_over_ranks(e2e_ms, device="cuda")
    e2e_value = replicas.whole_job_rate(flops_step, args.e2e_steps, world, e2e_ms) / 1e9

    # warm cache: each matrix back to back (x, y and much of the matrix stay in L2 when it fits)
    warm_us = []
    for p in mats:
        for _ in range(3):
            B.spmv_run(p["h"], 1.0, p["x"], 0.0, p["y"], sh)
        w0, w1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0.record(stream)
        for _ in range(50):
            B.spmv_run(p["h"], 1.0, p["x"], 0.0, p["y"], sh)
        w1.record(stream)
        torch.cuda.synchronize()
        warm_us.append(w0.elapsed_time(w1) * 1e3 / 50)

    copy_us = copy_floor_us(torch, stream, [p["bytes"] for p in mats])
    gather_us = gather_floor_us(B, torch, stream, mats)
    fp64_tflops = fp64_fma_peak(B, torch, stream)

    peak, peak_kind = measured_peak()
    per_kernel = []
    for p, ms, wu, cu, gu in zip(mats, per_ms, warm_us, copy_us, gather_us):
        gbs = p["bytes"] / (ms * 1e-3) / 1e9
        tflops = 2 * p["nnz"] / (ms * 1e-3) / 1e12
        row = {"matrix": p["matrix"], "kernel": fmt_name(p["cfg"]), "config": p["cfg"],
               "source": p["source"], "us": round(ms * 1e3, 2), "warm_cache_us": round(wu, 2),
               "gflops": round(tflops * 1e3, 1), "gbs": round(gbs, 1),
               "frac": round(gbs / peak, 4), "copy_floor_us": round(cu, 2),
               "frac_of_copy": round(cu / (ms * 1e3), 4), "gather_floor_us": round(gu, 2),
               "frac_of_gather_floor": round(gu / (ms * 1e3), 4)}
        if vt == B.SPMV_F64:   # one fp64 FMA per nonzero: the second ceiling
            row["fp64_frac"] = round(tflops / fp64_tflops, 4)
        per_kernel.append(row)
    dom = max(range(len(mats)), key=lambda i: per_ms[i])
    dp = mats[dom]
    achieved = dp["bytes"] / (per_ms[dom] * 1e-3) / 1e9
    tr = NCU_TRAFFIC.get((fmt_name(dp["cfg"]), dp["matrix"], args.dtype))
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": tr[0] if tr else None,
                "traffic_source": tr[1] if tr else None,
                "kernel": f"{fmt_name(dp['cfg'])} on {dp['matrix']}",
                "algorithmic_bytes_per_launch": dp["bytes"], "peak_source": peak_kind,
                "time_share": round(per_ms[dom] / sum(per_ms), 3),
                "fp64_fma_peak_tflops": round(fp64_tflops, 4)}
    if vt == B.SPMV_F64:
        # fp64 values: one FMA per nonzero against the measured fp64 FMA
        # rate; the roofline is whichever ceiling the kernel is closer to
        fp_ach = 2 * dp["nnz"] / (per_ms[dom] * 1e-3) / 1e12
        roofline["hbm_frac"] = roofline["frac"]
        roofline["fp64_frac"] = round(fp_ach / fp64_tflops, 4)
        if fp_ach / fp64_tflops > achieved / peak:
            roofline.update({"bound": "alu", "achieved": round(fp_ach, 4), "peak": round(fp64_tflops, 4),
                             "unit": "TFLOP/s", "frac": round(fp_ach / fp64_tflops, 4),
                             "peak_source": "measured fp64 FMA microkernel (spmv_probe_fp64_fma)"})
    for fs in format_sweep:
        fs["frac"] = round(fs["gbs"] / peak, 4)
        fs["format_frac"] = round(fs["format_gbs"] / peak, 4)
    clocks = clk.summary()
    batched = cg = None
    if not args.no_batched and only is None and not (args.fixed or args.config):
        batched = batched_section(B, matgen, torch)
    energy_rep = None
    if not args.no_energy and not (args.fixed or args.config):
        energy_rep = energy_section(B, torch, mats, gpu_index)
    profiling = bool(args.fixed or args.config)
    if not args.no_cg and only is None and not profiling and args.scale == "full" and vt == B.SPMV_F64:
        cg = cg_section(B, matgen, torch, S, have_v2)
    if rank != 0:
        for p in mats:
            B.spmv_destroy(p["h"])
        return
    cpu = None if args.no_cpu_baseline else cpu_baseline(mats_host)
    cfg = workload_config(args)
    cfg["parallelism"] = f"replicas{world}" if world > 1 else "single"
    cfg["matrices"] = {p["matrix"]: p["nnz"] for p in mats}
    sel_summary = None
    if selector_rows and all(r["slowdown"] for r in selector_rows):
        sl = np.array([r["slowdown"] for r in selector_rows])
        sel_summary = {"per_matrix": selector_rows, "geomean_slowdown": round(float(np.exp(np.mean(np.log(sl)))), 4),
                       "within_10pct": float(np.mean(sl <= 1.10))}
    line = {"metric": "SpMV GFLOP/s (selected format+config per matrix, 5 format-sweep matrices)",
            "value": round(value, 2), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic", "config": cfg,
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": round(e2e_value, 2), "unit": "GFLOP/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "clocks": clocks, "gpu_launches": sum(p["launches"] for p in mats) * args.steps,
            "per_kernel": per_kernel, "selector": sel_summary, "format_sweep": format_sweep,
            "batched": batched, "cg": cg, "energy": energy_rep}
    print(json.dumps(line), flush=True)
    for p in mats:
        B.spmv_destroy(p["h"])


def shard_bench(args, world, rank, local):
    """Strong scaling of the step: every matrix is split into nnz-balanced
    row blocks, one per rank (each rank's block a handle in the configuration
    the selector picks for it); x lives in equal blocks and one all-gather
    per product assembles it on every rank.  value = the step's flops over
    the slowest rank's time."""
    import torch
    import torch.distributed as dist
    from paper_2302_05662_gb300 import binding as B
    from paper_2302_05662_gb300 import build as build_mod
    from paper_2302_05662_gb300 import matgen, replicas, shard, sweep
    from paper_2302_05662_gb300 import selector as S

    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        build_mod.build()
    if world > 1:
        dist.barrier()
    B.load_library()
    if os.path.exists(S.DEFAULT_BLOB):
        S.load_default_selector()
    xdt = torch.float64 if args.dtype == "f64" else torch.float32
    only = set(args.only.split(",")) if args.only else None
    mats, flops, exchanged = [], 0, 0
    for k, (mname, coo) in enumerate(matgen.workload_matrices(args.scale, only=only)):
        rp = np.zeros(coo.m + 1, np.int64)
        np.cumsum(np.bincount(coo.rows, minlength=coo.m), out=rp[1:])
        bounds = shard.partition_rows(rp, world)
        r0, r1 = int(bounds[rank]), int(bounds[rank + 1])
        lr, lc, lv = shard.local_triplets(coo.rows, coo.cols, coo.vals, r0, r1)
        sub = matgen.Coo(r1 - r0, coo.n, lr.astype(np.int32), lc, lv)
        rows, cols, vals = sweep.device_matrix(sub, args.dtype)
        sm = shard.ShardedMatrix(coo.m, coo.n, rows + r0, cols, vals, bounds, rank, world, halo=args.halo)
        exchanged += sm.exchanged_entries()
        del rows, cols, vals
        cfg, _ = B.spmv_select(sm.h)
        B.spmv_set_config(sm.h, cfg)
        x = matgen.dense_vector(coo.n, 100 + k)
        xl = torch.zeros(sm.blk, dtype=xdt)
        part = x[rank * sm.blk:(rank + 1) * sm.blk]
        xl[:part.size] = torch.from_numpy(part)
        mats.append((sm, xl.cuda(), torch.zeros(r1 - r0, dtype=xdt, device="cuda")))
        flops += 2 * coo.nnz
    stream = torch.cuda.current_stream()

    def step():
        for sm, xl, y in mats:
            sm.run(1.0, xl, 0.0, y, stream=stream.cuda_stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = replicas.max_over_ranks(e0.elapsed_time(e1), device="cuda")
    value = flops * args.steps / (ms * 1e-3) / 1e9
    if rank == 0:
        cfgd = workload_config(args)
        cfgd["parallelism"] = f"rowshard{world}"
        cfgd["x_exchange"] = "halo all-to-all" if args.halo else "all-gather"
        cfgd["x_entries_received_per_step_rank0"] = exchanged
        print(json.dumps({"metric": "SpMV GFLOP/s (row-block sharded product, 5 format-sweep matrices)",
                          "value": round(value, 2), "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
                          "warmup": args.warmup, "ms_per_step": round(ms / args.steps, 4),
                          "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                          "dtype": args.dtype, "data": "synthetic", "config": cfgd,
                          "gpu_launches": None}), flush=True)
    for sm, _, _ in mats:
        sm.destroy()


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    if args.mode == "shard":
        shard_bench(args, world, rank, local)
    else:
        ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
