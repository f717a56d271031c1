"""Benchmark: the SpMV format sweep on one GB300 (or N independent replicas).

One step = y <- alpha*A*x + beta*y (alpha = 1, beta = 0) once for every
(matrix, kernel variant) pair of the format sweep: five synthetic matrices
(27-point stencil 128^3, Poisson(16) random rows n = 2^20, R-MAT scale 20
edge factor 16, banded n = 2^20 half-width 32, block-diagonal 4x4 n = 2^20)
times six kernels (vector CSR, split CSR, ELL, COO, HYB, BSR), fp64 values
and vectors with int32 indices.  value = 2 * (sum of nnz over the pairs) per
step / step time, in GFLOP/s.  Every step streams several GB, far more than
the 129 MB L2, and launches are ordered variant-major so that a kernel's
matrix has been evicted by the kernels launched in between.

--impl reference times the fp64 CPU oracle instead (the timed baseline of
this method; there is no other reference implementation).
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
    p.add_argument("--steps", type=int, default=400)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--dtype", default="f64", choices=["f64", "f32", "bf16"])
    p.add_argument("--scale", default="full", choices=["full", "small"])
    p.add_argument("--e2e-steps", type=int, default=20)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--only", default=None, help="comma-separated matrix names (profiling runs)")
    p.add_argument("--kernels", default=None, help="comma-separated kernel variants (profiling runs)")
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
    line = {"impl": "reference", "metric": "SpMV GFLOP/s (format sweep, 5 matrices x 6 kernels)",
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
    return {"workload": "format sweep: stencil27 128^3, poisson16 2^20, rmat s20 ef16, banded 2^20 w32, "
                        "blockdiag4 2^20; kernels csr, csr_split, ell, coo, hyb, bsr",
            "scale": args.scale, "value_dtype": args.dtype, "index_dtype": "int32", "alpha": 1.0, "beta": 0.0,
            "l2": "inputs larger than L2: each step streams several GB; launches are variant-major"}


def cpu_baseline(mats_host):
    """The fp64 oracle as it stands, single thread, on a bounded sample."""
    import oracle
    oracle.build()
    budget = 4_000_000
    flops = 0
    t = 0.0
    for name, coo, x in mats_host:
        cut = min(coo.nnz, budget)
        mrows = int(coo.rows[cut - 1]) + 1 if cut else 0
        k = int(np.searchsorted(coo.rows, mrows))
        r, c, v = coo.rows[:k], coo.cols[:k], coo.vals[:k]
        oracle.spmv_coo(mrows, coo.n, r, c, v, x)        # warm
        t0 = time.perf_counter()
        reps = 3
        for _ in range(reps):
            oracle.spmv_coo(mrows, coo.n, r, c, v, x)
        t += time.perf_counter() - t0
        flops += 2 * k * reps
    return {"value": round(flops / t / 1e9, 4), "unit": "GFLOP/s", "cores": 1, "kind": "oracle",
            "sample": f"first rows holding <= {budget} nonzeros of each of the five matrices, "
                      f"3 fp64 oracle products each"}


def ours(args, world, rank, local):
    import torch
    import torch.distributed as dist
    from paper_2302_05662_gb300 import binding as B
    from paper_2302_05662_gb300 import build as build_mod
    from paper_2302_05662_gb300 import matgen
    from paper_2302_05662_gb300.workload import SWEEP_VARIANTS

    torch.cuda.set_device(local)
    if rank == 0 or world == 1:
        build_mod.build()
    if world > 1:
        dist.barrier()
    B.load_library()
    vt = {"f64": B.SPMV_F64, "f32": B.SPMV_F32, "bf16": B.SPMV_BF16}[args.dtype]
    vdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[args.dtype]
    xdt = torch.float64 if vt == B.SPMV_F64 else torch.float32
    vsz = {"f64": 8, "f32": 4, "bf16": 2}[args.dtype]
    xsz = 8 if vt == B.SPMV_F64 else 4

    pairs = []           # (variant, matrix, handle, x, y, nnz, bytes, launches)
    skipped = []
    mats_host = []
    mats_info = {}
    names_all = [n for n in ("stencil27_128^3", "poisson16_2^20", "rmat_s20_ef16", "banded_2^20_w32",
                             "blockdiag4_2^20")]
    only = set(args.only.split(",")) if args.only else None
    kern_only = set(args.kernels.split(",")) if args.kernels else None
    for mname, coo in matgen.workload_matrices(args.scale, only=only):
        k = names_all.index(mname) if mname in names_all else len(mats_info)
        x_np = matgen.dense_vector(coo.n, 100 + k)
        mats_host.append((mname, coo, x_np))
        rows = torch.from_numpy(coo.rows).cuda()
        cols = torch.from_numpy(coo.cols).cuda()
        if vt == B.SPMV_BF16:
            bits = matgen.bf16_bits(matgen.round_to_bf16(coo.vals)).view(np.int16)
            vals = torch.from_numpy(bits).cuda().view(torch.bfloat16)
        else:
            vals = torch.from_numpy(coo.vals).cuda().to(vdt)
        x = torch.from_numpy(x_np).cuda().to(xdt)
        mats_info[mname] = {"m": coo.m, "n": coo.n, "nnz": coo.nnz}
        for vname, kw in SWEEP_VARIANTS:
            if kern_only is not None and vname not in kern_only:
                continue
            try:
                h = B.spmv_create(coo.m, coo.n, rows, cols, vals, B.make_config(**kw))
            except B.SpmvError as e:
                skipped.append({"matrix": mname, "kernel": vname, "why": str(e)[:160]})
                continue
            info = B.spmv_get_info(h)
            y = torch.zeros(coo.m, dtype=xdt, device="cuda")
            launches = 2 if (info.format == B.FMT_HYB and info.hyb_coo_nnz > 0) else 1
            pairs.append({"variant": vname, "matrix": mname, "h": h, "x": x, "y": y, "nnz": info.nnz,
                          "bytes": byte_model(coo.m, coo.n, info.nnz, vsz, xsz),
                          "format_bytes": info.format_bytes, "launches": launches})
        del rows, cols, vals
    torch.cuda.synchronize()
    order = {v: i for i, (v, _) in enumerate(SWEEP_VARIANTS)}
    pairs.sort(key=lambda p: (order[p["variant"]], list(mats_info).index(p["matrix"])))
    stream = torch.cuda.current_stream()
    sh = stream.cuda_stream

    def step(events=None):
        for i, p in enumerate(pairs):
            if events is not None:
                events[i][0].record(stream)
            B.spmv_run(p["h"], 1.0, p["x"], 0.0, p["y"], sh)
            if events is not None:
                events[i][1].record(stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()

    # --- device-timed region: inputs resident in HBM
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in pairs] for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0] or 0) \
        if os.environ.get("CUDA_VISIBLE_DEVICES", "").replace(",", "").isdigit() else local
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(gpu_index) as clk:
        t_start.record(stream)
        for s in range(args.steps):
            step(ev[s])
        t_end.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    elapsed_ms = t_start.elapsed_time(t_end)
    per_pair_ms = [statistics.mean(ev[s][i][0].elapsed_time(ev[s][i][1]) for s in range(args.steps))
                   for i in range(len(pairs))]
    if world > 1:
        t = torch.tensor([elapsed_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_ms = float(t.item())
    flops_step = sum(2 * p["nnz"] for p in pairs)
    value = flops_step * args.steps * world / (elapsed_ms * 1e-3) / 1e9

    # --- end to end through the C ABI: x from pinned host memory, y back
    xs_host = [p["x"].cpu().pin_memory() for p in pairs]
    ys_host = [torch.empty(p["y"].numel(), dtype=xdt).pin_memory() for p in pairs]
    h2d = sum(t.numel() * t.element_size() for t in xs_host)
    d2h = sum(t.numel() * t.element_size() for t in ys_host)

    def e2e_step():
        for i, p in enumerate(pairs):
            p["x"].copy_(xs_host[i], non_blocking=True)
            B.spmv_run(p["h"], 1.0, p["x"], 0.0, p["y"], sh)
            ys_host[i].copy_(p["y"], non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    if world > 1:
        t = torch.tensor([e2e_ms], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e_value = flops_step * args.e2e_steps * world / (e2e_ms * 1e-3) / 1e9

    # --- roofline of the dominant kernel (largest share of the step)
    peak, peak_kind = measured_peak()
    per_kernel = []
    for p, ms in zip(pairs, per_pair_ms):
        gbs = p["bytes"] / (ms * 1e-3) / 1e9
        per_kernel.append({"matrix": p["matrix"], "kernel": p["variant"], "us": round(ms * 1e3, 2),
                           "gflops": round(2 * p["nnz"] / (ms * 1e-3) / 1e9, 2), "gbs": round(gbs, 1),
                           "frac": round(gbs / peak, 4),
                           "format_gbs": round(p["format_bytes"] / (ms * 1e-3) / 1e9, 1)})
    dom = max(range(len(pairs)), key=lambda i: per_pair_ms[i])
    dp = pairs[dom]
    achieved = dp["bytes"] / (per_pair_ms[dom] * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": None,
                "kernel": f"{dp['variant']} on {dp['matrix']}",
                "algorithmic_bytes_per_launch": dp["bytes"], "peak_source": peak_kind}
    best = {}
    for pk in per_kernel:
        if pk["matrix"] not in best or pk["frac"] > best[pk["matrix"]]["frac"]:
            best[pk["matrix"]] = pk
    clocks = clk.summary()
    if rank != 0:
        return
    cpu = None if args.no_cpu_baseline else cpu_baseline(mats_host)
    cfg = workload_config(args)
    cfg["parallelism"] = f"replicas{world}" if world > 1 else "single"
    cfg["matrices"] = mats_info
    cfg["skipped"] = skipped
    line = {"metric": "SpMV GFLOP/s (format sweep, 5 matrices x 6 kernels)", "value": round(value, 2),
            "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(elapsed_ms / args.steps, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.dtype, "data": "synthetic", "config": cfg,
            "roofline": roofline, "cpu_baseline": cpu,
            "e2e": {"value": round(e2e_value, 2), "unit": "GFLOP/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "clocks": clocks, "gpu_launches": sum(p["launches"] for p in pairs) * args.steps,
            "best_per_matrix": {m: {"kernel": v["kernel"], "gflops": v["gflops"], "frac": v["frac"]}
                                for m, v in best.items()},
            "per_kernel": per_kernel}
    print(json.dumps(line), flush=True)
    for p in pairs:
        B.spmv_destroy(p["h"])


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
    ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
