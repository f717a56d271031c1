"""Helpers shared by the GPU parity tests: move seeded inputs to the device,
run the C ABI, and compare with the fp64 oracle."""
from __future__ import annotations

import numpy as np

from paper_2302_05662_gb300 import binding as B
from paper_2302_05662_gb300 import matgen

# normwise relative error bounds stated for each value type
TOL = {B.SPMV_F64: 1e-13, B.SPMV_F32: 1e-5, B.SPMV_BF16: 1e-2}
VT_NAMES = {B.SPMV_F64: "f64", B.SPMV_F32: "f32", B.SPMV_BF16: "bf16"}


def torch_dtype(vt):
    import torch
    return {B.SPMV_F64: torch.float64, B.SPMV_F32: torch.float32, B.SPMV_BF16: torch.bfloat16}[vt]


def vec_dtype(vt):
    import torch
    return torch.float64 if vt == B.SPMV_F64 else torch.float32


def stored_values(vals: np.ndarray, vt) -> np.ndarray:
    """The values the device holds, as fp64."""
    if vt == B.SPMV_F64:
        return np.asarray(vals, np.float64)
    if vt == B.SPMV_F32:
        return matgen.round_to_f32(vals)
    return matgen.round_to_bf16(vals)


def stored_vector(v: np.ndarray, vt) -> np.ndarray:
    return np.asarray(v, np.float64) if vt == B.SPMV_F64 else matgen.round_to_f32(v)


def device_values(vals: np.ndarray, vt):
    import torch
    if vt == B.SPMV_F64:
        return torch.from_numpy(np.ascontiguousarray(vals, np.float64)).cuda()
    if vt == B.SPMV_F32:
        return torch.from_numpy(np.ascontiguousarray(vals, np.float32)).cuda()
    bits = matgen.bf16_bits(matgen.round_to_bf16(vals)).view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(bits)).cuda().view(torch.bfloat16)


def create(coo, vt, cfg=None, rows=None, cols=None, vals=None):
    import torch
    r = torch.from_numpy(np.ascontiguousarray(coo.rows if rows is None else rows, np.int32)).cuda()
    c = torch.from_numpy(np.ascontiguousarray(coo.cols if cols is None else cols, np.int32)).cuda()
    v = device_values(coo.vals if vals is None else vals, vt)
    return B.spmv_create(coo.m, coo.n, r, c, v, cfg)


def run(h, vt, x: np.ndarray, alpha=1.0, beta=0.0, y0: np.ndarray | None = None, m=None):
    import torch
    xt = torch.from_numpy(np.ascontiguousarray(x)).to(vec_dtype(vt)).cuda()
    if y0 is None:
        yt = torch.full((m,), float("nan"), dtype=vec_dtype(vt), device="cuda")
    else:
        yt = torch.from_numpy(np.ascontiguousarray(y0)).to(vec_dtype(vt)).cuda()
    B.spmv_run(h, alpha, xt, beta, yt)
    torch.cuda.synchronize()
    return yt.cpu().double().numpy()


def rel_err(got, want) -> float:
    nw = float(np.linalg.norm(want))
    d = float(np.linalg.norm(np.asarray(got) - np.asarray(want)))
    return d / nw if nw > 0 else d


def oracle_for(oracle, coo, vt, x, alpha=1.0, beta=0.0, y0=None):
    """Oracle on the inputs the device actually holds (rounded values and
    vectors for f32/bf16)."""
    return oracle.spmv_coo(coo.m, coo.n, coo.rows, coo.cols, stored_values(coo.vals, vt),
                           stored_vector(x, vt), alpha, beta,
                           None if y0 is None else stored_vector(y0, vt))
