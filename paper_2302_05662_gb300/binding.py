"""Thin Python binding of the C ABI in include/spmv.h (argument marshalling).

Every function here has the name of the C entry point it calls and only
converts arguments: torch tensors become device pointers, the current torch
CUDA stream becomes the stream argument, status codes become SpmvError.
All computation happens in libspmv_gb300.so; if the library is missing the
calls raise instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libspmv_gb300.so")

SPMV_OK = 0
SPMV_ERR_INVALID = -1
STATUS_NAMES = {0: "SPMV_OK", -1: "SPMV_ERR_INVALID", -2: "SPMV_ERR_OOM", -3: "SPMV_ERR_CUDA",
                -4: "SPMV_ERR_UNSUPPORTED", -5: "SPMV_ERR_BOUNDS", -6: "SPMV_ERR_TIMEOUT"}
SPMV_F64, SPMV_F32, SPMV_BF16 = 0, 1, 2
FMT_CSR, FMT_ELL, FMT_COO, FMT_HYB, FMT_BSR, FMT_SELL = 0, 1, 2, 3, 4, 5
FORMAT_NAMES = {FMT_CSR: "csr", FMT_ELL: "ell", FMT_COO: "coo", FMT_HYB: "hyb", FMT_BSR: "bsr", FMT_SELL: "sell"}
TPR_SPLIT = -1
(ARR_CSR_ROWPTR, ARR_CSR_COLIDX, ARR_CSR_VALS, ARR_ELL_COLIDX, ARR_ELL_VALS, ARR_COO_ROWS,
 ARR_COO_COLS, ARR_COO_VALS, ARR_BSR_ROWPTR, ARR_BSR_COLIDX, ARR_BSR_VALS, ARR_ELL_PITCH,
 ARR_SELL_PTR, ARR_SELL_COLIDX, ARR_SELL_VALS, ARR_SELL_PERM) = range(16)

# every entry point include/spmv.h declares (checked by the CPU test suite)
EXPORTED = ("spmv_config_default", "spmv_create", "spmv_set_config", "spmv_get_config",
            "spmv_get_info", "spmv_run", "spmv_export_bytes", "spmv_export", "spmv_destroy",
            "spmv_last_error", "spmv_coo_run_noalloc", "spmv_features", "spmv_selector_load", "spmv_selector_load_vt",
            "spmv_selector_infer", "spmv_select", "spmv_batch_create", "spmv_batch_tune",
            "spmv_batch_launch", "spmv_batch_get_plan", "spmv_batch_destroy", "spmv_batch_run",
            "spmv_select_runtime", "spmv_cg", "spmv_set_panel_limit", "spmv_get_panel_limit",
            "spmv_probe_gather_floor", "spmv_probe_fp64_fma", "spmv_check")


class SpmvError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class spmv_config(ctypes.Structure):
    _fields_ = [("format", ctypes.c_int32), ("threads_per_block", ctypes.c_int32),
                ("threads_per_row", ctypes.c_int32), ("unroll", ctypes.c_int32),
                ("regcap", ctypes.c_int32), ("carveout", ctypes.c_int32),
                ("bsr_block", ctypes.c_int32), ("hyb_ell_width", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class spmv_runtime_decision(ctypes.Structure):
    _fields_ = [("convert", ctypes.c_int32), ("current_class", ctypes.c_int32),
                ("selected_class", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("predicted_us_current", ctypes.c_double), ("predicted_us_selected", ctypes.c_double),
                ("predicted_pack_us", ctypes.c_double), ("measured_select_us", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class spmv_cg_result(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("breakdown", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("rho0", ctypes.c_double), ("rho", ctypes.c_double), ("bb", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


CG_MAX_ITERATIONS = 16777216


class spmv_info(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("max_row", ctypes.c_int64), ("ell_width", ctypes.c_int64),
                ("hyb_coo_nnz", ctypes.c_int64), ("bsr_blocks", ctypes.c_int64), ("sell_slots", ctypes.c_int64),
                ("format_bytes", ctypes.c_int64), ("value_type", ctypes.c_int32),
                ("format", ctypes.c_int32), ("panels", ctypes.c_int32), ("reserved", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None
_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_I32 = ctypes.c_int32
_D = ctypes.c_double


def load_library(path: str | None = None):
    """Load libspmv_gb300.so (built by build.py); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise FileNotFoundError(
            f"{path} is missing: build it with paper_2302_05662_gb300.build.build()")
    lib = ctypes.CDLL(path)
    sig = {
        "spmv_config_default": (None, [ctypes.POINTER(spmv_config), _I32]),
        "spmv_create": (ctypes.c_int, [ctypes.POINTER(_VP), _I64, _I64, _I64, _VP, _VP, _VP, _I32,
                                       ctypes.POINTER(spmv_config), _VP]),
        "spmv_set_config": (ctypes.c_int, [_VP, ctypes.POINTER(spmv_config), _VP]),
        "spmv_get_config": (ctypes.c_int, [_VP, ctypes.POINTER(spmv_config)]),
        "spmv_get_info": (ctypes.c_int, [_VP, ctypes.POINTER(spmv_info)]),
        "spmv_run": (ctypes.c_int, [_VP, _D, _VP, _D, _VP, _VP]),
        "spmv_export_bytes": (ctypes.c_int, [_VP, _I32, ctypes.POINTER(_I64)]),
        "spmv_export": (ctypes.c_int, [_VP, _I32, _VP, _I64, _VP]),
        "spmv_destroy": (ctypes.c_int, [_VP]),
        "spmv_batch_create": (ctypes.c_int, [ctypes.POINTER(_VP), _VP, _I32, _VP, _VP, _VP, _VP, _VP]),
        "spmv_batch_tune": (ctypes.c_int, [_VP, _VP]),
        "spmv_batch_launch": (ctypes.c_int, [_VP, _VP]),
        "spmv_batch_get_plan": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
        "spmv_batch_destroy": (ctypes.c_int, [_VP]),
        "spmv_batch_run": (ctypes.c_int, [_VP, _I32, _VP, _VP, _VP, _VP, _VP]),
        "spmv_features": (ctypes.c_int, [_VP, _VP, _VP]),
        "spmv_selector_load": (ctypes.c_int, [_VP, _I64]),
        "spmv_selector_load_vt": (ctypes.c_int, [ctypes.c_int32, _VP, _I64]),
        "spmv_selector_infer": (ctypes.c_int, [_VP, _VP, ctypes.POINTER(_I32), _VP]),
        "spmv_select": (ctypes.c_int, [_VP, ctypes.POINTER(spmv_config), _VP, _VP]),
        "spmv_select_runtime": (ctypes.c_int, [_VP, _I64, ctypes.POINTER(spmv_config),
                                               ctypes.POINTER(spmv_runtime_decision), _VP]),
        "spmv_coo_run_noalloc": (ctypes.c_int, [_I64, _I64, _I64, _VP, _VP, _VP, _I32, _D, _VP, _D, _VP,
                                                _VP]),
        "spmv_cg": (ctypes.c_int, [_VP, _VP, _VP, _D, _I32, _VP, ctypes.POINTER(spmv_cg_result), _VP]),
        "spmv_set_panel_limit": (ctypes.c_int, [_I64]),
        "spmv_get_panel_limit": (_I64, []),
        "spmv_probe_gather_floor": (ctypes.c_int, [_VP, _VP, _VP, _VP]),
        "spmv_check": (ctypes.c_int, [_VP, _VP]),
        "spmv_probe_fp64_fma": (ctypes.c_int, [_I64, _VP, ctypes.POINTER(_I64), _VP]),
        "spmv_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int):
    if status != SPMV_OK:
        raise SpmvError(status, spmv_last_error())


def _stream(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _ptr(t):
    """Device address of a dense CUDA tensor (None gives NULL).  Host tensors
    and strided views are refused before the call: the library reads every
    buffer as a dense device array."""
    if t is None:
        return None
    if not getattr(t, "is_cuda", False):
        raise SpmvError(SPMV_ERR_INVALID, "expected a CUDA tensor (a device buffer)")
    if not t.is_contiguous():
        raise SpmvError(SPMV_ERR_INVALID, "expected a contiguous tensor")
    return t.data_ptr()


def _vec(t, need: int, vt: int, what: str):
    """Device address of a vector the library reads or writes `need` entries
    of, in the vector type of value type vt (fp64 for fp64 values, else
    fp32)."""
    if t is None:
        if need > 0:
            raise SpmvError(SPMV_ERR_INVALID, f"{what}: NULL where {need} entries are needed")
        return None
    import torch
    want = torch.float64 if vt == SPMV_F64 else torch.float32
    if t.dtype != want:
        raise SpmvError(SPMV_ERR_INVALID, f"{what}: dtype {t.dtype}, the matrix's vectors are {want}")
    if t.numel() < need:
        raise SpmvError(SPMV_ERR_INVALID, f"{what}: {t.numel()} entries, {need} needed")
    return _ptr(t)


def _triplets(rows, cols, vals):
    """(nnz, value type, pointers) of device COO triplets: int32 rows and
    columns and fp64/fp32/bf16 values of one length."""
    import torch
    if rows is None or cols is None or vals is None:
        if any(t is not None and t.numel() > 0 for t in (rows, cols, vals)):
            raise SpmvError(SPMV_ERR_INVALID, "triplets: rows, cols and vals must all be given")
        return 0, SPMV_F64, None, None, None
    if rows.dtype != torch.int32 or cols.dtype != torch.int32:
        raise SpmvError(SPMV_ERR_INVALID, "triplets: rows and cols must be int32")
    if vals.dtype not in (torch.float64, torch.float32, torch.bfloat16):
        raise SpmvError(SPMV_ERR_INVALID, f"triplets: value dtype {vals.dtype} is not fp64, fp32 or bf16")
    nnz = int(rows.numel())
    if cols.numel() != nnz or vals.numel() != nnz:
        raise SpmvError(SPMV_ERR_INVALID, "triplets: rows, cols and vals differ in length")
    return nnz, value_type_of(vals.dtype), _ptr(rows), _ptr(cols), _ptr(vals)


def value_type_of(dtype) -> int:
    import torch
    return {torch.float64: SPMV_F64, torch.float32: SPMV_F32, torch.bfloat16: SPMV_BF16}[dtype]


def make_config(format=FMT_CSR, **kw) -> spmv_config:
    """spmv_config with library defaults, then overridden by keyword fields."""
    cfg = spmv_config()
    load_library().spmv_config_default(ctypes.byref(cfg), int(format))
    for k, v in kw.items():
        setattr(cfg, k, int(v))
    return cfg


def spmv_last_error() -> str:
    return load_library().spmv_last_error().decode(errors="replace")


def spmv_create(m: int, n: int, rows, cols, vals, cfg: spmv_config | None = None, stream=None) -> int:
    """Handle from device COO triplets (int32 rows/cols, f64/f32/bf16 vals)."""
    lib = load_library()
    h = _VP()
    nnz, vt, rp, cp, vp = _triplets(rows, cols, vals)
    _check(lib.spmv_create(ctypes.byref(h), int(m), int(n), nnz, rp, cp, vp, vt,
                           ctypes.byref(cfg) if cfg is not None else None, _stream(stream)))
    _shapes[h.value] = (int(m), int(n), vt)
    return h.value


def spmv_set_config(h: int, cfg: spmv_config, stream=None):
    _check(load_library().spmv_set_config(h, ctypes.byref(cfg), _stream(stream)))


def spmv_get_config(h: int) -> spmv_config:
    cfg = spmv_config()
    _check(load_library().spmv_get_config(h, ctypes.byref(cfg)))
    return cfg


def spmv_get_info(h: int) -> spmv_info:
    info = spmv_info()
    _check(load_library().spmv_get_info(h, ctypes.byref(info)))
    return info


# (m, n, value type) of the handles this process created: the vector checks
# of spmv_run and friends then cost a dictionary lookup, not a library call
_shapes: dict = {}


def _shape(h: int):
    s = _shapes.get(h)
    if s is None:
        info = spmv_get_info(h)
        s = _shapes[h] = (int(info.m), int(info.n), int(info.value_type))
    return s


def spmv_run(h: int, alpha: float, x, beta: float, y, stream=None):
    """y <- alpha*A*x + beta*y on the device (x, y: torch CUDA tensors of
    the matrix's vector type, at least n and m entries)."""
    if h:
        m, n, vt = _shape(h)
        xp, yp = _vec(x, n, vt, "x"), _vec(y, m, vt, "y")
    else:
        xp, yp = _ptr(x), _ptr(y)
    _check(load_library().spmv_run(h, float(alpha), xp, float(beta), yp, _stream(stream)))


def spmv_export_bytes(h: int, array_id: int) -> int:
    b = _I64()
    _check(load_library().spmv_export_bytes(h, int(array_id), ctypes.byref(b)))
    return b.value


def spmv_export(h: int, array_id: int, out, stream=None):
    """Copy an internal array into the device tensor `out` (exact size)."""
    nbytes = out.numel() * out.element_size()
    _check(load_library().spmv_export(h, int(array_id), _ptr(out), nbytes, _stream(stream)))


NUM_FEATURES = 20


def spmv_features(h: int, stream=None):
    """The 20 sparsity features of the handle's matrix (numpy float64)."""
    import numpy as np
    out = np.zeros(NUM_FEATURES, dtype=np.float64)
    _check(load_library().spmv_features(h, out.ctypes.data, _stream(stream)))
    return out


def spmv_selector_load(blob):
    """Load a selector blob (sequence of float32) on the current device."""
    import numpy as np
    b = np.ascontiguousarray(blob, dtype=np.float32)
    _check(load_library().spmv_selector_load(b.ctypes.data, int(b.size)))


def spmv_selector_unload():
    """Unload the selector on the current device (spmv_selector_load(NULL, 0))."""
    _check(load_library().spmv_selector_load(None, 0))


def spmv_selector_load_vt(value_type: int, blob=None):
    """Load (or, with blob None, unload) the selector used for handles of
    one value type on the current device."""
    import numpy as np
    if blob is None:
        _check(load_library().spmv_selector_load_vt(int(value_type), None, 0))
        return
    b = np.ascontiguousarray(blob, dtype=np.float32)
    _check(load_library().spmv_selector_load_vt(int(value_type), b.ctypes.data, int(b.size)))


def spmv_selector_infer(features, k: int, stream=None):
    """(choice, logits[k]) of the loaded selector for host features."""
    import numpy as np
    f = np.ascontiguousarray(features, dtype=np.float64)
    logits = np.zeros(k, dtype=np.float32)
    c = _I32()
    _check(load_library().spmv_selector_infer(f.ctypes.data, logits.ctypes.data, ctypes.byref(c),
                                              _stream(stream)))
    return c.value, logits


def spmv_select(h: int, stream=None):
    """(chosen spmv_config, features) for the handle's matrix."""
    import numpy as np
    cfg = spmv_config()
    f = np.zeros(NUM_FEATURES, dtype=np.float64)
    _check(load_library().spmv_select(h, ctypes.byref(cfg), f.ctypes.data, _stream(stream)))
    return cfg, f


def _batch_arrays(handles, alphas, xs, betas, ys):
    import numpy as np
    n = len(handles)
    hs = (_VP * n)(*handles)
    al = np.ascontiguousarray(alphas, dtype=np.float64)
    be = np.ascontiguousarray(betas, dtype=np.float64)
    if len(xs) != n or len(ys) != n or al.size != n or be.size != n:
        raise SpmvError(SPMV_ERR_INVALID, "batch: handles, alphas, xs, betas and ys differ in length")
    px, py = [], []
    for i, h in enumerate(handles):
        if h:
            m, n_, vt = _shape(h)
            px.append(_vec(xs[i], n_, vt, f"xs[{i}]"))
            py.append(_vec(ys[i], m, vt, f"ys[{i}]"))
        else:
            px.append(_ptr(xs[i]))
            py.append(_ptr(ys[i]))
    xp = (_VP * n)(*px)
    yp = (_VP * n)(*py)
    return n, hs, al, be, xp, yp


def spmv_batch_create(handles, alphas, xs, betas, ys, stream=None) -> int:
    """Batch plan over handles with device vectors xs, ys (torch tensors)."""
    n, hs, al, be, xp, yp = _batch_arrays(handles, alphas, xs, betas, ys)
    b = _VP()
    _check(load_library().spmv_batch_create(ctypes.byref(b), hs, n, al.ctypes.data, xp, be.ctypes.data, yp,
                                            _stream(stream)))
    return b.value


def spmv_batch_tune(b: int, stream=None):
    _check(load_library().spmv_batch_tune(b, _stream(stream)))


def spmv_batch_launch(b: int, stream=None):
    _check(load_library().spmv_batch_launch(b, _stream(stream)))


def spmv_batch_get_plan(b: int, count: int):
    import numpy as np
    modes = np.zeros(count, dtype=np.int32)
    it, tpb = _I32(), _I32()
    _check(load_library().spmv_batch_get_plan(b, modes.ctypes.data, ctypes.byref(it), ctypes.byref(tpb)))
    return modes, it.value, tpb.value


def spmv_batch_destroy(b: int):
    if b:
        _check(load_library().spmv_batch_destroy(b))


def spmv_batch_run(handles, alphas, xs, betas, ys, stream=None):
    n, hs, al, be, xp, yp = _batch_arrays(handles, alphas, xs, betas, ys)
    _check(load_library().spmv_batch_run(hs, n, al.ctypes.data, xp, be.ctypes.data, yp, _stream(stream)))


def spmv_select_runtime(h: int, expected_runs: int, stream=None):
    """(chosen spmv_config, spmv_runtime_decision) for the handle's matrix."""
    cfg = spmv_config()
    dec = spmv_runtime_decision()
    _check(load_library().spmv_select_runtime(h, int(expected_runs), ctypes.byref(cfg), ctypes.byref(dec),
                                              _stream(stream)))
    return cfg, dec


def spmv_cg(h: int, b, x, tol: float, maxit: int, rho=None, stream=None) -> spmv_cg_result:
    """Conjugate gradients on the handle's matrix: x (device tensor) holds x_0
    on entry and the last iterate on return; rho (optional float64 device
    tensor of maxit + 1 entries) receives r_k.r_k per iteration."""
    out = spmv_cg_result()
    if h:
        m, n, vt = _shape(h)
        bp, xp = _vec(b, m, vt, "b"), _vec(x, n, vt, "x")
    else:
        bp, xp = _ptr(b), _ptr(x)
    rp = None
    if rho is not None:
        rp = _vec(rho, max(0, int(maxit)) + 1, SPMV_F64, "rho")
    _check(load_library().spmv_cg(h, bp, xp, float(tol), int(maxit), rp, ctypes.byref(out),
                                  _stream(stream)))
    return out


def spmv_set_panel_limit(max_triplets: int):
    """Triplet count above which spmv_create holds a matrix in row panels."""
    _check(load_library().spmv_set_panel_limit(int(max_triplets)))


def spmv_get_panel_limit() -> int:
    return int(load_library().spmv_get_panel_limit())


PANEL_LIMIT_DEFAULT = (1 << 31) - (1 << 20)
NOALLOC_MAX_NNZ = 1 << 25


def spmv_coo_run_noalloc(m: int, n: int, rows, cols, vals, alpha: float, x, beta: float, y, stream=None):
    """y <- alpha*A*x + beta*y from row-sorted device COO triplets, with no
    device allocation (the library's fixed scratch array is used)."""
    nnz, vt, rp, cp, vp = _triplets(rows, cols, vals)
    _check(load_library().spmv_coo_run_noalloc(int(m), int(n), nnz, rp, cp, vp, vt, float(alpha),
                                               _vec(x, int(n), vt, "x"), float(beta),
                                               _vec(y, int(m), vt, "y"), _stream(stream)))


def spmv_check(h: int, stream=None):
    """Raise SpmvError if a product since the last check recorded a device
    error (a copy wait that timed out, a skipped out-of-range index)."""
    _check(load_library().spmv_check(h, _stream(stream)))


def spmv_probe_gather_floor(h: int, x, y, stream=None):
    """Measurement kernel (include/spmv_probe.h): the handle's bytes moved
    with ideal access and its x gathers, no floating-point arithmetic; y
    receives meaningless bits."""
    m, n, vt = _shape(h)
    _check(load_library().spmv_probe_gather_floor(h, _vec(x, n, vt, "x"), _vec(y, m, vt, "y"),
                                                  _stream(stream)))


def spmv_probe_fp64_fma(iterations: int, sink, stream=None) -> int:
    """Measurement kernel: a full wave of independent fp64 FMA chains.
    Returns the number of fused multiply-adds launched (2 flops each)."""
    import torch
    if sink.dtype != torch.float64 or sink.numel() < 1:
        raise SpmvError(SPMV_ERR_INVALID, "sink: one float64 entry needed")
    count = _I64(0)
    _check(load_library().spmv_probe_fp64_fma(int(iterations), _ptr(sink), ctypes.byref(count),
                                              _stream(stream)))
    return int(count.value)


def spmv_destroy(h: int):
    if h:
        _shapes.pop(h, None)
        _check(load_library().spmv_destroy(h))
