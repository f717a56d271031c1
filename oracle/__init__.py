"""CPU oracle for the SpMV engine -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library and its Python
binding never import, link or call anything here, and nothing here imports
them: the two sides share only the seeded input generators.

Contents (each function cites the part of the paper it follows):

* ``spmv_coo``      -- y = alpha*A*x + beta*y from COO triplets in fp64
                       (plain C, Kahan-compensated; Section 2.2).
* ``csr_from_coo``  -- the CSR arrays of Section 2.3 built by sorting.
* ``features``      -- the sparsity features of Table 2 (Section 5.5) plus
                       the extra structural features of the selector.
* ``hyb_ell_width`` -- the ELL width rule used for the HYB format.
* ``mlp_forward``   -- the selector's 2-layer MLP (Section 5.4 relies on
                       multi-class classification; this is its forward pass).
* ``time_head``, ``conversion_cost_us``, ``gate``
                    -- the run-time mode's decision (Section 5.3 steps 3-4):
                       predicted product times, predicted conversion cost,
                       and the convert-only-if-it-pays rule.
* ``cg``            -- conjugate gradients (Hestenes-Stiefel) with its
                       products from ``spmv_coo``: the iterative solver whose
                       repeated SpMV amortises selection and conversion
                       (Section 7.5).

Parity pins: every function here is checked in ``tests/test_oracle_*.py``
against closed forms, invariants, brute force or values printed in the paper.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_SRC = os.path.join(_HERE, "spmv_oracle.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle into oracle/_build/liboracle.so (gcc, fp64,
    no FP contraction so results are identical on x86-64 and aarch64)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            f = lib.oracle_spmv_coo_f64
            f.restype = ctypes.c_int
            f.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                          ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                          ctypes.c_double, ctypes.c_void_p, ctypes.c_double,
                          ctypes.c_void_p, ctypes.c_void_p]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data if a.size else 0


def spmv_coo(m: int, n: int, rows, cols, vals, x, alpha: float = 1.0,
             beta: float = 0.0, y=None) -> np.ndarray:
    """y_out = alpha * A x + beta * y, A given by COO triplets (Section 2.2).

    Duplicates are summed; beta == 0 ignores y.  All arithmetic in fp64.
    """
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    vals = np.ascontiguousarray(vals, dtype=np.float64)
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.shape[0] < n:
        raise ValueError("x shorter than n")
    out = np.empty(m, dtype=np.float64)
    yin = None
    if beta != 0.0:
        yin = np.ascontiguousarray(y, dtype=np.float64)
        if yin.shape[0] < m:
            raise ValueError("y shorter than m")
    rc = _load().oracle_spmv_coo_f64(
        m, n, rows.shape[0], _ptr(rows), _ptr(cols), _ptr(vals),
        float(alpha), _ptr(x), float(beta),
        _ptr(yin) if yin is not None else 0, _ptr(out) if m else 0)
    if rc == -1:
        raise ValueError("triplet index out of range")
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return out


def spmv_coo_obj(coo, x, alpha=1.0, beta=0.0, y=None, vals=None):
    """spmv_coo on a matgen.Coo (optionally with substituted values)."""
    return spmv_coo(coo.m, coo.n, coo.rows, coo.cols,
                    coo.vals if vals is None else vals, x, alpha, beta, y)


# ---------------------------------------------------------------------------
# CSR built by sorting (Section 2.3: Data, Column Index, Row Index arrays)
# ---------------------------------------------------------------------------

def csr_from_coo(m: int, n: int, rows, cols, vals):
    """Return (rowptr int64[m+1], colidx int32[nnz_u], vals f64[nnz_u]).

    Entries are ordered by (row, col); duplicate pairs are merged by summing
    their values sequentially in triplet order.
    """
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    order = np.lexsort((cols, rows))            # stable: keeps triplet order
    r, c, v = rows[order], cols[order], vals[order]
    if r.size:
        head = np.ones(r.size, dtype=bool)
        head[1:] = (r[1:] != r[:-1]) | (c[1:] != c[:-1])
        starts = np.flatnonzero(head)
        ends = np.append(starts[1:], r.size)
        uv = v[starts].copy()
        for k in np.flatnonzero(ends - starts > 1):
            s = 0.0
            for t in range(starts[k], ends[k]):
                s += v[t]
            uv[k] = s
        ur, uc = r[starts], c[starts]
    else:
        ur = np.zeros(0, np.int64)
        uc = np.zeros(0, np.int64)
        uv = np.zeros(0, np.float64)
    counts = np.bincount(ur, minlength=m) if m else np.zeros(0, np.int64)
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr, uc.astype(np.int32), uv


# ---------------------------------------------------------------------------
# Sparsity features (Table 2 of Section 5.5, plus the selector's extras)
# ---------------------------------------------------------------------------

FEATURE_NAMES = (
    "n_rows", "nnz", "density", "mean_row", "var_row", "std_row", "min_row",
    "max_row", "median_row", "mode_row", "ell_ratio", "gini", "cv_row",
    "empty_frac", "bandwidth", "mean_dist", "diag_frac", "fill_4x4",
    "fill_2x2", "hyb_tail_frac",
)


def hyb_ell_width(row_lengths, m: int) -> int:
    """ELL width of the HYB format: the largest k >= 1 such that at least
    max(4096, m/3) rows hold k or more nonzeros (Bell and Garland's rule,
    the HYB paper cited with COO/CSR/ELL in the introduction); 0 if none."""
    ell = np.asarray(row_lengths, dtype=np.int64)
    best = 0
    kmax = int(ell.max()) if ell.size else 0
    for k in range(1, kmax + 1):
        cnt = int((ell >= k).sum())
        if cnt >= 4096 and 3 * cnt >= m:
            best = k
        else:
            break
    return best


def features(m: int, n: int, rows, cols) -> dict:
    """Sparsity features of the matrix with the given (row, col) pattern.

    Duplicated pairs count once.  Definitions (Table 2; readings where the
    paper leaves a choice):
      n_rows = m (Table 2: "number of rows"); mean = nnz/m; variance is the
      population variance of the row lengths and std its square root (the
      printed Var_nnz equals Std_nnz squared); ELL_ratio = nnz/(m*max_len)
      (0 when max_len = 0); median = lower middle of the sorted row lengths;
      mode = most frequent row length, smallest on ties.
    Extra selector features: density nnz/(m*n); min row length; Gini
    coefficient sum_i (2i-m-1) l_(i) / (m * sum l) over ascending lengths;
    coefficient of variation std/mean; fraction of empty rows; bandwidth
    max|i-j|; mean |i-j|; fraction of diagonal entries; 4x4 and 2x2 block
    fill nnz/(r^2 * #nonempty r x r blocks); fraction of nonzeros beyond the
    HYB ELL width.  Ratios with a zero denominator are 0.
    """
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    if rows.size:
        key = np.unique(rows * max(n, 1) + cols)
        rows, cols = key // max(n, 1), key % max(n, 1)
    nnz = int(rows.size)
    ell = (np.bincount(rows, minlength=m).astype(np.int64) if m
           else np.zeros(0, np.int64))
    f = {}
    f["n_rows"] = float(m)
    f["nnz"] = float(nnz)
    f["density"] = nnz / (m * n) if m and n else 0.0
    mean = nnz / m if m else 0.0
    f["mean_row"] = mean
    # population variance, accumulated exactly in integers then divided
    if m:
        s2 = int((ell * ell).sum())
        var = (s2 * m - nnz * nnz) / (m * m)
    else:
        var = 0.0
    f["var_row"] = float(var)
    f["std_row"] = float(np.sqrt(var))
    f["min_row"] = float(ell.min()) if m else 0.0
    mx = int(ell.max()) if m else 0
    f["max_row"] = float(mx)
    srt = np.sort(ell)
    f["median_row"] = float(srt[(m - 1) // 2]) if m else 0.0
    if m:
        cnt = np.bincount(ell)
        f["mode_row"] = float(int(np.argmax(cnt)))   # argmax: first = smallest
    else:
        f["mode_row"] = 0.0
    f["ell_ratio"] = nnz / (m * mx) if m and mx else 0.0
    if m and nnz:
        i = np.arange(1, m + 1, dtype=np.int64)
        f["gini"] = float(int(((2 * i - m - 1) * srt).sum())) / (m * nnz)
    else:
        f["gini"] = 0.0
    f["cv_row"] = f["std_row"] / mean if mean else 0.0
    f["empty_frac"] = float((ell == 0).sum()) / m if m else 0.0
    d = np.abs(rows - cols)
    f["bandwidth"] = float(d.max()) if nnz else 0.0
    f["mean_dist"] = float(int(d.sum())) / nnz if nnz else 0.0
    f["diag_frac"] = float((d == 0).sum()) / nnz if nnz else 0.0
    for r, name in ((4, "fill_4x4"), (2, "fill_2x2")):
        if nnz:
            nb = (n + r - 1) // r
            blocks = np.unique((rows // r) * nb + cols // r).size
            f[name] = nnz / (r * r * blocks)
        else:
            f[name] = 0.0
    K = hyb_ell_width(ell, m)
    f["hyb_tail_frac"] = (float(int(np.maximum(ell - K, 0).sum())) / nnz
                          if nnz else 0.0)
    return f


def features_vector(m, n, rows, cols) -> np.ndarray:
    f = features(m, n, rows, cols)
    return np.array([f[k] for k in FEATURE_NAMES], dtype=np.float64)


# ---------------------------------------------------------------------------
# Selector MLP (multi-class classification, Section 5.4)
# ---------------------------------------------------------------------------

# Features that are counts or lengths enter the network as log1p(value).
LOG_FEATURES = ("n_rows", "nnz", "mean_row", "var_row", "std_row", "min_row",
                "max_row", "median_row", "mode_row", "bandwidth", "mean_dist")


def mlp_inputs(fvec: np.ndarray, mu: np.ndarray, sigma: np.ndarray) -> np.ndarray:
    """log1p on the count-like features, then z-score with training stats."""
    z = np.array(fvec, dtype=np.float64)
    for k, name in enumerate(FEATURE_NAMES):
        if name in LOG_FEATURES:
            z[k] = np.log1p(z[k])
    return (z - mu) / sigma


def mlp_forward(fvec, mu, sigma, W1, b1, W2, b2) -> np.ndarray:
    """Logits of the 20 -> H -> K ReLU network: W2 relu(W1 z + b1) + b2.

    W1 is H x 20 and W2 is K x H (row-major, output by input)."""
    z = mlp_inputs(fvec, mu, sigma)
    h = np.maximum(np.asarray(W1, np.float64) @ z + np.asarray(b1, np.float64), 0.0)
    return np.asarray(W2, np.float64) @ h + np.asarray(b2, np.float64)


# ---------------------------------------------------------------------------
# Run-time mode decision (Section 5.3, steps 3-4; overheads in Section 7.5)
# ---------------------------------------------------------------------------

def time_head(fvec, mu, sigma, W1, b1, W3, b3) -> np.ndarray:
    """Predicted natural log of microseconds per product: W3 relu(W1 z + b1)
    + b3 on the same hidden layer as ``mlp_forward``.

    One output per label class, then one for default CSR (the configuration
    a fresh matrix runs in).  This is the regression counterpart of the
    classifier that Section 5.3 uses to weigh the gain of a new format
    against the optimisation overhead.  W3 is (K+1) x H."""
    z = mlp_inputs(fvec, mu, sigma)
    h = np.maximum(np.asarray(W1, np.float64) @ z + np.asarray(b1, np.float64), 0.0)
    return np.asarray(W3, np.float64) @ h + np.asarray(b3, np.float64)


def conversion_cost_us(coef, nnz: int, m: int) -> float:
    """Predicted time of converting to one format (Section 5.3 step 3, the
    c_latency of Section 7.5): the linear model a + b*nnz + c*m in
    microseconds, clamped below at zero.  ``coef`` = (a, b, c)."""
    a, b, c = (float(v) for v in coef)
    return max(0.0, a + b * float(nnz) + c * float(m))


def gate(t_current_us: float, t_selected_us: float, select_us: float,
         pack_us: float, expected_runs: int) -> bool:
    """Section 5.3 step 4: convert only when the predicted benefit over the
    expected number of products is larger than the overhead.

    benefit  = (t_current - t_selected) * expected_runs
    overhead = select_us (feature extraction + prediction, f_latency +
               o_latency + p_latency of Section 7.5) + pack_us (c_latency)
    Returns True to convert; a tie keeps the current format."""
    benefit = (float(t_current_us) - float(t_selected_us)) * float(expected_runs)
    return benefit > float(select_us) + float(pack_us)


# ---------------------------------------------------------------------------
# Conjugate gradients: the repeated-SpMV setting of Section 7.5
# ---------------------------------------------------------------------------

def _dot(a: np.ndarray, b: np.ndarray) -> float:
    """Dot product: the fp64 products summed exactly (one final rounding)."""
    import math
    return math.fsum((np.asarray(a, np.float64) * np.asarray(b, np.float64)).tolist())


def cg(m: int, rows, cols, vals, b, x0=None, tol: float = 1e-8,
       maxit: int = 1000, record: bool = False) -> dict:
    """Conjugate gradients (Hestenes and Stiefel, 1952) for A x = b with A
    symmetric positive definite, given by COO triplets.

    Section 7.5 names the preconditioned conjugate gradient method as the
    iterative setting in which one matrix is multiplied many times, so the
    selection and conversion cost is paid once.  The method itself is the
    textbook one:

        r_0 = b - A x_0,  p_0 = r_0,  rho_0 = r_0.r_0
        while k < maxit and rho_k > tol^2 * (b.b):
            q = A p_k;  pq = p_k.q          (stop: breakdown if pq <= 0)
            alpha = rho_k / pq
            x_{k+1} = x_k + alpha p_k;  r_{k+1} = r_k - alpha q
            rho_{k+1} = r_{k+1}.r_{k+1};  beta = rho_{k+1} / rho_k
            p_{k+1} = r_{k+1} + beta p_k

    Products by ``spmv_coo``; dot products rounded once (``_dot``); each
    vector update is one multiply and one add per element, each rounded.
    Returns x, iterations (products A p), rho history (rho_0 .. rho_iters),
    converged, breakdown; with ``record`` also the lists of r_k and p_k.
    """
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(m) if x0 is None else np.array(x0, dtype=np.float64)
    r = spmv_coo(m, m, rows, cols, vals, x, -1.0, 1.0, b)
    p = r.copy()
    rho = _dot(r, r)
    stop = tol * tol * _dot(b, b)
    hist = [rho]
    rs, ps = ([r.copy()], [p.copy()]) if record else (None, None)
    k = 0
    breakdown = False
    while k < maxit and rho > stop:
        q = spmv_coo(m, m, rows, cols, vals, p)
        pq = _dot(p, q)
        if not pq > 0.0:
            breakdown = True
            break
        alpha = rho / pq
        x = x + alpha * p
        r = r - alpha * q
        rho_new = _dot(r, r)
        p = r + (rho_new / rho) * p
        rho = rho_new
        hist.append(rho)
        k += 1
        if record:
            rs.append(r.copy())
            ps.append(p.copy())
    out = {"x": x, "iterations": k, "rho": hist, "converged": rho <= stop,
           "breakdown": breakdown}
    if record:
        out["r"], out["p"] = rs, ps
    return out
