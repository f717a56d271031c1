"""Seeded synthetic sparse-matrix generators (test and benchmark inputs only).

The paper evaluates on 30 SuiteSparse matrices (Section 6.1) that are not
available here; these generators produce seeded stand-ins with the shapes,
row-length distributions and structures of that kind of workload: PDE
stencils, random rows, power-law graphs (R-MAT), banded and block-diagonal
matrices.  Every generator returns COO triplets (the input format the paper
starts from, Section 7.5) sorted by (row, col) with no duplicates, plus the
matrix size.  Randomness comes from numpy's PCG64 generator seeded by the
caller.

This module holds no SpMV arithmetic: it only builds inputs.  Both the CPU
oracle and the CUDA path receive the very same arrays from here.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Coo", "laplacian_1d", "laplacian_2d", "stencil_3d", "banded",
    "block_diagonal", "poisson_rows", "rmat", "random_coo", "dense_vector",
    "round_to_f32", "round_to_bf16", "bf16_bits", "family_matrix",
    "FAMILIES", "workload_matrices",
]


@dataclass
class Coo:
    """COO triplets of an m x n sparse matrix (int32 indices, fp64 values)."""

    m: int
    n: int
    rows: np.ndarray
    cols: np.ndarray
    vals: np.ndarray
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.rows.shape[0])

    def __post_init__(self):
        self.rows = np.ascontiguousarray(self.rows, dtype=np.int32)
        self.cols = np.ascontiguousarray(self.cols, dtype=np.int32)
        self.vals = np.ascontiguousarray(self.vals, dtype=np.float64)


def _from_offsets(nrows: int, ncols: int, cols_2d: np.ndarray,
                  valid_2d: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Flatten a (rows x offsets) candidate table, keeping valid entries.

    Columns in each row of ``cols_2d`` must already be increasing, so the
    row-major flattening is sorted by (row, col).
    """
    rows_2d = np.broadcast_to(np.arange(nrows, dtype=np.int32)[:, None],
                              cols_2d.shape)
    rows = rows_2d[valid_2d]
    cols = cols_2d[valid_2d].astype(np.int32)
    return rows, cols


def laplacian_1d(N: int) -> Coo:
    """tridiag(-1, 2, -1) of size N (Dirichlet 1D Laplacian)."""
    i = np.arange(N, dtype=np.int64)
    offs = np.array([-1, 0, 1], dtype=np.int64)
    cols = i[:, None] + offs[None, :]
    valid = (cols >= 0) & (cols < N)
    rows, c = _from_offsets(N, N, cols, valid)
    vals = np.where(rows == c, 2.0, -1.0)
    return Coo(N, N, rows, c, vals, name=f"lap1d_{N}")


def laplacian_2d(N: int) -> Coo:
    """5-point Laplacian on an N x N grid, Dirichlet boundary, values 4 / -1.

    Unknown (a, b) of the grid has index a*N + b.
    """
    n = N * N
    i = np.arange(n, dtype=np.int64)
    a, b = i // N, i % N
    offs = np.array([-N, -1, 0, 1, N], dtype=np.int64)
    cols = i[:, None] + offs[None, :]
    valid = np.stack([a > 0, b > 0, np.ones(n, bool), b < N - 1, a < N - 1],
                     axis=1)
    rows, c = _from_offsets(n, n, cols, valid)
    vals = np.where(rows == c, 4.0, -1.0)
    return Coo(n, n, rows, c, vals, name=f"lap2d_{N}x{N}")


def stencil_3d(M: int, points: int = 27, rng: np.random.Generator | None = None,
               values: str = "normal") -> Coo:
    """3D stencil (7 or 27 points) on an M^3 grid, Dirichlet boundary.

    values="normal" draws N(0,1) per entry from ``rng``; values="laplace"
    gives the constant-coefficient operator (centre = points-1, others -1).
    """
    n = M * M * M
    if points == 27:
        d = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1)
             for dx in (-1, 0, 1)]
    elif points == 7:
        d = [(-1, 0, 0), (0, -1, 0), (0, 0, -1), (0, 0, 0), (0, 0, 1),
             (0, 1, 0), (1, 0, 0)]
    else:
        raise ValueError("points must be 7 or 27")
    rows_l, cols_l = [], []
    # process in z-slabs to bound temporary memory
    slab = max(1, (1 << 22) // (M * M))
    for z0 in range(0, M, slab):
        z1 = min(M, z0 + slab)
        idx = np.arange(z0 * M * M, z1 * M * M, dtype=np.int64)
        z, y, x = idx // (M * M), (idx // M) % M, idx % M
        cols = np.empty((idx.size, len(d)), dtype=np.int64)
        valid = np.empty((idx.size, len(d)), dtype=bool)
        for k, (dz, dy, dx) in enumerate(d):
            cols[:, k] = idx + dz * M * M + dy * M + dx
            valid[:, k] = ((z + dz >= 0) & (z + dz < M) & (y + dy >= 0)
                           & (y + dy < M) & (x + dx >= 0) & (x + dx < M))
        r = np.broadcast_to(idx[:, None], cols.shape)[valid]
        rows_l.append(r.astype(np.int32))
        cols_l.append(cols[valid].astype(np.int32))
    rows = np.concatenate(rows_l)
    cols = np.concatenate(cols_l)
    if values == "normal":
        rng = rng if rng is not None else np.random.default_rng(0)
        vals = rng.standard_normal(rows.size)
    else:
        vals = np.where(rows == cols, float(points - 1), -1.0)
    return Coo(n, n, rows, cols, vals, name=f"stencil{points}_{M}^3")


def banded(n: int, w: int, rng: np.random.Generator) -> Coo:
    """Banded matrix with half-width w (all |i-j| <= w stored), N(0,1)."""
    rows_l, cols_l = [], []
    offs = np.arange(-w, w + 1, dtype=np.int64)
    step = max(1, (1 << 22) // (2 * w + 1))
    for r0 in range(0, n, step):
        i = np.arange(r0, min(n, r0 + step), dtype=np.int64)
        cols = i[:, None] + offs[None, :]
        valid = (cols >= 0) & (cols < n)
        rows_l.append(np.broadcast_to(i[:, None], cols.shape)[valid]
                      .astype(np.int32))
        cols_l.append(cols[valid].astype(np.int32))
    rows = np.concatenate(rows_l)
    cols = np.concatenate(cols_l)
    vals = rng.standard_normal(rows.size)
    return Coo(n, n, rows, cols, vals, name=f"banded_{n}_w{w}")


def block_diagonal(n: int, r: int, rng: np.random.Generator) -> Coo:
    """Block-diagonal matrix of dense r x r blocks (n rows, n % r == 0)."""
    if n % r:
        raise ValueError("n must be a multiple of r")
    i = np.arange(n, dtype=np.int64)
    cols = (i // r * r)[:, None] + np.arange(r, dtype=np.int64)[None, :]
    rows = np.broadcast_to(i[:, None], cols.shape).reshape(-1).astype(np.int32)
    cols = cols.reshape(-1).astype(np.int32)
    vals = rng.standard_normal(rows.size)
    return Coo(n, n, rows, cols, vals, name=f"blockdiag_{n}_r{r}")


def _sort_unique_keys(key: np.ndarray) -> np.ndarray:
    """Sorted distinct values of an int64 key array (sort + neighbour test;
    much faster than np.unique on large arrays)."""
    key = np.sort(key)
    if key.size < 2:
        return key
    keep = np.empty(key.size, dtype=bool)
    keep[0] = True
    np.not_equal(key[1:], key[:-1], out=keep[1:])
    return key[keep]


def _sorted_unique_per_row(rows: np.ndarray, cols: np.ndarray, n: int,
                           rng: np.random.Generator) -> tuple[np.ndarray, np.ndarray]:
    """Sort (row, col) pairs, redrawing columns that collide within a row."""
    key = np.sort(rows.astype(np.int64) * n + cols.astype(np.int64))
    while True:
        dup = np.zeros(key.size, dtype=bool)
        if key.size > 1:
            np.equal(key[1:], key[:-1], out=dup[1:])
        k = int(dup.sum())
        if k == 0:
            return (key // n).astype(np.int32), (key % n).astype(np.int32)
        key[dup] = (key[dup] // n) * n + rng.integers(0, n, size=k)
        key.sort()


def poisson_rows(n: int, lam: float, rng: np.random.Generator,
                 m: int | None = None) -> Coo:
    """Random rows: row length ~ Poisson(lam) (clipped to n), distinct
    uniform columns, N(0,1) values."""
    m = n if m is None else m
    lens = np.minimum(rng.poisson(lam, size=m), n).astype(np.int64)
    rows = np.repeat(np.arange(m, dtype=np.int64), lens)
    cols = rng.integers(0, n, size=rows.size)
    rows, cols = _sorted_unique_per_row(rows, cols, n, rng)
    vals = rng.standard_normal(rows.size)
    return Coo(m, n, rows, cols, vals, name=f"poisson_{m}_l{lam:g}")


def rmat(scale: int, edge_factor: int, rng: np.random.Generator,
         a: float = 0.57, b: float = 0.19, c: float = 0.19) -> Coo:
    """R-MAT power-law matrix: 2^scale rows, edge_factor * 2^scale edges drawn
    by recursive quadrant choice with probabilities (a, b, c, 1-a-b-c);
    duplicate edges are removed, then N(0,1) values drawn per unique entry."""
    n = 1 << scale
    E = edge_factor * n
    r = np.zeros(E, dtype=np.uint32)
    cc = np.zeros(E, dtype=np.uint32)
    fa, fab, fabc = np.float32(a), np.float32(a + b), np.float32(a + b + c)
    for level in range(scale):
        u = rng.random(E, dtype=np.float32)
        shift = np.uint32(scale - 1 - level)
        row_bit = u >= fab                                  # quadrants c, d
        col_bit = ((u >= fa) & (u < fab)) | (u >= fabc)     # quadrants b, d
        r |= row_bit.view(np.uint8).astype(np.uint32) << shift
        cc |= col_bit.view(np.uint8).astype(np.uint32) << shift
    key = _sort_unique_keys((r.astype(np.int64) << scale) | cc.astype(np.int64))
    rows = (key >> scale).astype(np.int32)
    cols = (key & (n - 1)).astype(np.int32)
    vals = rng.standard_normal(rows.size)
    return Coo(n, n, rows, cols, vals, name=f"rmat_s{scale}_ef{edge_factor}",
               meta={"edges_drawn": E, "a": a, "b": b, "c": c})


def random_coo(m: int, n: int, nnz: int, rng: np.random.Generator,
               duplicates: bool = False, shuffle: bool = False,
               integer_values: int = 0) -> Coo:
    """Unstructured random triplets for property tests.

    duplicates=False gives distinct (row, col) pairs sorted by (row, col);
    duplicates=True keeps repeated pairs.  shuffle=True permutes the triplet
    order.  integer_values=k > 0 draws values from the integers in [-k, k].
    """
    if m == 0 or n == 0:
        nnz = 0
    rows = rng.integers(0, max(m, 1), size=nnz)
    cols = rng.integers(0, max(n, 1), size=nnz)
    if not duplicates and nnz:
        key = _sort_unique_keys(rows.astype(np.int64) * n + cols)
        rows, cols = key // n, key % n
    elif nnz:
        order = np.lexsort((cols, rows))
        rows, cols = rows[order], cols[order]
    cnt = rows.size
    if integer_values:
        vals = rng.integers(-integer_values, integer_values + 1,
                            size=cnt).astype(np.float64)
    else:
        vals = rng.standard_normal(cnt)
    if shuffle and cnt:
        p = rng.permutation(cnt)
        rows, cols, vals = rows[p], cols[p], vals[p]
    return Coo(m, n, rows, cols, vals, name=f"random_{m}x{n}_{cnt}")


def dense_vector(n: int, seed: int, integer_values: int = 0) -> np.ndarray:
    """x ~ U[-1, 1] (or integers in [-k, k]) from its own seed."""
    rng = np.random.default_rng(seed)
    if integer_values:
        return rng.integers(-integer_values, integer_values + 1,
                            size=n).astype(np.float64)
    return rng.uniform(-1.0, 1.0, size=n)


def round_to_f32(v: np.ndarray) -> np.ndarray:
    """fp64 -> fp32 round-to-nearest-even, returned as fp64."""
    return np.asarray(v, dtype=np.float64).astype(np.float32).astype(np.float64)


def round_to_bf16(v: np.ndarray) -> np.ndarray:
    """fp64 -> bfloat16 round-to-nearest-even (single rounding, 8 significant
    bits), returned as fp64.  Finite inputs within the bf16 normal range."""
    v = np.asarray(v, dtype=np.float64)
    f, e = np.frexp(v)                 # v = f * 2^e, 0.5 <= |f| < 1
    q = np.rint(np.ldexp(f, 8))        # 8 significant bits, ties to even
    return np.ldexp(q, e - 8)


def bf16_bits(v_rounded: np.ndarray) -> np.ndarray:
    """uint16 bit patterns of values already rounded by round_to_bf16."""
    f32 = np.asarray(v_rounded, dtype=np.float64).astype(np.float32)
    return (f32.view(np.uint32) >> 16).astype(np.uint16)


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

FAMILIES = ("stencil", "poisson", "rmat", "banded", "blockdiag")


def family_matrix(family: str, n_target: int, seed: int,
                  jitter: bool = False) -> Coo:
    """One matrix of a structure family with about n_target rows.

    n is snapped per family: stencil side = round(n^(1/3)) (27-point, or 7/27
    point and 2D 5-point when jitter=True), R-MAT scale = round(log2 n),
    block-diagonal a multiple of the block size.  jitter=True also draws the
    family parameters (Poisson mean in [2, 64], band half-width in [1, 64],
    R-MAT a in [.45, .65], block size in {2, 4, 8}).
    """
    rng = np.random.default_rng(seed)
    n_target = max(int(n_target), 8)
    if family == "stencil":
        kind = int(rng.integers(0, 3)) if jitter else 2
        if kind == 0:
            N = max(2, int(round(math.sqrt(n_target))))
            coo = laplacian_2d(N)
            coo.vals = rng.standard_normal(coo.nnz)
            return coo
        M = max(2, int(round(n_target ** (1.0 / 3.0))))
        return stencil_3d(M, 7 if kind == 1 else 27, rng)
    if family == "poisson":
        lam = float(rng.uniform(2, 64)) if jitter else 16.0
        return poisson_rows(n_target, lam, rng)
    if family == "rmat":
        scale = max(3, int(round(math.log2(n_target))))
        a = float(rng.uniform(0.45, 0.65)) if jitter else 0.57
        bc = (1.0 - a) / 2.0 * 0.95 if jitter else 0.19
        return rmat(scale, 16, rng, a=a, b=bc, c=bc)
    if family == "banded":
        w = int(rng.integers(1, 65)) if jitter else 32
        return banded(n_target, w, rng)
    if family == "blockdiag":
        r = int(rng.choice([2, 4, 8])) if jitter else 4
        n = max(r, n_target // r * r)
        return block_diagonal(n, r, rng)
    raise ValueError(f"unknown family {family!r}")


def workload_matrices(scale: str = "full", seed: int = 1, only=None):
    """The five structure families of the format-sweep workload.

    scale="full": 27-point stencil 128^3 (n = 2,097,152), Poisson(16) rows
    n = 2^20, R-MAT scale 20 edge factor 16, banded n = 2^20 half-width 32,
    block-diagonal 4x4 n = 2^20.  scale="small": the same structures at
    about 2^14 rows, for parity tests the oracle finishes in seconds.
    Yields (name, Coo) lazily so only one matrix is generated at a time;
    `only` (a name or a collection of names) restricts the set.
    """
    if scale == "full":
        specs = [("stencil27_128^3", lambda r: stencil_3d(128, 27, r)),
                 ("poisson16_2^20", lambda r: poisson_rows(1 << 20, 16.0, r)),
                 ("rmat_s20_ef16", lambda r: rmat(20, 16, r)),
                 ("banded_2^20_w32", lambda r: banded(1 << 20, 32, r)),
                 ("blockdiag4_2^20", lambda r: block_diagonal(1 << 20, 4, r))]
    elif scale == "small":
        specs = [("stencil27_24^3", lambda r: stencil_3d(24, 27, r)),
                 ("poisson16_2^14", lambda r: poisson_rows(1 << 14, 16.0, r)),
                 ("rmat_s14_ef16", lambda r: rmat(14, 16, r)),
                 ("banded_2^14_w32", lambda r: banded(1 << 14, 32, r)),
                 ("blockdiag4_2^14", lambda r: block_diagonal(1 << 14, 4, r))]
    else:
        raise ValueError(scale)
    if isinstance(only, str):
        only = {only}
    for k, (name, fn) in enumerate(specs):
        if only is not None and name not in only:
            continue
        coo = fn(np.random.default_rng(seed * 1000 + k))
        coo.name = name
        yield name, coo


def batched_workload(count: int = 512, seed: int = 7):
    """The batched workload: `count` matrices with n log-uniform in
    [10^3, 2*10^5] (one draw per matrix from `seed`), families cycling
    through FAMILIES, jittered parameters, matrix i from seed 5000 + i.
    Yields (i, Coo) lazily; the x of matrix i is dense_vector(n, 9000 + i)."""
    import math
    rng = np.random.default_rng(seed)
    for i in range(count):
        fam = FAMILIES[i % len(FAMILIES)]
        n = int(math.exp(rng.uniform(math.log(1e3), math.log(2e5))))
        coo = family_matrix(fam, n, seed=5000 + i, jitter=True)
        coo.name = f"batch{i}_{fam}"
        yield i, coo
