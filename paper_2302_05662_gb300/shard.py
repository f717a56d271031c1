"""Row-block sharding of one product y = alpha A x + beta y over ranks.

The paper runs every product on one GPU (Section 6.2).  A matrix too large
or too slow for one GPU shards naturally by rows: rank r owns the rows
[bounds[r], bounds[r+1]) -- contiguous, chosen so every rank holds about
nnz / ranks nonzeros -- as an ordinary handle whose column indices stay
global.  x is distributed in equal blocks of ceil(n / ranks) entries (rank r
owns x[r*blk : (r+1)*blk]), so one all-gather per product assembles the whole
x on every rank with no reordering; each rank then multiplies its rows and
writes its own block of y.  The all-gather is the only exchange step (NCCL
on GPUs; gloo in the CPU tests of the host logic).

Everything here is orchestration around the C ABI: the partition is
integer bookkeeping on row pointers, the gather is torch.distributed, and
the product is spmv_run.
"""
from __future__ import annotations

import numpy as np

from . import binding as B


def partition_rows(rowptr, parts: int) -> np.ndarray:
    """Contiguous, nnz-balanced row ranges: bounds[0] = 0 <= ... <= bounds[parts]
    = m.  The boundary before part r is the first row that starts at or
    after r * nnz / parts nonzeros, so each part holds nnz / parts nonzeros
    to within one row."""
    rowptr = np.asarray(rowptr, dtype=np.int64)
    if parts < 1:
        raise ValueError("parts must be >= 1")
    m = rowptr.size - 1
    nnz = int(rowptr[-1]) if m >= 0 else 0
    targets = (np.arange(1, parts, dtype=np.int64) * nnz + parts - 1) // parts
    inner = np.searchsorted(rowptr[:m], targets, side="left") if m > 0 else np.zeros(parts - 1, np.int64)
    return np.concatenate([[0], np.minimum(inner, m), [m]]).astype(np.int64)


def x_block(n: int, parts: int) -> int:
    """Entries of x each rank owns (the last block may be padded)."""
    return max(1, -(-n // parts))


def local_triplets(rows, cols, vals, r0: int, r1: int):
    """The triplets of rows [r0, r1), rows renumbered from 0 (host or device
    arrays; numpy or torch)."""
    keep = (rows >= r0) & (rows < r1)
    return rows[keep] - r0, cols[keep], vals[keep]


class ShardedMatrix:
    """This rank's row block of a matrix as a handle, plus the buffers of
    the x all-gather.  rows/cols/vals: this rank's triplets with global row
    and column indices (device tensors; rows inside [bounds[rank],
    bounds[rank+1]))."""

    def __init__(self, m: int, n: int, rows, cols, vals, bounds, rank: int, parts: int, cfg=None):
        import torch
        self.m, self.n = int(m), int(n)
        self.bounds = np.asarray(bounds, dtype=np.int64)
        self.rank, self.parts = int(rank), int(parts)
        self.r0, self.r1 = int(self.bounds[rank]), int(self.bounds[rank + 1])
        self.blk = x_block(self.n, self.parts)
        vt = {torch.float64: B.SPMV_F64, torch.float32: B.SPMV_F32, torch.bfloat16: B.SPMV_BF16}[vals.dtype]
        self.vec_dtype = torch.float64 if vt == B.SPMV_F64 else torch.float32
        lr = (rows - self.r0).to(torch.int32).contiguous()
        self.h = B.spmv_create(self.r1 - self.r0, self.n, lr, cols.contiguous(), vals.contiguous(), cfg)
        self.x_full = torch.zeros(self.parts * self.blk, dtype=self.vec_dtype, device=vals.device)

    def x_slice(self):
        """This rank's block of x inside the gathered buffer."""
        return self.x_full[self.rank * self.blk:(self.rank + 1) * self.blk]

    def gather_x(self, x_local, group=None):
        """All-gather the ranks' x blocks (each blk entries) into x_full."""
        import torch.distributed as dist
        if self.parts == 1:
            self.x_full[:x_local.numel()].copy_(x_local)
            return self.x_full
        dist.all_gather_into_tensor(self.x_full, x_local.contiguous(), group=group)
        return self.x_full

    def run(self, alpha: float, x_local, beta: float, y_local, group=None, stream=None):
        """y_local <- alpha A[r0:r1, :] x + beta y_local, x gathered first."""
        self.gather_x(x_local, group)
        B.spmv_run(self.h, alpha, self.x_full, beta, y_local, stream)

    def destroy(self):
        if self.h:
            B.spmv_destroy(self.h)
            self.h = 0
