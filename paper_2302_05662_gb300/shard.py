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

With halo=True a rank receives only the x entries its rows touch: the
window [lo, hi) spanned by its columns (for a banded or stencil matrix, its
own rows plus a band on either side), assembled by one all-to-all in which
every owner sends each rank the part of the window inside its own block.
The handle then indexes columns from lo, so the product reads the window.
A banded matrix of half-width w exchanges about 2 w entries per rank
instead of n.

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


def column_window(cols) -> tuple:
    """[lo, hi): the columns a rank's rows touch; (0, 1) with no entries
    (a one-entry window keeps the handle's x length positive)."""
    if len(cols) == 0:
        return 0, 1
    lo, hi = int(cols.min()), int(cols.max()) + 1
    return lo, hi


def halo_plan(windows, blk: int, rank: int):
    """The all-to-all of x windows, for this rank.  windows[q] = (lo_q, hi_q)
    for every rank q; rank q owns x[q blk : (q+1) blk].  Returns (send, recv):
    send[q] = (offset in this rank's block, count) of the entries rank q's
    window needs from it; recv[q] = entries of this rank's window that rank
    q owns.  Received in rank order, the parts are the window in order."""
    lo, hi = windows[rank]
    b0, b1 = rank * blk, (rank + 1) * blk
    recv, send = [], []
    for q, (lq, hq) in enumerate(windows):
        recv.append(max(0, min(hi, (q + 1) * blk) - max(lo, q * blk)))
        a, e = max(lq, b0), min(hq, b1)
        send.append((a - b0, e - a) if e > a else (0, 0))
    return send, recv


def all_windows(lo: int, hi: int, parts: int, device="cpu", group=None):
    """Every rank's column window, from one all-gather of two integers."""
    if parts == 1:
        return [(int(lo), int(hi))]
    import torch
    import torch.distributed as dist
    mine = torch.tensor([lo, hi], dtype=torch.int64, device=device)
    every = torch.zeros(2 * parts, dtype=torch.int64, device=device)
    dist.all_gather_into_tensor(every, mine, group=group)
    w = every.cpu().numpy().reshape(parts, 2)
    return [(int(a), int(b)) for a, b in w]


def send_index(send):
    """Positions in this rank's x block of the entries it sends, peers in
    rank order (the all-to-all's input)."""
    parts = [np.arange(o, o + c, dtype=np.int64) for o, c in send if c > 0]
    return np.concatenate(parts) if parts else np.zeros(0, np.int64)


def gather_window(x_local, send_idx, send_counts, recv_counts, out, group=None):
    """out <- this rank's window of x: one all-to-all in which each rank
    sends every peer the entries of its own block (x_local, blk entries)
    that the peer's window needs."""
    import torch.distributed as dist
    dist.all_to_all_single(out, x_local.index_select(0, send_idx), output_split_sizes=list(recv_counts),
                           input_split_sizes=list(send_counts), group=group)
    return out


class ShardedMatrix:
    """This rank's row block of a matrix as a handle, plus the buffers of
    the x exchange (the whole x, or with halo this rank's window of it).
    rows/cols/vals: this rank's triplets with global row and column indices
    (device tensors; rows inside [bounds[rank], bounds[rank+1]))."""

    def __init__(self, m: int, n: int, rows, cols, vals, bounds, rank: int, parts: int, cfg=None,
                 halo: bool = False, group=None, windows=None):
        import torch
        self.m, self.n = int(m), int(n)
        self.bounds = np.asarray(bounds, dtype=np.int64)
        self.rank, self.parts = int(rank), int(parts)
        self.r0, self.r1 = int(self.bounds[rank]), int(self.bounds[rank + 1])
        self.blk = x_block(self.n, self.parts)
        self.halo = bool(halo)
        vt = {torch.float64: B.SPMV_F64, torch.float32: B.SPMV_F32, torch.bfloat16: B.SPMV_BF16}[vals.dtype]
        self.vec_dtype = torch.float64 if vt == B.SPMV_F64 else torch.float32
        lr = (rows - self.r0).to(torch.int32).contiguous()
        if self.halo:
            # every rank's window: given by the caller (a plan made where all
            # the triplets are known), else one all-gather
            self.lo, self.hi = column_window(cols)
            if windows is not None:
                self.windows = [(int(a), int(b)) for a, b in windows]
                if len(self.windows) != self.parts or self.windows[self.rank] != (self.lo, self.hi):
                    raise ValueError("windows: one (lo, hi) per rank, this rank's equal to its columns' span")
            else:
                self.windows = all_windows(self.lo, self.hi, self.parts, vals.device, group)
            send, self.recv = halo_plan(self.windows, self.blk, self.rank)
            self.send_counts = [c for _, c in send]
            self.send_idx = torch.from_numpy(send_index(send)).to(vals.device)
            lc = (cols - self.lo).to(torch.int32).contiguous()
            self.h = B.spmv_create(self.r1 - self.r0, self.hi - self.lo, lr, lc, vals.contiguous(), cfg)
            self.x_win = torch.zeros(self.hi - self.lo, dtype=self.vec_dtype, device=vals.device)
        else:
            self.h = B.spmv_create(self.r1 - self.r0, self.n, lr, cols.contiguous(), vals.contiguous(), cfg)
            self.x_full = torch.zeros(self.parts * self.blk, dtype=self.vec_dtype, device=vals.device)

    def exchanged_entries(self) -> int:
        """x entries this rank receives from other ranks per product."""
        if self.halo:
            return int(sum(c for q, c in enumerate(self.recv) if q != self.rank))
        return int((self.parts - 1) * self.blk)

    def gather_halo(self, x_local, group=None):
        """The window x[lo:hi] from its owners (one all-to-all) into x_win."""
        if self.parts == 1:
            self.x_win.copy_(x_local[self.lo:self.hi])
            return self.x_win
        return gather_window(x_local, self.send_idx, self.send_counts, self.recv, self.x_win, group)

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
        """y_local <- alpha A[r0:r1, :] x + beta y_local, x (or, with halo,
        this rank's window of it) gathered first."""
        if self.halo:
            self.gather_halo(x_local, group)
            B.spmv_run(self.h, alpha, self.x_win, beta, y_local, stream)
            return
        self.gather_x(x_local, group)
        B.spmv_run(self.h, alpha, self.x_full, beta, y_local, stream)

    def destroy(self):
        if self.h:
            B.spmv_destroy(self.h)
            self.h = 0
