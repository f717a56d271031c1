"""Host logic of the row-block sharded product on CPU: the nnz-balanced row
partition, the renumbering of each rank's triplets, and the all-gather of
x over a real 2-rank gloo process group.  The products themselves run on
the GPU (tests/test_gpu_shard.py); here the oracle multiplies each rank's
block, so the plan is checked against the unsharded product."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2302_05662_gb300 import matgen, shard


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rowptr(coo):
    rp = np.zeros(coo.m + 1, np.int64)
    np.cumsum(np.bincount(coo.rows, minlength=coo.m), out=rp[1:])
    return rp


@pytest.mark.parametrize("parts", [1, 2, 3, 8, 64])
@pytest.mark.parametrize("case", ["stencil", "rmat", "empty_tail", "one_row"])
def test_partition_covers_rows_and_balances_nnz(case, parts):
    rng = np.random.default_rng(3)
    coo = {"stencil": lambda: matgen.stencil_3d(12, 27, rng),
           "rmat": lambda: matgen.rmat(11, 16, rng),
           "empty_tail": lambda: matgen.random_coo(4000, 300, 900, rng),
           "one_row": lambda: matgen.Coo(5, 50, np.full(40, 2, np.int32), np.arange(40, dtype=np.int32),
                                         np.ones(40))}[case]()
    rp = _rowptr(coo)
    b = shard.partition_rows(rp, parts)
    assert b.size == parts + 1 and b[0] == 0 and b[-1] == coo.m
    assert np.all(np.diff(b) >= 0)
    per = rp[b[1:]] - rp[b[:-1]]
    assert per.sum() == coo.nnz
    max_row = int(np.diff(rp).max())
    assert np.all(np.abs(per - coo.nnz / parts) <= max_row + 1)


def test_local_triplets_renumber_rows():
    coo = matgen.poisson_rows(500, 6.0, np.random.default_rng(4))
    r, c, v = shard.local_triplets(coo.rows, coo.cols, coo.vals, 100, 250)
    assert r.min() >= 0 and r.max() < 150
    assert np.array_equal(np.sort(r + 100), np.sort(coo.rows[(coo.rows >= 100) & (coo.rows < 250)]))


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        coo = matgen.banded(3001, 7, np.random.default_rng(5))
        x = matgen.dense_vector(coo.n, 6)
        rp = _rowptr(coo)
        b = shard.partition_rows(rp, world)
        blk = shard.x_block(coo.n, world)
        xl = np.zeros(blk)
        part = x[rank * blk:(rank + 1) * blk]
        xl[:part.size] = part
        full = torch.zeros(world * blk, dtype=torch.float64)
        dist.all_gather_into_tensor(full, torch.from_numpy(xl))
        xg = full.numpy()[:coo.n]
        r0, r1 = int(b[rank]), int(b[rank + 1])
        lr, lc, lv = shard.local_triplets(coo.rows, coo.cols, coo.vals, r0, r1)
        y = oracle.spmv_coo(r1 - r0, coo.n, lr, lc, lv, xg)
        out[rank] = (r0, r1, np.array_equal(xg, x), y.tolist())
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_rank_gloo_gather_and_blocks_reassemble_the_product(oracle):
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    coo = matgen.banded(3001, 7, np.random.default_rng(5))
    want = oracle.spmv_coo(coo.m, coo.n, coo.rows, coo.cols, coo.vals, matgen.dense_vector(coo.n, 6))
    (a0, a1, g0, y0), (b0, b1, g1, y1) = out[0], out[1]
    assert g0 and g1                      # every rank gathered the whole x
    assert a0 == 0 and a1 == b0 and b1 == coo.m
    assert np.array_equal(np.concatenate([y0, y1]), want)


# ------------------------------------------------------------ halo exchange
def _halo_cases():
    rng = np.random.default_rng(9)
    return {"banded": matgen.banded(5003, 9, rng),
            "stencil": matgen.stencil_3d(14, 27, rng),
            "random": matgen.random_coo(3000, 2500, 20000, rng),
            "empty_block": matgen.Coo(4000, 4000, np.concatenate([np.arange(100), np.arange(3900, 4000)]).astype(np.int32),
                                      np.concatenate([np.arange(100), np.arange(3900, 4000)]).astype(np.int32),
                                      np.ones(200))}


@pytest.mark.parametrize("parts", [1, 2, 3, 7])
@pytest.mark.parametrize("case", ["banded", "stencil", "random", "empty_block"])
def test_halo_plan_moves_each_window_entry_once(case, parts):
    """Every rank's window is covered exactly by what its owners send it:
    receive counts match the peers' send counts, the sent slices lie in the
    sender's block and, laid end to end in rank order, the received parts
    are the window's entries in order."""
    coo = _halo_cases()[case]
    b = shard.partition_rows(_rowptr(coo), parts)
    blk = shard.x_block(coo.n, parts)
    wins = [shard.column_window(shard.local_triplets(coo.rows, coo.cols, coo.vals, int(b[r]), int(b[r + 1]))[1])
            for r in range(parts)]
    plans = [shard.halo_plan(wins, blk, r) for r in range(parts)]
    for r, (lo, hi) in enumerate(wins):
        assert 0 <= lo < hi <= max(coo.n, 1)
        got = []
        for q in range(parts):
            off, cnt = plans[q][0][r]                  # what q sends to r
            assert cnt == plans[r][1][q]               # what r expects from q
            assert 0 <= off and off + cnt <= blk
            got.extend(range(q * blk + off, q * blk + off + cnt))
        assert got == list(range(lo, hi))
    if case == "banded" and parts > 1:
        # a half-width-9 band: each rank receives at most 2 x 9 entries from others
        for r in range(parts):
            assert sum(c for q, c in enumerate(plans[r][1]) if q != r) <= 18


def _halo_worker(rank, world, port, case, out):
    import torch
    import torch.distributed as dist
    import oracle
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        coo = _halo_cases()[case]
        x = matgen.dense_vector(coo.n, 12)
        b = shard.partition_rows(_rowptr(coo), world)
        blk = shard.x_block(coo.n, world)
        xl = np.zeros(blk)
        part = x[rank * blk:(rank + 1) * blk]
        xl[:part.size] = part
        r0, r1 = int(b[rank]), int(b[rank + 1])
        lr, lc, lv = shard.local_triplets(coo.rows, coo.cols, coo.vals, r0, r1)
        lo, hi = shard.column_window(lc)
        wins = shard.all_windows(lo, hi, world)
        send, recv = shard.halo_plan(wins, blk, rank)
        win = torch.zeros(hi - lo, dtype=torch.float64)
        shard.gather_window(torch.from_numpy(xl), torch.from_numpy(shard.send_index(send)),
                            [c for _, c in send], recv, win)
        xw = win.numpy()
        y = oracle.spmv_coo(r1 - r0, hi - lo, lr, lc - lo, lv, xw)   # columns counted from lo
        out[rank] = (r0, r1, bool(np.array_equal(xw, x[lo:hi])), y.tolist(),
                     int(sum(c for q, c in enumerate(recv) if q != rank)))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,case", [(2, "banded"), (3, "stencil"), (2, "random"), (3, "empty_block")])
def test_gloo_halo_exchange_windows_reassemble_the_product(oracle, world, case):
    """Over a real gloo group: each rank's all-to-all window equals x[lo:hi],
    the oracle product of its rows with columns counted from lo equals its
    rows of the unsharded product, and a banded matrix moves only its band
    between ranks."""
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_halo_worker, args=(r, world, port, case, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    coo = _halo_cases()[case]
    want = oracle.spmv_coo(coo.m, coo.n, coo.rows, coo.cols, coo.vals, matgen.dense_vector(coo.n, 12))
    ys, prev = [], 0
    for r in range(world):
        r0, r1, same, y, moved = out[r]
        assert same and r0 == prev
        prev = r1
        ys.extend(y)
        if case == "banded":
            assert moved <= 2 * 9
    assert prev == coo.m
    assert np.array_equal(np.array(ys), want)
