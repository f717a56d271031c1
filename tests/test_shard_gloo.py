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
