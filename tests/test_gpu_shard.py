"""Row-block sharded product on one GPU: every rank's block, built as its
own handle from its rows' triplets (global columns), multiplies the whole x
into exactly the oracle's rows of that block; with the halo exchange, the
block's handle counts columns from the start of its window and multiplies
the window of x.  The all-gather and the all-to-all of x are exercised over
gloo on CPU (tests/test_shard_gloo.py); here the gathered buffers are
filled directly, as the exchange would leave them."""
import numpy as np
import pytest

from paper_2302_05662_gb300 import binding as B
from paper_2302_05662_gb300 import matgen, shard

from gpu_util import TOL, rel_err, stored_values, stored_vector, device_values

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2302_05662_gb300 import build
    build.build()
    return B.load_library()


CASES = [("stencil27_16", lambda: matgen.stencil_3d(16, 27, np.random.default_rng(1))),
         ("rmat_s12", lambda: matgen.rmat(12, 16, np.random.default_rng(2))),
         ("banded_5000_w32", lambda: matgen.banded(5000, 32, np.random.default_rng(3)))]


@pytest.mark.parametrize("vt", [B.SPMV_F64, B.SPMV_F32])
@pytest.mark.parametrize("parts", [1, 3, 8])
@pytest.mark.parametrize("case", [c[0] for c in CASES])
def test_every_rank_block_matches_the_oracle_rows(oracle, case, parts, vt):
    import torch
    coo = dict(CASES)[case]()
    rp = np.zeros(coo.m + 1, np.int64)
    np.cumsum(np.bincount(coo.rows, minlength=coo.m), out=rp[1:])
    bounds = shard.partition_rows(rp, parts)
    x = matgen.dense_vector(coo.n, 7)
    want = oracle.spmv_coo(coo.m, coo.n, coo.rows, coo.cols, stored_values(coo.vals, vt), stored_vector(x, vt))
    rows = torch.from_numpy(coo.rows).cuda()
    cols = torch.from_numpy(coo.cols).cuda()
    vals = device_values(coo.vals, vt)
    xt = torch.from_numpy(x).to(torch.float64 if vt == B.SPMV_F64 else torch.float32).cuda()
    got = []
    for rank in range(parts):
        r0, r1 = int(bounds[rank]), int(bounds[rank + 1])
        lr, lc, lv = shard.local_triplets(rows, cols, vals, r0, r1)
        sm = shard.ShardedMatrix(coo.m, coo.n, lr + r0, lc, lv, bounds, rank, parts)
        try:
            y = torch.full((r1 - r0,), float("nan"), dtype=sm.vec_dtype, device="cuda")
            if parts == 1:
                sm.run(1.0, xt, 0.0, y)               # the gather of one rank is a copy
            else:
                sm.x_full[:coo.n].copy_(xt)           # as the all-gather leaves it
                B.spmv_run(sm.h, 1.0, sm.x_full, 0.0, y)
            torch.cuda.synchronize()
            got.append(y.cpu().double().numpy())
        finally:
            sm.destroy()
    for rank in range(parts):
        r0, r1 = int(bounds[rank]), int(bounds[rank + 1])
        if r1 > r0:
            assert rel_err(got[rank], want[r0:r1]) <= TOL[vt], rank
    assert rel_err(np.concatenate(got), want) <= TOL[vt]


@pytest.mark.parametrize("vt", [B.SPMV_F64, B.SPMV_F32])
@pytest.mark.parametrize("parts", [1, 3, 8])
@pytest.mark.parametrize("case", [c[0] for c in CASES])
def test_every_rank_window_matches_the_oracle_rows(oracle, case, parts, vt):
    import torch
    coo = dict(CASES)[case]()
    rp = np.zeros(coo.m + 1, np.int64)
    np.cumsum(np.bincount(coo.rows, minlength=coo.m), out=rp[1:])
    bounds = shard.partition_rows(rp, parts)
    x = matgen.dense_vector(coo.n, 8)
    want = oracle.spmv_coo(coo.m, coo.n, coo.rows, coo.cols, stored_values(coo.vals, vt), stored_vector(x, vt))
    wins = [shard.column_window(shard.local_triplets(coo.rows, coo.cols, coo.vals, int(bounds[r]),
                                                     int(bounds[r + 1]))[1]) for r in range(parts)]
    rows = torch.from_numpy(coo.rows).cuda()
    cols = torch.from_numpy(coo.cols).cuda()
    vals = device_values(coo.vals, vt)
    xt = torch.from_numpy(x).to(torch.float64 if vt == B.SPMV_F64 else torch.float32).cuda()
    got = []
    for rank in range(parts):
        r0, r1 = int(bounds[rank]), int(bounds[rank + 1])
        lr, lc, lv = shard.local_triplets(rows, cols, vals, r0, r1)
        sm = shard.ShardedMatrix(coo.m, coo.n, lr + r0, lc, lv, bounds, rank, parts, halo=True, windows=wins)
        try:
            assert (sm.lo, sm.hi) == wins[rank] and sm.x_win.numel() == sm.hi - sm.lo
            y = torch.full((r1 - r0,), float("nan"), dtype=sm.vec_dtype, device="cuda")
            if parts == 1:
                sm.run(1.0, xt, 0.0, y)               # one rank: the window is a copy
            else:
                sm.x_win.copy_(xt[sm.lo:sm.hi])       # as the all-to-all leaves it
                B.spmv_run(sm.h, 1.0, sm.x_win, 0.0, y)
            torch.cuda.synchronize()
            got.append(y.cpu().double().numpy())
        finally:
            sm.destroy()
    for rank in range(parts):
        r0, r1 = int(bounds[rank]), int(bounds[rank + 1])
        if r1 > r0:
            assert rel_err(got[rank], want[r0:r1]) <= TOL[vt], rank
    assert rel_err(np.concatenate(got), want) <= TOL[vt]
