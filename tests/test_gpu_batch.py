"""Batched persistent SpMV: every matrix of an uneven batch matches the
oracle and the single-matrix path, graph replays are repeatable, and the
autotuned plan stays correct."""
import math

import numpy as np
import pytest

from paper_2302_05662_gb300 import binding as B
from paper_2302_05662_gb300 import matgen

from gpu_util import TOL, create, oracle_for, rel_err, vec_dtype

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2302_05662_gb300 import build
    build.build()
    return B.load_library()


def batch_matrices(count=40, n_lo=50, n_hi=20000, seed=0):
    rng = np.random.default_rng(seed)
    mats = []
    for i in range(count):
        fam = matgen.FAMILIES[i % len(matgen.FAMILIES)]
        n = int(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi))))
        mats.append(matgen.family_matrix(fam, n, seed=1000 + i, jitter=True))
    # edge cases inside a batch: an empty matrix and a single long row
    mats.append(matgen.Coo(7, 5, np.zeros(0, np.int32), np.zeros(0, np.int32), np.zeros(0)))
    mats.append(matgen.Coo(2, 30000, np.ones(30000, np.int32), np.arange(30000, dtype=np.int32),
                           rng.standard_normal(30000)))
    return mats


@pytest.mark.parametrize("vt", [B.SPMV_F32, B.SPMV_F64, B.SPMV_BF16])
def test_batch_matches_oracle_and_replays(oracle, vt):
    import torch
    mats = batch_matrices()
    hs, xs, ys, xh, y0 = [], [], [], [], []
    rng = np.random.default_rng(9)
    alphas = rng.uniform(-2, 2, len(mats))
    betas = np.where(np.arange(len(mats)) % 3 == 0, 0.0, rng.uniform(-1, 1, len(mats)))
    for i, coo in enumerate(mats):
        hs.append(create(coo, vt))
        x = matgen.dense_vector(coo.n, 50 + i)
        y = matgen.dense_vector(coo.m, 90 + i)
        xh.append(x)
        y0.append(y)
        xs.append(torch.from_numpy(x).to(vec_dtype(vt)).cuda())
        ys.append(torch.from_numpy(y).to(vec_dtype(vt)).cuda())
    b = B.spmv_batch_create(hs, alphas, xs, betas, ys)
    try:
        for rep in range(3):        # graph replays from the same initial y
            for i, coo in enumerate(mats):
                ys[i].copy_(torch.from_numpy(y0[i]).to(vec_dtype(vt)))
            B.spmv_batch_launch(b)
            torch.cuda.synchronize()
            outs = [y.cpu().double().numpy() for y in ys]
            if rep == 0:
                first = outs
            else:
                for o, f in zip(outs, first):
                    assert np.array_equal(o, f)
        for i, coo in enumerate(mats):
            want = oracle_for(oracle, coo, vt, xh[i], alphas[i], betas[i], y0[i])
            assert rel_err(first[i], want) <= TOL[vt], (i, coo.name)
        modes, items, tpb = B.spmv_batch_get_plan(b, len(mats))
        assert set(modes.tolist()) <= {0, 1, 2, 4, 8, 16, 32}
        assert 0 in modes.tolist()                       # the long-row matrix runs split
        # autotune, then the plan must still be right
        B.spmv_batch_tune(b)
        for i, coo in enumerate(mats):
            ys[i].copy_(torch.from_numpy(y0[i]).to(vec_dtype(vt)))
        B.spmv_batch_launch(b)
        torch.cuda.synchronize()
        for i, coo in enumerate(mats):
            want = oracle_for(oracle, coo, vt, xh[i], alphas[i], betas[i], y0[i])
            assert rel_err(ys[i].cpu().double().numpy(), want) <= TOL[vt], (i, coo.name)
        modes2, items2, tpb2 = B.spmv_batch_get_plan(b, len(mats))
        assert items2 in (4, 8, 16) and tpb2 in (128, 256, 512)
    finally:
        B.spmv_batch_destroy(b)
        for h in hs:
            B.spmv_destroy(h)


def test_batch_run_one_shot_integer_exact(oracle):
    import torch
    mats = batch_matrices(count=12, seed=3)
    for coo in mats:
        coo.vals = np.round(np.clip(coo.vals * 3, -8, 8))
    hs = [create(c, B.SPMV_F64) for c in mats]
    xs = [torch.from_numpy(matgen.dense_vector(c.n, k, integer_values=5)).cuda() for k, c in enumerate(mats)]
    ys = [torch.zeros(c.m, dtype=torch.float64, device="cuda") for c in mats]
    try:
        B.spmv_batch_run(hs, np.ones(len(mats)), xs, np.zeros(len(mats)), ys)
        for k, c in enumerate(mats):
            want = oracle.spmv_coo_obj(c, xs[k].cpu().numpy())
            assert np.array_equal(ys[k].cpu().numpy(), want), k
    finally:
        for h in hs:
            B.spmv_destroy(h)


def test_batch_of_more_matrices_than_shared_memory_offsets(oracle):
    """4200 small matrices: past 4095 the kernel searches the item offsets
    in global memory instead of shared memory; integer inputs, exact."""
    import torch
    rng = np.random.default_rng(11)
    mats = []
    for i in range(4200):
        n = int(rng.integers(1, 90))
        nnz = int(rng.integers(0, 4 * n + 1))
        coo = matgen.random_coo(n, n, nnz, np.random.default_rng(5000 + i))
        coo.vals = rng.integers(-4, 5, size=coo.nnz).astype(np.float64)
        mats.append(coo)
    hs = [create(c, B.SPMV_F64) for c in mats]
    xs = [torch.from_numpy(matgen.dense_vector(c.n, k, integer_values=5)).cuda() for k, c in enumerate(mats)]
    ys = [torch.full((c.m,), 7.0, dtype=torch.float64, device="cuda") for c in mats]
    try:
        B.spmv_batch_run(hs, np.ones(len(mats)), xs, np.full(len(mats), -1.0), ys)
        for k, c in enumerate(mats):
            want = oracle.spmv_coo_obj(c, xs[k].cpu().numpy()) - 7.0
            assert np.array_equal(ys[k].cpu().numpy(), want), k
    finally:
        for h in hs:
            B.spmv_destroy(h)


def test_batch_rejects_mixed_types():
    import torch
    a = matgen.laplacian_2d(8)
    h1 = create(a, B.SPMV_F64)
    h2 = create(a, B.SPMV_F32)
    x = torch.zeros(64, dtype=torch.float64, device="cuda")
    try:
        with pytest.raises(B.SpmvError):
            B.spmv_batch_create([h1, h2], [1, 1], [x, x], [0, 0], [x, x])
    finally:
        B.spmv_destroy(h1)
        B.spmv_destroy(h2)


def test_batch_fullsize_512_fp32_tuned(oracle):
    """The benchmark's batched workload at full size (512 fp32 matrices, n
    log-uniform in [10^3, 2*10^5], about 5.2*10^8 nonzeros), after the
    autotuner, in the graph the benchmark replays: every matrix against the
    oracle on the inputs the device holds (fp32-rounded values and x).  The
    matrices are generated again for the check so host memory stays small."""
    import torch
    hs, xs, ys = [], [], []
    try:
        for i, coo in matgen.batched_workload():
            hs.append(create(coo, B.SPMV_F32))
            xs.append(torch.from_numpy(matgen.dense_vector(coo.n, 9000 + i)).float().cuda())
            ys.append(torch.full((coo.m,), float("nan"), dtype=torch.float32, device="cuda"))
        count = len(hs)
        assert count == 512
        b = B.spmv_batch_create(hs, np.ones(count), xs, np.zeros(count), ys)
        try:
            B.spmv_batch_tune(b)
            for y in ys:
                y.fill_(float("nan"))
            B.spmv_batch_launch(b)
            torch.cuda.synchronize()
            modes, items, tpb = B.spmv_batch_get_plan(b, count)
            assert 0 in modes.tolist() and any(m != 0 for m in modes.tolist())
        finally:
            B.spmv_batch_destroy(b)
        worst = 0.0
        for i, coo in matgen.batched_workload():
            got = ys[i].cpu().double().numpy()
            want = oracle_for(oracle, coo, B.SPMV_F32, matgen.dense_vector(coo.n, 9000 + i))
            err = rel_err(got, want)
            assert err <= TOL[B.SPMV_F32], (i, coo.name, err)
            worst = max(worst, err)
        assert worst > 0.0          # fp32 accumulation differs from the fp64 oracle somewhere
    finally:
        for h in hs:
            B.spmv_destroy(h)


FORMAT_CYCLE = [B.FMT_ELL, B.FMT_SELL, B.FMT_CSR, B.FMT_COO, B.FMT_HYB, B.FMT_BSR]


@pytest.mark.parametrize("vt", [B.SPMV_F32, B.SPMV_F64, B.SPMV_BF16])
def test_batch_runs_each_matrix_in_its_format(oracle, vt):
    """Handles in ELL and SELL run in their own format inside the batch
    (modes -1 and -5), COO and BSR handles as COO chunks and BSR block rows
    (modes -2, -4) until the tuner picks, the others from their CSR arrays;
    every product matches the oracle before and after the autotuner."""
    import torch
    mats = batch_matrices(count=36, seed=3)
    hs, xs, ys, xh = [], [], [], []
    want_modes = []
    for i, coo in enumerate(mats):
        h = create(coo, vt)
        fmt = FORMAT_CYCLE[i % len(FORMAT_CYCLE)]
        try:
            B.spmv_set_config(h, B.make_config(format=fmt))
        except B.SpmvError:
            fmt = B.FMT_CSR                      # a padded format over its limit: the handle stays CSR
        hs.append(h)
        want_modes.append(-fmt if fmt in (B.FMT_ELL, B.FMT_SELL) or (fmt in (B.FMT_COO, B.FMT_BSR) and coo.nnz > 0)
                          else None)
        x = matgen.dense_vector(coo.n, 70 + i)
        xh.append(x)
        xs.append(torch.from_numpy(x).to(vec_dtype(vt)).cuda())
        ys.append(torch.full((coo.m,), float("nan"), dtype=vec_dtype(vt), device="cuda"))
    ones, zeros = np.ones(len(mats)), np.zeros(len(mats))
    b = B.spmv_batch_create(hs, ones, xs, zeros, ys)
    try:
        modes, _, _ = B.spmv_batch_get_plan(b, len(mats))
        for i, wm in enumerate(want_modes):
            if wm is not None and mats[i].m > 0:
                assert modes[i] == wm, i
            elif wm is None:
                assert modes[i] >= 0, i
        for tuned in (False, True):
            if tuned:
                B.spmv_batch_tune(b)
                modes, _, _ = B.spmv_batch_get_plan(b, len(mats))
                for i, wm in enumerate(want_modes):   # the tuner keeps ELL and SELL, may move COO, BSR to CSR
                    if wm in (-B.FMT_COO, -B.FMT_BSR):
                        assert modes[i] == wm or modes[i] >= 0, i
                    elif wm is not None and mats[i].m > 0:
                        assert modes[i] == wm, i
            for y in ys:
                y.fill_(float("nan"))
            B.spmv_batch_launch(b)
            torch.cuda.synchronize()
            for i, coo in enumerate(mats):
                want = oracle_for(oracle, coo, vt, xh[i])
                assert rel_err(ys[i].cpu().double().numpy(), want) <= TOL[vt], (tuned, i)
    finally:
        B.spmv_batch_destroy(b)
        for h in hs:
            B.spmv_destroy(h)
