"""GPU parity of row panels: matrices given with more triplets than one
handle indexes with int32 offsets are held as sub-handles over row ranges.

Small cases lower the panel limit so every format runs on several panels
and must give what one handle gives: the oracle's products (bit-exact on
integer inputs), identical features, identical CG iterates for a row-local
kernel.  The full-size case builds a banded matrix with more than 2^31
nonzeros at the default limit and checks sampled rows exactly.
"""
import numpy as np
import pytest

from paper_2302_05662_gb300 import binding as B
from paper_2302_05662_gb300 import matgen
from paper_2302_05662_gb300.workload import SWEEP_VARIANTS

from gpu_util import TOL, create, oracle_for, rel_err, run

pytestmark = pytest.mark.gpu
VARIANTS = dict(SWEEP_VARIANTS)
SMALL = dict(matgen.workload_matrices("small"))
FEAT_BANDWIDTH, FEAT_DIAG = 14, 16       # positions in the 20-feature vector


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2302_05662_gb300 import build
    build.build()
    return B.load_library()


@pytest.fixture
def panel_limit():
    """Set a small panel limit for the test; the default comes back after."""
    def set_(v):
        B.spmv_set_panel_limit(v)
    yield set_
    B.spmv_set_panel_limit(B.PANEL_LIMIT_DEFAULT)


def test_panel_limit_bounds():
    assert B.spmv_get_panel_limit() == B.PANEL_LIMIT_DEFAULT
    for bad in (0, -5, (1 << 31) - 1, 1 << 31):
        with pytest.raises(B.SpmvError) as ei:
            B.spmv_set_panel_limit(bad)
        assert ei.value.status == -1
    assert B.spmv_get_panel_limit() == B.PANEL_LIMIT_DEFAULT


@pytest.mark.parametrize("vt", (B.SPMV_F64, B.SPMV_F32, B.SPMV_BF16))
@pytest.mark.parametrize("name", list(VARIANTS))
@pytest.mark.parametrize("family", list(SMALL))
def test_panels_match_oracle(oracle, panel_limit, family, name, vt):
    coo = SMALL[family]
    panel_limit(max(coo.nnz // 5, 64))
    x = matgen.dense_vector(coo.n, 5)
    try:
        h = create(coo, vt, B.make_config(**VARIANTS[name]))
    except B.SpmvError as e:      # a padded format over its limit on some panel
        assert e.status == -4 and name in ("ell", "bsr", "sell")
        return
    try:
        info = B.spmv_get_info(h)
        assert info.panels >= 4 and info.nnz == coo.nnz and info.format == VARIANTS[name]["format"]
        got = run(h, vt, x, m=coo.m)
        y0 = matgen.dense_vector(coo.m, 6)
        got2 = run(h, vt, x, 2.0, -0.5, y0, m=coo.m)
    finally:
        B.spmv_destroy(h)
    assert rel_err(got, oracle_for(oracle, coo, vt, x)) <= TOL[vt]
    assert rel_err(got2, oracle_for(oracle, coo, vt, x, 2.0, -0.5, y0)) <= TOL[vt]


@pytest.mark.parametrize("name", list(VARIANTS))
def test_panels_unsorted_duplicates_bit_exact(oracle, panel_limit, name):
    rng = np.random.default_rng(3)
    coo = matgen.random_coo(2001, 900, 12000, rng, integer_values=6)
    dup = rng.integers(0, coo.nnz, 3000)
    rows = np.concatenate([coo.rows, coo.rows[dup]])
    cols = np.concatenate([coo.cols, coo.cols[dup]])
    vals = np.concatenate([coo.vals, rng.integers(-6, 7, dup.size).astype(float)])
    perm = rng.permutation(rows.size)
    full = matgen.Coo(coo.m, coo.n, rows[perm], cols[perm], vals[perm])
    panel_limit(2500)
    x = matgen.dense_vector(coo.n, 7, integer_values=5)
    h = create(full, B.SPMV_F64, B.make_config(**VARIANTS[name]))
    try:
        assert B.spmv_get_info(h).panels >= 6
        got = run(h, B.SPMV_F64, x, m=coo.m)
    finally:
        B.spmv_destroy(h)
    assert np.array_equal(got, oracle.spmv_coo_obj(full, x))


def test_panel_boundaries_and_features(panel_limit):
    """Features of a panelled handle equal those of one handle; panel row
    ranges start at multiples of 4 (the 4x4 block feature stays exact)."""
    for family, coo in SMALL.items():
        h1 = create(coo, B.SPMV_F64)
        try:
            f1 = B.spmv_features(h1)
        finally:
            B.spmv_destroy(h1)
        panel_limit(max(coo.nnz // 7, 64))
        h2 = create(coo, B.SPMV_F64)
        try:
            assert B.spmv_get_info(h2).panels >= 7
            f2 = B.spmv_features(h2)
        finally:
            B.spmv_destroy(h2)
            B.spmv_set_panel_limit(B.PANEL_LIMIT_DEFAULT)
        assert np.array_equal(f1, f2), family


def test_cg_on_panels_equals_one_handle(panel_limit):
    coo = matgen.stencil_3d(16, 27, values="laplace")
    import torch
    b = torch.from_numpy(matgen.dense_vector(coo.m, 1)).cuda()
    out = []
    for limit in (B.PANEL_LIMIT_DEFAULT, 9000):
        panel_limit(limit)
        h = create(coo, B.SPMV_F64, B.make_config(format=B.FMT_CSR, threads_per_row=8))
        try:
            x = torch.zeros(coo.m, dtype=torch.float64, device="cuda")
            res = B.spmv_cg(h, b, x, 1e-10, 500)
            out.append((B.spmv_get_info(h).panels, res.iterations, x.cpu().numpy()))
        finally:
            B.spmv_destroy(h)
    assert out[0][0] == 1 and out[1][0] >= 8
    assert out[0][1] == out[1][1] and np.array_equal(out[0][2], out[1][2])


def test_set_config_and_refusals_on_panels(oracle, panel_limit):
    coo = SMALL["rmat_s14_ef16"]
    panel_limit(coo.nnz // 4)
    h = create(coo, B.SPMV_F64)
    x = matgen.dense_vector(coo.n, 2)
    try:
        for name in VARIANTS:
            try:
                B.spmv_set_config(h, B.make_config(**VARIANTS[name]))
            except B.SpmvError as e:          # refused on some panel: every panel back on CSR
                assert e.status == -4
                assert B.spmv_get_config(h).format == B.FMT_CSR
            got = run(h, B.SPMV_F64, x, m=coo.m)
            assert rel_err(got, oracle.spmv_coo_obj(coo, x)) <= 1e-13
        with pytest.raises(B.SpmvError) as ei:
            B.spmv_export_bytes(h, B.ARR_CSR_ROWPTR)
        assert ei.value.status == -4
        import torch
        xt = torch.from_numpy(x).cuda()
        yt = torch.zeros(coo.m, dtype=torch.float64, device="cuda")
        with pytest.raises(B.SpmvError) as ei:
            B.spmv_batch_create([h], np.ones(1), [xt], np.zeros(1), [yt])
        assert ei.value.status == -4
    finally:
        B.spmv_destroy(h)


def test_four_rows_over_the_limit_refused(panel_limit):
    coo = matgen.Coo(8, 100, np.zeros(60, np.int32), np.arange(60, dtype=np.int32), np.ones(60))
    panel_limit(50)
    with pytest.raises(B.SpmvError) as ei:
        create(coo, B.SPMV_F64)
    assert ei.value.status == -4


def test_more_than_2_31_nonzeros_banded():
    """Banded matrix, n = 2^25, half-width 32: 65 n - 1056 > 2^31 triplets
    at the default panel limit.  Integer values and x make every row sum
    exact; sampled rows (both panel sides, the ends, random rows) are
    checked bit for bit against the closed-form row."""
    import torch
    n, w = 1 << 25, 32
    nnz = (2 * w + 1) * n - w * (w + 1)
    assert nnz >= 1 << 31
    free, _ = torch.cuda.mem_get_info()
    if free < 120 << 30:
        pytest.skip("needs about 100 GB of free device memory")
    dev = "cuda"
    rows = torch.empty(nnz, dtype=torch.int32, device=dev)
    cols = torch.empty(nnz, dtype=torch.int32, device=dev)
    vals = torch.empty(nnz, dtype=torch.float64, device=dev)
    off = torch.arange(-w, w + 1, device=dev, dtype=torch.int64)
    pos, R = 0, 1 << 20
    for r0 in range(0, n, R):
        r = torch.arange(r0, min(n, r0 + R), device=dev, dtype=torch.int64)
        c = r[:, None] + off[None, :]
        ok = (c >= 0) & (c < n)
        rr = r[:, None].expand_as(c)[ok]
        cc = c[ok]
        k = rr.numel()
        rows[pos:pos + k] = rr.to(torch.int32)
        cols[pos:pos + k] = cc.to(torch.int32)
        vals[pos:pos + k] = ((rr * 7 + cc * 13) % 17 - 8).to(torch.float64)
        pos += k
    assert pos == nnz
    xs = torch.arange(n, device=dev, dtype=torch.int64)
    x = ((xs * 5) % 11 - 5).to(torch.float64)
    y = torch.full((n,), float("nan"), dtype=torch.float64, device=dev)
    h = B.spmv_create(n, n, rows, cols, vals)
    del rows, cols, vals
    torch.cuda.empty_cache()
    try:
        info = B.spmv_get_info(h)
        assert info.panels >= 2 and info.nnz == nnz and info.max_row == 2 * w + 1
        f = B.spmv_features(h)
        B.spmv_run(h, 1.0, x, 0.0, y)
        torch.cuda.synchronize()
        yh = y.cpu().numpy()
    finally:
        B.spmv_destroy(h)
        del x, y
        torch.cuda.empty_cache()
    rng = np.random.default_rng(0)
    sample = np.unique(np.concatenate([[0, 1, w, n // 2 - 1, n // 2, n // 2 + 1, n - 2, n - 1],
                                       rng.integers(0, n, 2000)]))
    for i in sample:
        j = np.arange(max(0, i - w), min(n, i + w + 1))
        want = float(np.sum(((i * 7 + j * 13) % 17 - 8) * ((j * 5) % 11 - 5)))
        assert yh[i] == want, i
    assert not np.isnan(yh).any()
    # features over both panels: n, nnz, max row length, bandwidth, diagonal fraction
    assert f[0] == n and f[1] == nnz and f[7] == 2 * w + 1
    assert f[FEAT_BANDWIDTH] == w and f[FEAT_DIAG] == pytest.approx(n / nnz, rel=1e-12)
