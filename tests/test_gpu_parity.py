"""GPU parity: every format kernel, value type and launch variant against the
fp64 oracle, through the C ABI.

Bars: bit-exact on integer-valued inputs (all partial sums exact in every
value type) and for the index arrays of the conversions; otherwise the
normwise relative error bounds 1e-13 (fp64), 1e-5 (fp32) and 1e-2 (bf16,
against the oracle on the rounded inputs the device holds).
"""
import numpy as np
import pytest

from paper_2302_05662_gb300 import binding as B
from paper_2302_05662_gb300 import matgen
from paper_2302_05662_gb300.workload import SWEEP_VARIANTS

from gpu_util import TOL, create, oracle_for, rel_err, run, stored_vector

pytestmark = pytest.mark.gpu

VTS = (B.SPMV_F64, B.SPMV_F32, B.SPMV_BF16)
VARIANTS = dict(SWEEP_VARIANTS)


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2302_05662_gb300 import build
    build.build()
    return B.load_library()


def ell_supported(coo):
    """The library's ELL size limit: width * pitch <= 8 nnz + 2^24 slots."""
    lens = np.bincount(coo.rows, minlength=coo.m) if coo.m else np.zeros(1, np.int64)
    pitch = (coo.m + 31) // 32 * 32
    return int(lens.max()) * pitch <= 8 * coo.nnz + (1 << 24)


def cfg_of(name, **extra):
    kw = dict(VARIANTS[name])
    kw.update(extra)
    return B.make_config(**kw)


def check(oracle, coo, vt, cfg, x, alpha=1.0, beta=0.0, y0=None, exact=False):
    if cfg.format == B.FMT_ELL and not ell_supported(coo):
        with pytest.raises(B.SpmvError) as ei:      # padded size over the limit
            create(coo, vt, cfg)
        assert ei.value.status == -4
        return None
    h = create(coo, vt, cfg)
    try:
        got = run(h, vt, x, alpha, beta, y0, m=coo.m)
    finally:
        B.spmv_destroy(h)
    want = oracle_for(oracle, coo, vt, x, alpha, beta, y0)
    if exact:
        assert np.array_equal(got, want), f"max diff {np.max(np.abs(got - want))}"
    else:
        err = rel_err(got, want)
        assert err <= TOL[vt], f"normwise error {err:.3e} > {TOL[vt]:.0e}"
    return got


# ------------------------------------------------------------------ config 1
@pytest.mark.parametrize("name", list(VARIANTS))
def test_laplacian_64x64_fp64(oracle, name):
    """2D 5-point Laplacian on 64x64 (n = 4096, nnz = 20224, values 4/-1),
    x ~ U[-1,1] seed 0, alpha = 1, beta = 0."""
    coo = matgen.laplacian_2d(64)
    assert coo.nnz == 20224
    x = matgen.dense_vector(coo.n, 0)
    check(oracle, coo, B.SPMV_F64, cfg_of(name), x)
    xi = matgen.dense_vector(coo.n, 0, integer_values=8)
    for vt in VTS:
        check(oracle, coo, vt, cfg_of(name), xi, exact=True)


# ----------------------------------------------- small versions of config 2/3
SMALL = dict(matgen.workload_matrices("small"))


@pytest.mark.parametrize("vt", VTS)
@pytest.mark.parametrize("name", list(VARIANTS))
@pytest.mark.parametrize("family", list(SMALL))
def test_small_workload(oracle, family, name, vt):
    coo = SMALL[family]
    x = matgen.dense_vector(coo.n, 5)
    got = check(oracle, coo, vt, cfg_of(name), x)
    if got is not None and vt == B.SPMV_F32:   # also against the original fp64 inputs
        want = oracle.spmv_coo_obj(coo, x)
        assert rel_err(got, want) <= 1e-5


@pytest.mark.parametrize("vt", VTS)
@pytest.mark.parametrize("name", list(VARIANTS))
def test_integer_inputs_bit_exact(oracle, name, vt):
    rng = np.random.default_rng(11)
    for m, n, nnz in ((1000, 700, 9000), (37, 1000, 2000), (3000, 3, 4000), (1, 5000, 4000)):
        coo = matgen.random_coo(m, n, nnz, rng, integer_values=8)
        x = matgen.dense_vector(n, m, integer_values=8)
        y0 = matgen.dense_vector(m, n, integer_values=8)
        check(oracle, coo, vt, cfg_of(name), x, exact=True)
        check(oracle, coo, vt, cfg_of(name), x, alpha=2.0, beta=-3.0, y0=y0, exact=True)


# ------------------------------------------------------- launch-parameter space
def _power_law_int(seed=3):
    rng = np.random.default_rng(seed)
    coo = matgen.rmat(12, 16, rng)
    coo.vals = rng.integers(-8, 9, size=coo.nnz).astype(np.float64)
    return coo


LAUNCH_CASES = (
    [("csr", dict(threads_per_row=t, unroll=u, regcap=rc))
     for t in (1, 2, 4, 8, 16, 32) for u in (1, 2, 4) for rc in (32, 64)]
    + [("csr_split", dict(unroll=u)) for u in (1, 2, 4)]
    + [("csr_split", dict(hyb_ell_width=w, unroll=u)) for w in (256, 1024, 8192) for u in (2, 4)]
    + [(nm, dict(unroll=u, regcap=rc)) for nm in ("ell", "hyb", "sell")
       for u in (1, 2, 4, 8) for rc in (32, 48, 64)]
    + [("coo", dict(unroll=u)) for u in (1, 2, 4)]
    + [("hyb", dict(hyb_ell_width=w)) for w in (1, 3, 100)]
    + [("sell", dict(hyb_ell_width=w)) for w in (8, 24, 64, 1024)]
    + [("bsr", dict(bsr_block=r, threads_per_row=s)) for r in (2, 4) for s in (1, 2, 4, 8)]
    + [(nm, dict(threads_per_block=t)) for nm in VARIANTS for t in (32, 1024)]
    + [(nm, dict(carveout=cv)) for nm in ("csr", "coo") for cv in (0, 50, 100, -1)]
)


@pytest.mark.parametrize("vt", VTS)
@pytest.mark.parametrize("case", range(len(LAUNCH_CASES)))
def test_launch_variants_bit_exact(oracle, case, vt):
    name, kw = LAUNCH_CASES[case]
    coo = _power_law_int()
    x = matgen.dense_vector(coo.n, 1, integer_values=8)
    y0 = matgen.dense_vector(coo.m, 2, integer_values=8)
    check(oracle, coo, vt, cfg_of(name, **kw), x, 1.0, 0.0, exact=True)
    check(oracle, coo, vt, cfg_of(name, **kw), x, -1.0, 2.0, y0, exact=True)


# --------------------------------------------------------------- edge cases
def _edge_cases():
    rng = np.random.default_rng(17)
    out = []
    out.append(("one_long_row", matgen.Coo(1, 20000, np.zeros(20000, np.int32),
                                           np.arange(20000, dtype=np.int32),
                                           rng.integers(-4, 5, 20000).astype(float))))
    r = np.concatenate([np.zeros(3, np.int32), np.full(9000, 4000, np.int32), np.full(2, 9999, np.int32)])
    c = np.concatenate([np.arange(3), np.arange(9000), np.arange(2)]).astype(np.int32)
    out.append(("empty_rows_long_row", matgen.Coo(10000, 9001, r, c, rng.integers(-4, 5, r.size).astype(float))))
    out.append(("single_entry", matgen.Coo(7, 5, np.array([6], np.int32), np.array([4], np.int32),
                                           np.array([3.0]))))
    out.append(("ragged_bsr", matgen.random_coo(1001, 1003, 5000, rng, integer_values=5)))
    out.append(("wide", matgen.random_coo(3, 4000, 3000, rng, integer_values=5)))
    out.append(("tall", matgen.random_coo(4000, 3, 3000, rng, integer_values=5)))
    out.append(("chunk_multiple", matgen.random_coo(256, 256, 8192, rng, integer_values=5)))
    # ELL stores 16-bit column offsets while every |col - row| <= 32767
    r = np.array([0, 1, 32767, 39999], np.int32)
    out.append(("offset_32767", matgen.Coo(40000, 40000, r, np.array([32767, 1, 0, 7232], np.int32),
                                           np.array([3.0, -2.0, 5.0, 1.0]))))
    out.append(("offset_32768", matgen.Coo(40000, 40001, r, np.array([32768, 1, 0, 40000], np.int32),
                                           np.array([3.0, -2.0, 5.0, 1.0]))))
    return out


EDGE = _edge_cases()


@pytest.mark.parametrize("vt", VTS)
@pytest.mark.parametrize("name", list(VARIANTS))
@pytest.mark.parametrize("case", [e[0] for e in EDGE])
def test_edge_cases_bit_exact(oracle, case, name, vt):
    coo = dict(EDGE)[case]
    x = matgen.dense_vector(coo.n, 9, integer_values=6)
    y0 = matgen.dense_vector(coo.m, 8, integer_values=6)
    check(oracle, coo, vt, cfg_of(name), x, exact=True)
    check(oracle, coo, vt, cfg_of(name), x, 3.0, -1.0, y0, exact=True)


@pytest.mark.parametrize("name", list(VARIANTS))
def test_empty_matrices(name):
    import torch
    for m, n in ((5, 4), (0, 3), (3, 0)):
        empty = torch.zeros(0, dtype=torch.int32, device="cuda")
        h = B.spmv_create(m, n, empty, empty, torch.zeros(0, dtype=torch.float64, device="cuda"), cfg_of(name))
        try:
            x = torch.ones(n, dtype=torch.float64, device="cuda")
            y = torch.full((m,), float("nan"), dtype=torch.float64, device="cuda")
            B.spmv_run(h, 1.0, x, 0.0, y)
            assert torch.equal(y, torch.zeros(m, dtype=torch.float64, device="cuda"))
            y = torch.arange(m, dtype=torch.float64, device="cuda")
            B.spmv_run(h, 1.0, x, 2.5, y)
            assert torch.equal(y, 2.5 * torch.arange(m, dtype=torch.float64, device="cuda"))
        finally:
            B.spmv_destroy(h)


def test_beta_zero_ignores_nan_y(oracle):
    coo = SMALL["poisson16_2^14"]
    x = matgen.dense_vector(coo.n, 1)
    for name in VARIANTS:
        h = create(coo, B.SPMV_F64, cfg_of(name))
        try:
            got = run(h, B.SPMV_F64, x, 1.0, 0.0, None, m=coo.m)   # y starts as NaN
        finally:
            B.spmv_destroy(h)
        assert np.all(np.isfinite(got)), name


# ------------------------------------------------------------ conversions
def test_unsorted_duplicates_convert_like_oracle(oracle):
    import torch
    rng = np.random.default_rng(23)
    coo = matgen.random_coo(3000, 2500, 40000, rng, duplicates=True, shuffle=True, integer_values=7)
    rp, ci, cv = oracle.csr_from_coo(coo.m, coo.n, coo.rows, coo.cols, coo.vals)
    for vt in VTS:
        h = create(coo, vt)
        try:
            info = B.spmv_get_info(h)
            assert info.nnz == ci.size
            g_rp = torch.empty(coo.m + 1, dtype=torch.int32, device="cuda")
            g_ci = torch.empty(info.nnz, dtype=torch.int32, device="cuda")
            B.spmv_export(h, B.ARR_CSR_ROWPTR, g_rp)
            B.spmv_export(h, B.ARR_CSR_COLIDX, g_ci)
            assert np.array_equal(g_rp.cpu().numpy(), rp)
            assert np.array_equal(g_ci.cpu().numpy(), ci)
            from gpu_util import torch_dtype
            g_v = torch.empty(info.nnz, dtype=torch_dtype(vt), device="cuda")
            B.spmv_export(h, B.ARR_CSR_VALS, g_v)
            assert np.array_equal(g_v.cpu().double().numpy(), cv)
            x = matgen.dense_vector(coo.n, 4, integer_values=5)
            assert np.array_equal(run(h, vt, x, m=coo.m), oracle_for(oracle, coo, vt, x))
        finally:
            B.spmv_destroy(h)


def _export(h, arr, dtype):
    import torch
    nbytes = B.spmv_export_bytes(h, arr)
    t = torch.empty(nbytes // torch.tensor([], dtype=dtype).element_size(), dtype=dtype, device="cuda")
    B.spmv_export(h, arr, t)
    return t.cpu()


def test_format_layouts_decode_to_the_matrix(oracle):
    import torch
    coo = SMALL["rmat_s14_ef16"]
    coo_i = matgen.Coo(coo.m, coo.n, coo.rows, coo.cols,
                       np.random.default_rng(1).integers(-9, 10, coo.nnz).astype(float))
    dense_keys = set(zip(coo_i.rows.tolist(), coo_i.cols.tolist()))
    ref = {(r, c): v for r, c, v in zip(coo_i.rows.tolist(), coo_i.cols.tolist(), coo_i.vals.tolist())}
    lens = np.bincount(coo_i.rows, minlength=coo_i.m)
    # ELL (on the Poisson-row matrix; the R-MAT one is over the ELL size
    # limit): column-major [width][pitch], -1 padding, left-packed rows
    pe = SMALL["poisson16_2^14"]
    pe = matgen.Coo(pe.m, pe.n, pe.rows, pe.cols,
                    np.random.default_rng(2).integers(-9, 10, pe.nnz).astype(float))
    ref_e = {(r, c): v for r, c, v in zip(pe.rows.tolist(), pe.cols.tolist(), pe.vals.tolist())}
    h = create(pe, B.SPMV_F64, cfg_of("ell"))
    info = B.spmv_get_info(h)
    pitch = B.spmv_export_bytes(h, B.ARR_ELL_PITCH)
    col = _export(h, B.ARR_ELL_COLIDX, torch.int32).numpy().reshape(info.ell_width, pitch)
    val = _export(h, B.ARR_ELL_VALS, torch.float64).numpy().reshape(info.ell_width, pitch)
    B.spmv_destroy(h)
    assert info.ell_width == np.bincount(pe.rows, minlength=pe.m).max() and pitch % 32 == 0
    got = {}
    for r in range(pe.m):
        for k in range(info.ell_width):
            if col[k, r] < 0:
                assert np.all(col[k:, r] < 0) and np.all(val[k:, r] == 0)
                break
            got[(r, int(col[k, r]))] = val[k, r]
    assert got == ref_e
    # HYB: width from the rule, ELL part + COO tail
    h = create(coo_i, B.SPMV_F64, cfg_of("hyb"))
    info = B.spmv_get_info(h)
    K = oracle.hyb_ell_width(lens, coo_i.m)
    assert info.ell_width == K
    assert info.hyb_coo_nnz == int(np.maximum(lens - K, 0).sum())
    pitch = B.spmv_export_bytes(h, B.ARR_ELL_PITCH)
    got = {}
    if K:
        col = _export(h, B.ARR_ELL_COLIDX, torch.int32).numpy().reshape(K, pitch)
        val = _export(h, B.ARR_ELL_VALS, torch.float64).numpy().reshape(K, pitch)
        for r in range(coo_i.m):
            for k in range(K):
                if col[k, r] >= 0:
                    got[(r, int(col[k, r]))] = val[k, r]
    tr = _export(h, B.ARR_COO_ROWS, torch.int32).numpy()
    tc = _export(h, B.ARR_COO_COLS, torch.int32).numpy()
    tv = _export(h, B.ARR_COO_VALS, torch.float64).numpy()
    B.spmv_destroy(h)
    assert np.all(np.diff(tr) >= 0)
    for r, c, v in zip(tr.tolist(), tc.tolist(), tv.tolist()):
        assert (r, c) not in got
        got[(r, c)] = v
    assert got == ref
    # BSR: r x r row-major blocks, sorted block columns per block row
    for r in (2, 4):
        h = create(coo_i, B.SPMV_F64, cfg_of("bsr", bsr_block=r))
        info = B.spmv_get_info(h)
        brp = _export(h, B.ARR_BSR_ROWPTR, torch.int32).numpy()
        bci = _export(h, B.ARR_BSR_COLIDX, torch.int32).numpy()
        bv = _export(h, B.ARR_BSR_VALS, torch.float64).numpy().reshape(-1, r, r)
        B.spmv_destroy(h)
        blocks = {(a // r, b // r) for a, b in dense_keys}
        assert info.bsr_blocks == len(blocks)
        got = {}
        for br in range(brp.size - 1):
            seg = bci[brp[br]:brp[br + 1]]
            assert np.all(np.diff(seg) > 0)
            for k in range(brp[br], brp[br + 1]):
                for i in range(r):
                    for j in range(r):
                        if (br * r + i, bci[k] * r + j) in ref:
                            got[(br * r + i, int(bci[k]) * r + j)] = bv[k, i, j]
                        else:
                            assert bv[k, i, j] == 0
        assert got == ref


def test_sell_layout_decodes_to_the_matrix():
    """SELL: 32-row slices of width w; with column groups, entry k of lane l
    (sorted row p, slice s = p // 32, l = p % 32) at ptr[s] + 128 (k // 4) +
    4 l + k % 4 for the first w & ~3 columns (a lane's four entries of a
    group contiguous) and at ptr[s] + 32 (w & ~3) + 32 (k - (w & ~3)) + l
    after them; column-major, entry k at ptr[s] + 32 k + l; rows
    sorted by descending length (stable), perm maps a sorted row back to its
    matrix row, padding -1 / 0 after each row."""
    import torch
    cases = [(coo, g) for coo in (SMALL["rmat_s14_ef16"], matgen.random_coo(1000, 700, 6000, np.random.default_rng(4)),
                                  matgen.Coo(37, 9, np.array([0, 36], np.int32), np.array([1, 8], np.int32),
                                             np.array([2.0, 3.0])))
             for g in (0, 1, 4)]     # column groups: chosen per matrix, column-major, groups of four
    for coo, g in cases:
        vals = np.random.default_rng(5).integers(-9, 10, coo.nnz).astype(float)
        ci = matgen.Coo(coo.m, coo.n, coo.rows, coo.cols, vals)
        ref = {(r, c): v for r, c, v in zip(ci.rows.tolist(), ci.cols.tolist(), ci.vals.tolist())}
        lens = np.bincount(ci.rows, minlength=ci.m)
        h = create(ci, B.SPMV_F64, B.make_config(format=B.FMT_SELL, bsr_block=g))
        try:
            grouped = B.spmv_get_config(h).bsr_block == 4
            assert g == 0 or grouped == (g == 4)
            info = B.spmv_get_info(h)
            ptr = _export(h, B.ARR_SELL_PTR, torch.int32).numpy()
            col = _export(h, B.ARR_SELL_COLIDX, torch.int32).numpy()
            val = _export(h, B.ARR_SELL_VALS, torch.float64).numpy()
            perm = _export(h, B.ARR_SELL_PERM, torch.int32).numpy()
        finally:
            B.spmv_destroy(h)
        assert sorted(perm.tolist()) == list(range(ci.m))
        pl = lens[perm]
        assert np.all(np.diff(pl) <= 0)                                 # descending lengths
        same = np.flatnonzero(np.diff(pl) == 0)
        assert np.all(perm[same] < perm[same + 1])                      # stable among equal lengths
        assert info.sell_slots == ptr[-1]
        def slot(sl, width, k, l):
            w4 = width & ~3 if grouped else 0
            return ptr[sl] + (128 * (k // 4) + 4 * l + k % 4 if k < w4 else 32 * w4 + 32 * (k - w4) + l)

        got = {}
        for p in range(ci.m):
            sl, l = divmod(p, 32)
            width = (ptr[sl + 1] - ptr[sl]) // 32
            for k in range(width):
                c = col[slot(sl, width, k, l)]
                if c < 0:
                    assert all(col[slot(sl, width, j, l)] < 0 for j in range(k, width))
                    break
                got[(int(perm[p]), int(c))] = val[slot(sl, width, k, l)]
        assert got == ref
        # every slot is filled exactly once by the layout
        seen = sorted(slot(sl, (ptr[sl + 1] - ptr[sl]) // 32, k, l) for sl in range(len(ptr) - 1)
                      for k in range((ptr[sl + 1] - ptr[sl]) // 32) for l in range(32))
        assert seen == list(range(int(ptr[-1])))


def test_invalid_triplets_rejected():
    import torch
    r = torch.tensor([0, 5], dtype=torch.int32, device="cuda")
    c = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    v = torch.ones(2, dtype=torch.float64, device="cuda")
    with pytest.raises(B.SpmvError) as ei:
        B.spmv_create(5, 5, r, c, v)
    assert ei.value.status == -1
    c2 = torch.tensor([0, -1], dtype=torch.int32, device="cuda")
    r2 = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    with pytest.raises(B.SpmvError):
        B.spmv_create(5, 5, r2, c2, v)


def test_ell_width_limit_reported():
    coo = matgen.Coo(100000, 100000, np.concatenate([np.zeros(50000, np.int32), np.arange(1, 100000, dtype=np.int32)]),
                     np.concatenate([np.arange(50000, dtype=np.int32), np.zeros(99999, np.int32)]),
                     np.ones(149999))
    with pytest.raises(B.SpmvError) as ei:
        create(coo, B.SPMV_F64, cfg_of("ell"))
    assert ei.value.status == -4


@pytest.mark.parametrize("name", ["coo", "csr_split", "csr_tiles", "hyb"])
def test_repeated_runs_bitwise_identical(oracle, name):
    """The cross-chunk counters reset themselves: back-to-back products on
    one handle give identical bits (sums in a fixed order)."""
    import torch
    coo = SMALL["rmat_s14_ef16"]
    x = matgen.dense_vector(coo.n, 3)
    h = create(coo, B.SPMV_F64, cfg_of(name))
    try:
        xt = torch.from_numpy(x).cuda()
        outs = []
        for _ in range(5):
            y = torch.empty(coo.m, dtype=torch.float64, device="cuda")
            B.spmv_run(h, 1.0, xt, 0.0, y)
            outs.append(y.cpu().numpy())
        for o in outs[1:]:
            assert np.array_equal(o, outs[0])
        assert rel_err(outs[0], oracle.spmv_coo_obj(coo, x)) <= 1e-13
    finally:
        B.spmv_destroy(h)


def test_set_config_switches_formats(oracle):
    coo = SMALL["banded_2^14_w32"]
    x = matgen.dense_vector(coo.n, 2)
    want = oracle.spmv_coo_obj(coo, x)
    h = create(coo, B.SPMV_F64)
    try:
        for name in VARIANTS:
            B.spmv_set_config(h, cfg_of(name))
            assert B.spmv_get_config(h).format == VARIANTS[name]["format"]
            assert rel_err(run(h, B.SPMV_F64, x, m=coo.m), want) <= 1e-13
    finally:
        B.spmv_destroy(h)


def test_config_defaults_resolve_per_format_and_value_type():
    """unroll/regcap 0 resolve per format and value type; out-of-family
    values are refused without changing the handle."""
    coo = matgen.laplacian_2d(32)
    want = {(B.SPMV_F64, B.FMT_ELL): (2, 32), (B.SPMV_F32, B.FMT_ELL): (4, 64), (B.SPMV_BF16, B.FMT_HYB): (4, 64),
            (B.SPMV_F64, B.FMT_SELL): (8, 64), (B.SPMV_F64, B.FMT_CSR): (2, 64), (B.SPMV_F32, B.FMT_COO): (2, 64)}
    for (vt, fmt), (u, rc) in want.items():
        h = create(coo, vt, B.make_config(format=fmt))
        try:
            c = B.spmv_get_config(h)
            assert (c.unroll, c.regcap) == (u, rc), (vt, fmt)
            for bad in (dict(format=B.FMT_CSR, regcap=48), dict(format=B.FMT_COO, unroll=8),
                        dict(format=fmt, regcap=40), dict(format=fmt, unroll=3),
                        dict(format=B.FMT_SELL, threads_per_row=2, unroll=8),
                        dict(format=B.FMT_SELL, threads_per_row=4), dict(format=B.FMT_ELL, threads_per_row=2)):
                with pytest.raises(B.SpmvError) as ei:
                    B.spmv_set_config(h, B.make_config(**bad))
                assert ei.value.status == -1
                assert B.spmv_get_config(h).format == fmt          # refused before any re-pack
        finally:
            B.spmv_destroy(h)


@pytest.mark.parametrize("vt", VTS)
def test_ell_column_offsets_16_bit_when_they_fit(vt):
    """bf16 ELL keeps 2-byte column offsets iff every |col - row| <= 32767
    (fp32/fp64 always int32): the format's byte count says which, and the
    exported columns are the same int32 layout either way."""
    import torch
    vs = {B.SPMV_F64: 8, B.SPMV_F32: 4, B.SPMV_BF16: 2}[vt]
    for case, fits in (("offset_32767", True), ("offset_32768", False)):
        coo = dict(EDGE)[case]
        h = create(coo, vt, cfg_of("ell"))
        try:
            info = B.spmv_get_info(h)
            w = info.ell_width
            col = _export(h, B.ARR_ELL_COLIDX, torch.int32).numpy()
        finally:
            B.spmv_destroy(h)
        p = col.size // w
        d16 = fits and vt == B.SPMV_BF16
        assert info.format_bytes == w * p * (vs + (2 if d16 else 4)), case
        got = {(int(r), int(c)) for k in range(w) for r, c in enumerate(col[k * p:(k + 1) * p]) if c >= 0}
        assert got == set(zip(coo.rows.tolist(), coo.cols.tolist())), case
