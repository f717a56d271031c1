"""spmv_coo_run_noalloc: the COO product for callers that cannot allocate
device memory (code inside another library's memory pool or callback,
real-time code that may not allocate after start-up, processes whose
allocator is exhausted).  Its scratch is the library's fixed device array,
so these tests make two calls in a row -- the second reuses the array the
first one left behind -- and check both against the fp64 oracle: bit-exact
on integer-valued inputs, within the normwise tolerances of the other parity
tests otherwise.  They also check that a call after the first leaves the
device's free memory unchanged, the largest accepted size, the empty cases,
and the refusals (oversize, unsorted, misaligned, capturing stream).  This
file is collected last."""
import numpy as np
import pytest

from paper_2302_05662_gb300 import binding as B
from paper_2302_05662_gb300 import matgen

from gpu_util import TOL, device_values, oracle_for, rel_err, stored_vector, vec_dtype

pytestmark = pytest.mark.gpu

VTS = [B.SPMV_F64, B.SPMV_F32, B.SPMV_BF16]


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2302_05662_gb300 import build
    build.build()
    return B.load_library()


def _int_valued(coo, seed):
    """Same pattern with small integer values (exact in every value type,
    and every partial sum exact in fp32)."""
    rng = np.random.default_rng(seed)
    v = rng.integers(-4, 5, coo.nnz).astype(np.float64)
    return matgen.Coo(coo.m, coo.n, coo.rows, coo.cols, v)


CASES = [
    ("rmat", lambda: matgen.rmat(14, 16, np.random.default_rng(5))),
    ("stencil", lambda: matgen.stencil_3d(24, 27, np.random.default_rng(6))),
    ("one_long_row", lambda: matgen.Coo(3, 9000, np.full(9000, 1, np.int32), np.arange(9000, dtype=np.int32),
                                        np.random.default_rng(7).standard_normal(9000))),
    ("empty_rows", lambda: matgen.random_coo(5000, 300, 700, np.random.default_rng(8))),
    ("rmat_int", lambda: _int_valued(matgen.rmat(13, 16, np.random.default_rng(9)), 10)),
    ("poisson_int", lambda: _int_valued(matgen.poisson_rows(20000, 12.0, np.random.default_rng(11)), 12)),
]
INTEGER_CASES = ("rmat_int", "poisson_int")


def _vectors(coo, integer):
    if integer:
        rng = np.random.default_rng(13)
        return rng.integers(-4, 5, coo.n).astype(np.float64), rng.integers(-4, 5, coo.m).astype(np.float64)
    return matgen.dense_vector(coo.n, 3), matgen.dense_vector(coo.m, 4)


def _call(coo, rows, cols, vals, vt, x, alpha, beta, y0):
    import torch
    y = torch.from_numpy(stored_vector(y0, vt)).to(vec_dtype(vt)).cuda()
    B.spmv_coo_run_noalloc(coo.m, coo.n, rows, cols, vals, alpha, x, beta, y)
    torch.cuda.synchronize()
    return y.cpu().double().numpy()


@pytest.mark.parametrize("vt", VTS)
@pytest.mark.parametrize("case", [c[0] for c in CASES])
def test_noalloc_matches_oracle_twice(oracle, case, vt):
    import torch
    coo = dict(CASES)[case]()
    integer = case in INTEGER_CASES
    rows = torch.from_numpy(coo.rows).cuda()
    cols = torch.from_numpy(coo.cols).cuda()
    vals = device_values(coo.vals, vt)
    x_np, y0 = _vectors(coo, integer)
    x = torch.from_numpy(stored_vector(x_np, vt)).to(vec_dtype(vt)).cuda()
    for alpha, beta in ((1.0, 0.0), (0.5, -2.0)):
        want = oracle_for(oracle, coo, vt, x_np, alpha, beta, y0)
        for _ in range(2):     # the second call reuses the fixed scratch array
            got = _call(coo, rows, cols, vals, vt, x, alpha, beta, y0)
            if integer:
                assert np.array_equal(got, want)
            else:
                err = rel_err(got, want)
                assert err <= TOL[vt], f"normwise error {err:.3e}"


def test_noalloc_second_call_allocates_nothing(oracle):
    import torch
    coo = matgen.rmat(14, 16, np.random.default_rng(21))
    rows = torch.from_numpy(coo.rows).cuda()
    cols = torch.from_numpy(coo.cols).cuda()
    vals = device_values(coo.vals, B.SPMV_F64)
    x = torch.from_numpy(matgen.dense_vector(coo.n, 22)).cuda()
    y = torch.zeros(coo.m, dtype=torch.float64, device="cuda")
    B.spmv_coo_run_noalloc(coo.m, coo.n, rows, cols, vals, 1.0, x, 0.0, y)    # first call: set-up
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    B.spmv_coo_run_noalloc(coo.m, coo.n, rows, cols, vals, 1.0, x, 0.0, y)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    want = oracle.spmv_coo(coo.m, coo.n, coo.rows, coo.cols, coo.vals, x.cpu().numpy())
    assert rel_err(y.cpu().numpy(), want) <= TOL[B.SPMV_F64]


def test_noalloc_at_the_size_limit(oracle):
    """Exactly SPMV_NOALLOC_MAX_NNZ triplets (the fixed array's last chunk
    and bound): 2^20 rows of 32 entries, integer values, every value type
    bit-exact against the oracle."""
    import torch
    m = n = 1 << 20
    w = B.NOALLOC_MAX_NNZ // m
    assert w * m == B.NOALLOC_MAX_NNZ
    r = np.repeat(np.arange(m, dtype=np.int32), w)
    c = ((r.astype(np.int64) + np.tile(np.arange(w, dtype=np.int64) * 97 - 1500, m)) % n).astype(np.int32)
    rng = np.random.default_rng(31)
    v = rng.integers(-4, 5, r.size).astype(np.float64)
    coo = matgen.Coo(m, n, r, c, v)
    x_np = rng.integers(-4, 5, n).astype(np.float64)
    want = oracle.spmv_coo(m, n, r, c, v, x_np)
    rows = torch.from_numpy(r).cuda()
    cols = torch.from_numpy(c).cuda()
    for vt in VTS:
        vals = device_values(v, vt)
        x = torch.from_numpy(x_np).to(vec_dtype(vt)).cuda()
        for _ in range(2):
            got = _call(coo, rows, cols, vals, vt, x, 1.0, 0.0, np.zeros(m))
            assert np.array_equal(got, want)
        del vals


def test_noalloc_empty_cases(oracle):
    import torch
    e = torch.zeros(0, dtype=torch.int32, device="cuda")
    ev = torch.zeros(0, dtype=torch.float64, device="cuda")
    # nnz = 0: y <- beta y (beta = 0 writes zeros without reading y)
    y0 = matgen.dense_vector(700, 41)
    y = torch.from_numpy(y0).cuda()
    x = torch.ones(5, dtype=torch.float64, device="cuda")
    B.spmv_coo_run_noalloc(700, 5, e, e, ev, 1.0, x, -1.5, y)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), oracle.spmv_coo(700, 5, [], [], [], np.ones(5), 1.0, -1.5, y0))
    y.fill_(float("nan"))
    B.spmv_coo_run_noalloc(700, 5, e, e, ev, 1.0, x, 0.0, y)
    torch.cuda.synchronize()
    assert np.array_equal(y.cpu().numpy(), np.zeros(700))
    # m = 0: nothing to write
    y = torch.zeros(0, dtype=torch.float64, device="cuda")
    B.spmv_coo_run_noalloc(0, 5, e, e, ev, 1.0, x, 0.0, y)
    torch.cuda.synchronize()


def test_noalloc_rejects_oversize_and_unsorted():
    import torch
    r = torch.tensor([1, 0], dtype=torch.int32, device="cuda")
    c = torch.tensor([0, 0], dtype=torch.int32, device="cuda")
    v = torch.ones(2, dtype=torch.float64, device="cuda")
    x = torch.ones(2, dtype=torch.float64, device="cuda")
    y = torch.full((2,), 7.0, dtype=torch.float64, device="cuda")
    with pytest.raises(B.SpmvError) as ei:        # rows out of order
        B.spmv_coo_run_noalloc(2, 2, r, c, v, 1.0, x, 0.0, y)
    assert ei.value.status == -1
    assert torch.equal(y, torch.full((2,), 7.0, dtype=torch.float64, device="cuda"))
    lib = B.load_library()
    big = B.NOALLOC_MAX_NNZ + 1        # refused on the host before any device access
    rc = lib.spmv_coo_run_noalloc(4, 4, big, r.data_ptr(), c.data_ptr(), v.data_ptr(), B.SPMV_F64, 1.0,
                                  x.data_ptr(), 0.0, y.data_ptr(), None)
    assert rc == -4 and "scratch limit" in B.spmv_last_error()


def test_noalloc_rejects_misaligned_triplets():
    """A view that starts 4 bytes into an array is refused on the host
    (SPMV_ERR_INVALID) before any launch; y keeps its contents."""
    import torch
    r = torch.arange(65, dtype=torch.int32, device="cuda")
    c = torch.arange(65, dtype=torch.int32, device="cuda")
    v = torch.ones(65, dtype=torch.float64, device="cuda")
    x = torch.ones(65, dtype=torch.float64, device="cuda")
    y = torch.full((65,), 7.0, dtype=torch.float64, device="cuda")
    lib = B.load_library()
    for rr, cc, vv in ((r[1:], c[:-1], v[:-1]), (r[:-1], c[1:], v[:-1]), (r[:-1], c[:-1], v[1:])):
        rc = lib.spmv_coo_run_noalloc(65, 65, 64, rr.data_ptr(), cc.data_ptr(), vv.data_ptr(), B.SPMV_F64, 1.0,
                                      x.data_ptr(), 0.0, y.data_ptr(), None)
        assert rc == -1 and "aligned" in B.spmv_last_error()
    torch.cuda.synchronize()
    assert torch.equal(y, torch.full((65,), 7.0, dtype=torch.float64, device="cuda"))


def test_noalloc_refuses_a_capturing_stream():
    """The call waits on its stream, so a stream being captured into a graph
    is refused before anything is enqueued; the capture stays valid."""
    import torch
    r = torch.arange(8, dtype=torch.int32, device="cuda")
    v = torch.ones(8, dtype=torch.float64, device="cuda")
    x = torch.ones(8, dtype=torch.float64, device="cuda")
    y = torch.full((8,), 7.0, dtype=torch.float64, device="cuda")
    z = torch.zeros(1, dtype=torch.float64, device="cuda")
    lib = B.load_library()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        rc = lib.spmv_coo_run_noalloc(8, 8, 8, r.data_ptr(), r.data_ptr(), v.data_ptr(), B.SPMV_F64, 1.0,
                                      x.data_ptr(), 0.0, y.data_ptr(), torch.cuda.current_stream().cuda_stream)
        z.add_(1.0)
    assert rc == -4 and "captured" in B.spmv_last_error()
    g.replay()
    torch.cuda.synchronize()
    assert z.item() == 1.0
    assert torch.equal(y, torch.full((8,), 7.0, dtype=torch.float64, device="cuda"))
