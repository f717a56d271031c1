"""spmv_coo_run_noalloc: the COO product for callers that cannot allocate
device memory (code inside another library's pool or callback, real-time
code that may not allocate after start-up, processes whose allocator is
exhausted).  Its scratch is the library's fixed device array, so these tests
check that two calls in a row -- which reuse that array -- both match the
regular entry point (spmv_create in COO format + spmv_run), within the
tolerances the other parity tests use.  This file is collected last."""
import numpy as np
import pytest

from paper_2302_05662_gb300 import binding as B
from paper_2302_05662_gb300 import matgen

from gpu_util import TOL, create, device_values, vec_dtype

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2302_05662_gb300 import build
    build.build()
    return B.load_library()


def _regular(coo, vt, x, alpha, beta, y0):
    import torch
    h = create(coo, vt, B.make_config(format=B.FMT_COO))
    try:
        y = torch.from_numpy(y0).to(vec_dtype(vt)).cuda()
        B.spmv_run(h, alpha, x, beta, y)
        torch.cuda.synchronize()
        return y.cpu().double().numpy()
    finally:
        B.spmv_destroy(h)


CASES = [
    ("rmat", lambda: matgen.rmat(14, 16, np.random.default_rng(5))),
    ("stencil", lambda: matgen.stencil_3d(24, 27, np.random.default_rng(6))),
    ("one_long_row", lambda: matgen.Coo(3, 9000, np.full(9000, 1, np.int32), np.arange(9000, dtype=np.int32),
                                        np.random.default_rng(7).standard_normal(9000))),
    ("empty_rows", lambda: matgen.random_coo(5000, 300, 700, np.random.default_rng(8))),
]


@pytest.mark.parametrize("vt", [B.SPMV_F64, B.SPMV_F32, B.SPMV_BF16])
@pytest.mark.parametrize("case", [c[0] for c in CASES])
def test_noalloc_matches_regular_entry_point_twice(case, vt):
    import torch
    coo = dict(CASES)[case]()
    rows = torch.from_numpy(coo.rows).cuda()
    cols = torch.from_numpy(coo.cols).cuda()
    vals = device_values(coo.vals, vt)
    x = torch.from_numpy(matgen.dense_vector(coo.n, 3)).to(vec_dtype(vt)).cuda()
    y0 = matgen.dense_vector(coo.m, 4)
    for alpha, beta in ((1.0, 0.0), (0.5, -2.0)):
        want = _regular(coo, vt, x, alpha, beta, y0)
        for _ in range(2):     # the second call reuses the fixed scratch array
            y = torch.from_numpy(y0).to(vec_dtype(vt)).cuda()
            B.spmv_coo_run_noalloc(coo.m, coo.n, rows, cols, vals, alpha, x, beta, y)
            torch.cuda.synchronize()
            got = y.cpu().double().numpy()
            err = np.linalg.norm(got - want) / max(np.linalg.norm(want), 1e-300)
            assert err <= TOL[vt], f"normwise difference {err:.3e}"


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
