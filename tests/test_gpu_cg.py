"""GPU parity of spmv_cg (conjugate gradients on the device, the repeated
SpMV setting of Section 7.5) against the oracle's CG.

CG iterates from the two sides differ only by the rounding of the dot
products (fixed-order fp64 tree on the device, exactly rounded on the CPU),
which CG amplifies slowly.  Bars: after a few iterations the iterate and the
rho history agree to 1e-10 (fp64); converged solutions agree to the accuracy
the tolerance implies; the true residual b - A x, formed by the oracle's
SpMV, meets the tolerance; iteration counts agree within one.
"""
import numpy as np
import pytest

from paper_2302_05662_gb300 import binding as B
from paper_2302_05662_gb300 import matgen
from paper_2302_05662_gb300.workload import SWEEP_VARIANTS

from gpu_util import create, rel_err, vec_dtype

pytestmark = pytest.mark.gpu
VARIANTS = dict(SWEEP_VARIANTS)


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2302_05662_gb300 import build
    build.build()
    return B.load_library()


def spd_random(n, per_row, seed):
    """Symmetric, strictly diagonally dominant (so positive definite) matrix
    with about 2*per_row random off-diagonal entries per row."""
    rng = np.random.default_rng(seed)
    r = rng.integers(0, n, n * per_row)
    c = rng.integers(0, n, n * per_row)
    keep = r != c
    r, c = r[keep], c[keep]
    key = np.unique(np.minimum(r, c).astype(np.int64) * n + np.maximum(r, c))
    lo, hi = key // n, key % n
    v = rng.uniform(-1, 1, key.size)
    rows = np.concatenate([lo, hi, np.arange(n)])
    cols = np.concatenate([hi, lo, np.arange(n)])
    dom = np.zeros(n)
    np.add.at(dom, lo, np.abs(v))
    np.add.at(dom, hi, np.abs(v))
    vals = np.concatenate([v, v, dom + 1.0])
    return matgen.Coo(n, n, rows.astype(np.int32), cols.astype(np.int32), vals)


MATS = {
    "lap2d_32": lambda: matgen.laplacian_2d(32),
    "stencil27_16": lambda: matgen.stencil_3d(16, 27, values="laplace"),
    "spd_random_3000": lambda: spd_random(3000, 6, 1),
}


def dev(v, vt=B.SPMV_F64):
    import torch
    return torch.from_numpy(np.ascontiguousarray(v)).to(vec_dtype(vt)).cuda()


def solve(h, b, x0, tol, maxit, vt=B.SPMV_F64):
    import torch
    bt, xt = dev(b, vt), dev(x0, vt)
    rho = torch.full((maxit + 1,), float("nan"), dtype=torch.float64, device="cuda")
    res = B.spmv_cg(h, bt, xt, tol, maxit, rho)
    torch.cuda.synchronize()
    return xt.cpu().double().numpy(), rho.cpu().numpy()[:res.iterations + 1], res


def ocg(oracle, coo, b, x0, tol, maxit):
    return oracle.cg(coo.m, coo.rows, coo.cols, coo.vals, b, x0=x0, tol=tol, maxit=maxit)


@pytest.mark.parametrize("fmt", [n for n, _ in SWEEP_VARIANTS])
@pytest.mark.parametrize("name", sorted(MATS))
def test_iterates_match_oracle(oracle, name, fmt):
    coo = MATS[name]()
    b = matgen.dense_vector(coo.m, 21)
    x0 = matgen.dense_vector(coo.m, 22)
    h = create(coo, B.SPMV_F64, B.make_config(**VARIANTS[fmt]))
    try:
        for k in (1, 2, 8):
            x, rho, res = solve(h, b, x0, 0.0, k)
            want = ocg(oracle, coo, b, x0, 0.0, k)
            assert res.iterations == k == want["iterations"]
            assert not res.breakdown
            assert rel_err(x, want["x"]) <= 1e-10
            np.testing.assert_allclose(rho, want["rho"], rtol=1e-10)
        # to convergence
        x, rho, res = solve(h, b, x0, 1e-10, 2000)
        want = ocg(oracle, coo, b, x0, 1e-10, 2000)
    finally:
        B.spmv_destroy(h)
    assert res.converged and want["converged"]
    assert abs(res.iterations - want["iterations"]) <= 1
    assert rel_err(x, want["x"]) <= 1e-7
    assert res.rho == rho[-1] and res.rho0 == rho[0]
    assert res.bb == pytest.approx(float(b @ b), rel=1e-13)
    r_true = b - oracle.spmv_coo(coo.m, coo.n, coo.rows, coo.cols, coo.vals, x)
    assert np.linalg.norm(r_true) <= 1.5e-10 * np.linalg.norm(b)


def test_repeat_solves_bit_identical():
    coo = MATS["stencil27_16"]()
    b = matgen.dense_vector(coo.m, 3)
    h = create(coo, B.SPMV_F64, B.make_config(format=B.FMT_COO))
    try:
        x1, rho1, r1 = solve(h, b, np.zeros(coo.m), 1e-9, 500)
        x2, rho2, r2 = solve(h, b, np.zeros(coo.m), 1e-9, 500)   # same plan, replayed
        b2 = np.array(b)
        x3, rho3, r3 = solve(h, b2, np.zeros(coo.m), 1e-9, 500)  # new buffers: plan rebuilt
    finally:
        B.spmv_destroy(h)
    assert r1.iterations == r2.iterations == r3.iterations
    assert np.array_equal(x1, x2) and np.array_equal(x1, x3)
    assert np.array_equal(rho1, rho2) and np.array_equal(rho1, rho3)


def test_plan_follows_set_config(oracle):
    coo = MATS["lap2d_32"]()
    b = matgen.dense_vector(coo.m, 4)
    h = create(coo, B.SPMV_F64)
    try:
        xa, _, ra = solve(h, b, np.zeros(coo.m), 1e-10, 1000)
        B.spmv_set_config(h, B.make_config(format=B.FMT_ELL, threads_per_block=128))
        xb, _, rb = solve(h, b, np.zeros(coo.m), 1e-10, 1000)
    finally:
        B.spmv_destroy(h)
    assert ra.converged and rb.converged
    assert rel_err(xb, xa) <= 1e-8
    r_true = b - oracle.spmv_coo(coo.m, coo.n, coo.rows, coo.cols, coo.vals, xb)
    assert np.linalg.norm(r_true) <= 1.5e-10 * np.linalg.norm(b)


def test_fp32_converges_to_its_precision(oracle):
    coo = MATS["stencil27_16"]()
    b = matgen.dense_vector(coo.m, 5)
    for vt in (B.SPMV_F32, B.SPMV_BF16):
        h = create(coo, vt, B.make_config(format=B.FMT_ELL))
        try:
            x, rho, res = solve(h, b, np.zeros(coo.m), 1e-4, 500, vt)
        finally:
            B.spmv_destroy(h)
        assert res.converged and not res.breakdown and res.iterations < 500
        # the Laplacian's values (26, -1) are exact in bf16 and fp32
        r_true = matgen.round_to_f32(b) - oracle.spmv_coo(coo.m, coo.n, coo.rows, coo.cols, coo.vals, x)
        assert np.linalg.norm(r_true) <= 2e-4 * np.linalg.norm(b)


def test_breakdown_on_indefinite_matrix():
    i = np.arange(2, dtype=np.int32)
    coo = matgen.Coo(2, 2, i, i.copy(), np.array([1.0, -1.0]))
    h = create(coo, B.SPMV_F64)
    try:
        x, rho, res = solve(h, np.array([1.0, 1.0]), np.zeros(2), 1e-12, 10)
    finally:
        B.spmv_destroy(h)
    assert res.breakdown and not res.converged and res.iterations == 0
    assert np.array_equal(x, [0.0, 0.0]) and rho.tolist() == [2.0]


def test_zero_rhs_maxit_zero_and_exact_start():
    coo = matgen.laplacian_1d(50)
    h = create(coo, B.SPMV_F64)
    try:
        x, rho, res = solve(h, np.zeros(50), np.zeros(50), 1e-8, 100)
        assert res.iterations == 0 and res.converged and rho.tolist() == [0.0]
        b = matgen.dense_vector(50, 1)
        x, rho, res = solve(h, b, np.zeros(50), 1e-8, 0)
        assert res.iterations == 0 and not res.converged
        assert rho[0] == pytest.approx(float(b @ b), rel=1e-14) and np.array_equal(x, np.zeros(50))
        xs = np.arange(1.0, 51.0)
        A = np.zeros((50, 50))
        A[coo.rows, coo.cols] = coo.vals
        x, rho, res = solve(h, A @ xs, xs, 1e-8, 100)
        assert res.iterations == 0 and res.converged and np.array_equal(x, xs)
    finally:
        B.spmv_destroy(h)


def test_invalid_arguments_rejected():
    import torch
    rect = matgen.random_coo(5, 7, 10, np.random.default_rng(0))
    h = create(rect, B.SPMV_F64)
    try:
        v = torch.zeros(7, dtype=torch.float64, device="cuda")
        with pytest.raises(B.SpmvError) as ei:
            B.spmv_cg(h, v, v.clone(), 1e-8, 10)
        assert ei.value.status == -1
    finally:
        B.spmv_destroy(h)
    coo = matgen.laplacian_1d(8)
    h = create(coo, B.SPMV_F64)
    try:
        b = torch.ones(8, dtype=torch.float64, device="cuda")
        x = torch.zeros(8, dtype=torch.float64, device="cuda")
        for tol, maxit in ((-1.0, 10), (float("nan"), 10), (float("inf"), 10), (1e-8, -1),
                           (1e-8, B.CG_MAX_ITERATIONS + 1)):
            with pytest.raises(B.SpmvError) as ei:
                B.spmv_cg(h, b, x, tol, maxit)
            assert ei.value.status == -1
        res = B.spmv_cg(h, b, x, 1e-12, 100)       # the handle still works
        assert res.converged
    finally:
        B.spmv_destroy(h)


def test_fullsize_stencil27_selected_config(oracle):
    """27-point Laplacian 128^3 (centre 26, neighbours -1), the selector's
    configuration, to 1e-8: the true residual from the oracle's SpMV."""
    from paper_2302_05662_gb300 import selector as S
    coo = matgen.stencil_3d(128, 27, values="laplace")
    b = matgen.dense_vector(coo.m, 9)
    h = create(coo, B.SPMV_F64)
    try:
        S.load_default_selector()
        cfg, _ = B.spmv_select(h)
        B.spmv_set_config(h, cfg)
        x, rho, res = solve(h, b, np.zeros(coo.m), 1e-8, 2000)
    finally:
        B.spmv_destroy(h)
        B.spmv_selector_unload()
    assert res.converged and 10 < res.iterations < 2000
    assert rho[-1] <= 1e-16 * res.bb < rho[-2]
    r_true = b - oracle.spmv_coo(coo.m, coo.n, coo.rows, coo.cols, coo.vals, x)
    assert np.linalg.norm(r_true) <= 1.5e-8 * np.linalg.norm(b)
