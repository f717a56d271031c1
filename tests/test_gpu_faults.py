"""Failure handling, driven from the host (no GPU fault, trap or hang).

* Allocation failure: with SPMV_FAULT_ALLOC=k the library's k-th device
  allocation inside an entry-point call fails as if the device were out of
  memory.  For every k up to the call's allocation count, the entry points
  must return SPMV_ERR_OOM and release everything they had allocated: the
  device's free memory returns to its value before the call (within the
  2 MiB granularity of the driver's accounting; the matrix is large enough
  that any leaked format array exceeds it), and the handle or plan stays
  usable afterwards.
* The device status word: a product on valid inputs leaves it clear, so
  spmv_check returns SPMV_OK after every kernel family.
"""
import os

import numpy as np
import pytest

from paper_2302_05662_gb300 import binding as B
from paper_2302_05662_gb300 import matgen

from gpu_util import create, oracle_for, rel_err, TOL

pytestmark = pytest.mark.gpu

MIB = 1 << 20
FORMATS = [
    ("csr", dict(format=B.FMT_CSR)),
    ("csr_split", dict(format=B.FMT_CSR, threads_per_row=B.TPR_SPLIT)),
    ("csr_tiles", dict(format=B.FMT_CSR, threads_per_row=B.TPR_SPLIT, hyb_ell_width=4096)),
    ("ell", dict(format=B.FMT_ELL)),
    ("coo", dict(format=B.FMT_COO)),
    ("hyb", dict(format=B.FMT_HYB)),
    ("bsr", dict(format=B.FMT_BSR)),
    ("sell", dict(format=B.FMT_SELL)),
]


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2302_05662_gb300 import build
    build.build()
    return B.load_library()


@pytest.fixture(scope="module")
def matrix():
    import torch
    coo = matgen.poisson_rows(1 << 18, 8.0, np.random.default_rng(3))   # ~2.1M nonzeros
    r = torch.from_numpy(coo.rows).cuda()
    c = torch.from_numpy(coo.cols).cuda()
    v = torch.from_numpy(coo.vals).cuda()
    return coo, r, c, v


def _free():
    import torch
    torch.cuda.synchronize()
    return torch.cuda.mem_get_info()[0]


def _with_fault(k, fn):
    os.environ["SPMV_FAULT_ALLOC"] = str(k)
    try:
        return fn()
    finally:
        del os.environ["SPMV_FAULT_ALLOC"]


@pytest.mark.parametrize("name", [f[0] for f in FORMATS])
def test_create_fails_cleanly_at_every_allocation(matrix, name):
    coo, r, c, v = matrix
    cfg = dict(FORMATS)[name]
    B.spmv_destroy(B.spmv_create(coo.m, coo.n, r, c, v, B.make_config(**cfg)))   # warm every path once
    free0 = _free()
    failures = 0
    for k in range(1, 200):
        try:
            h = _with_fault(k, lambda: B.spmv_create(coo.m, coo.n, r, c, v, B.make_config(**cfg)))
        except B.SpmvError as e:
            assert e.status == -2, (k, str(e))
            failures += 1
            assert abs(_free() - free0) <= 2 * MIB, f"allocation {k} failed and left memory behind"
            continue
        B.spmv_destroy(h)          # k is past the call's last allocation: it succeeded
        break
    else:
        pytest.fail("create never succeeded")
    assert failures >= 3
    assert abs(_free() - free0) <= 2 * MIB


def test_set_config_failure_leaves_a_usable_csr_handle(matrix, oracle):
    import torch
    coo, r, c, v = matrix
    h = B.spmv_create(coo.m, coo.n, r, c, v)
    try:
        x = torch.from_numpy(matgen.dense_vector(coo.n, 4)).cuda()
        want = oracle_for(oracle, coo, B.SPMV_F64, x.cpu().numpy())
        for name, cfg in FORMATS[1:]:
            with pytest.raises(B.SpmvError) as ei:
                _with_fault(1, lambda: B.spmv_set_config(h, B.make_config(**cfg)))
            assert ei.value.status == -2
            assert B.spmv_get_config(h).format == B.FMT_CSR         # fell back to CSR
            y = torch.zeros(coo.m, dtype=torch.float64, device="cuda")
            B.spmv_run(h, 1.0, x, 0.0, y)
            assert rel_err(y.cpu().numpy(), want) <= TOL[B.SPMV_F64], name
    finally:
        B.spmv_destroy(h)


def test_features_select_and_cg_fail_cleanly(oracle):
    import torch
    coo = matgen.laplacian_2d(256)
    h = create(coo, B.SPMV_F64)
    try:
        free0 = _free()
        with pytest.raises(B.SpmvError) as ei:
            _with_fault(1, lambda: B.spmv_features(h))
        assert ei.value.status == -2
        with pytest.raises(B.SpmvError) as ei:
            _with_fault(1, lambda: B.spmv_select(h))
        assert ei.value.status == -2
        assert abs(_free() - free0) <= 2 * MIB
        b = torch.from_numpy(matgen.dense_vector(coo.m, 5)).cuda()
        x = torch.zeros(coo.m, dtype=torch.float64, device="cuda")
        failures = 0
        for k in range(1, 40):     # the plan's device buffers, one by one
            try:
                _with_fault(k, lambda: B.spmv_cg(h, b, x, 0.0, 10))
            except B.SpmvError as e:
                assert e.status == -2, (k, str(e))
                failures += 1
                continue
            break
        assert failures >= 6
        x.zero_()
        res = B.spmv_cg(h, b, x, 0.0, 10)     # half-built plans were released: this one is whole
        ref = oracle.cg(coo.m, coo.rows, coo.cols, coo.vals, b.cpu().numpy(), tol=0.0, maxit=10)
        assert res.iterations == 10
        assert rel_err(x.cpu().numpy(), ref["x"]) <= 1e-10
    finally:
        B.spmv_destroy(h)


def test_batch_create_fails_cleanly():
    import torch
    hs, xs, ys = [], [], []
    for i, coo in matgen.batched_workload(6, 11):
        r = torch.from_numpy(coo.rows).cuda()
        c = torch.from_numpy(coo.cols).cuda()
        v = torch.from_numpy(coo.vals).cuda().float()
        hs.append(B.spmv_create(coo.m, coo.n, r, c, v))
        xs.append(torch.ones(coo.n, dtype=torch.float32, device="cuda"))
        ys.append(torch.zeros(coo.m, dtype=torch.float32, device="cuda"))
    ones, zeros = np.ones(len(hs)), np.zeros(len(hs))
    try:
        B.spmv_batch_destroy(B.spmv_batch_create(hs, ones, xs, zeros, ys))
        free0 = _free()
        for k in range(1, 40):
            try:
                bt = _with_fault(k, lambda: B.spmv_batch_create(hs, ones, xs, zeros, ys))
            except B.SpmvError as e:
                assert e.status == -2, (k, str(e))
                assert abs(_free() - free0) <= 2 * MIB
                continue
            B.spmv_batch_destroy(bt)
            break
        else:
            pytest.fail("batch create never succeeded")
    finally:
        for h in hs:
            B.spmv_destroy(h)


@pytest.mark.parametrize("name", [f[0] for f in FORMATS])
def test_status_word_stays_clear_on_valid_products(name):
    import torch
    coo = matgen.rmat(13, 16, np.random.default_rng(9))
    h = create(coo, B.SPMV_F64, B.make_config(**dict(FORMATS)[name]))
    try:
        x = torch.ones(coo.n, dtype=torch.float64, device="cuda")
        y = torch.zeros(coo.m, dtype=torch.float64, device="cuda")
        for _ in range(3):
            B.spmv_run(h, 1.0, x, 0.0, y)
        B.spmv_check(h)       # raises on a recorded timeout or bounds error
    finally:
        B.spmv_destroy(h)


CHECK_CASES = [("rmat", lambda: matgen.rmat(12, 16, np.random.default_rng(21))),
               ("banded", lambda: matgen.banded(6000, 32, np.random.default_rng(22)))]


@pytest.mark.parametrize("vt", [B.SPMV_F64, B.SPMV_BF16])
@pytest.mark.parametrize("case", [c[0] for c in CHECK_CASES])
@pytest.mark.parametrize("name", [f[0] for f in FORMATS])
def test_checked_products_equal_unchecked(name, case, vt):
    """SPMV_CHECKED=1: the index pass finds nothing on valid matrices (status
    word clear) and the product is bit-identical to the unchecked one
    (bf16 on the banded matrix exercises ELL's 16-bit column offsets)."""
    import torch
    from gpu_util import run
    coo = dict(CHECK_CASES)[case]()
    try:
        h = create(coo, vt, B.make_config(**dict(FORMATS)[name]))
    except B.SpmvError as e:
        assert e.status == -4          # a padded format over its storage limit
        return
    try:
        x = matgen.dense_vector(coo.n, 12)
        plain = run(h, vt, x, m=coo.m)
        checked = _with_checked(lambda: run(h, vt, x, m=coo.m))
        assert np.array_equal(plain, checked)
        B.spmv_check(h)
    finally:
        B.spmv_destroy(h)


def _with_checked(fn):
    os.environ["SPMV_CHECKED"] = "1"
    try:
        return fn()
    finally:
        del os.environ["SPMV_CHECKED"]


def test_parity_suite_passes_in_checked_mode():
    """The whole parity module again, every product preceded by the index
    pass (valid inputs only): every case must still match the oracle."""
    import subprocess
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(here, "test_gpu_parity.py"), "-q", "-x",
                        "-m", "gpu", "-p", "no:cacheprovider"],
                       env=dict(os.environ, SPMV_CHECKED="1"), capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
