"""Parity at the benchmark's full sizes and launch configurations: the five
format-sweep matrices (27-point stencil 128^3, Poisson(16) rows 2^20, R-MAT
scale 20, banded 2^20 half-width 32, block-diagonal 4x4 2^20), every kernel
variant the benchmark times, in fp64, fp32 and bf16, against the fp64 oracle
over all rows (the oracle is a single pass over the triplets)."""
import numpy as np
import pytest

from paper_2302_05662_gb300 import binding as B
from paper_2302_05662_gb300 import matgen
from paper_2302_05662_gb300.workload import SWEEP_VARIANTS

from gpu_util import TOL, VT_NAMES, create, oracle_for, rel_err, run

pytestmark = pytest.mark.gpu

NAMES = ["stencil27_128^3", "poisson16_2^20", "rmat_s20_ef16", "banded_2^20_w32", "blockdiag4_2^20"]


@pytest.fixture(scope="module", autouse=True)
def lib():
    from paper_2302_05662_gb300 import build
    build.build()
    return B.load_library()


@pytest.mark.parametrize("mname", NAMES)
def test_full_size_sweep(oracle, mname):
    coo = next(c for n, c in matgen.workload_matrices("full", only=mname))
    k = NAMES.index(mname)
    x = matgen.dense_vector(coo.n, 100 + k)       # the benchmark's x for this matrix
    failures = []
    for vt in (B.SPMV_F64, B.SPMV_F32, B.SPMV_BF16):
        want = oracle_for(oracle, coo, vt, x)
        for vname, kw in SWEEP_VARIANTS:
            try:
                h = create(coo, vt, B.make_config(**kw))
            except B.SpmvError as e:
                # ELL / BSR padded storage over the limit (R-MAT; BSR also Poisson rows)
                assert vname in ("ell", "bsr") and e.status == -4, str(e)
                continue
            try:
                got = run(h, vt, x, m=coo.m)
            finally:
                B.spmv_destroy(h)
            err = rel_err(got, want)
            if not err <= TOL[vt]:
                failures.append(f"{vname}/{VT_NAMES[vt]}: {err:.3e}")
    assert not failures, failures
