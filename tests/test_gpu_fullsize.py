"""Parity at the benchmark's full sizes and launch configurations: the five
format-sweep matrices (27-point stencil 128^3, Poisson(16) rows 2^20, R-MAT
scale 20, banded 2^20 half-width 32, block-diagonal 4x4 2^20), every kernel
variant of the sweep at its default configuration plus the configuration
the selector picks (the one bench.py times), in fp64, fp32 and bf16, against
the fp64 oracle over all rows (the oracle is one pass over the triplets).

With SPMV_ERROR_REPORT=<path> the normwise error of every result is
appended to that file as JSON lines."""
import json
import os

import numpy as np
import pytest

from paper_2302_05662_gb300 import binding as B
from paper_2302_05662_gb300 import matgen
from paper_2302_05662_gb300 import selector as S
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
    report = os.environ.get("SPMV_ERROR_REPORT")
    have_sel = os.path.exists(S.DEFAULT_BLOB)
    if have_sel:
        S.load_default_selector()
    failures, records = [], []
    for vt in (B.SPMV_F64, B.SPMV_F32, B.SPMV_BF16):
        want = oracle_for(oracle, coo, vt, x)
        want64 = oracle.spmv_coo_obj(coo, x) if vt != B.SPMV_F64 else want
        variants = [(n, B.make_config(**kw)) for n, kw in SWEEP_VARIANTS]
        if have_sel:
            h = create(coo, vt)
            try:
                sel, _ = B.spmv_select(h)
            finally:
                B.spmv_destroy(h)
            variants.append(("selected", sel))
        for vname, cfg in variants:
            try:
                h = create(coo, vt, cfg)
            except B.SpmvError as e:
                # ELL / BSR padded storage over the limit (R-MAT; BSR also Poisson rows)
                assert cfg.format in (B.FMT_ELL, B.FMT_BSR, B.FMT_SELL) and e.status == -4, str(e)
                continue
            try:
                got = run(h, vt, x, m=coo.m)
            finally:
                B.spmv_destroy(h)
            err = rel_err(got, want)
            records.append({"matrix": mname, "kernel": vname, "format": int(cfg.format),
                            "dtype": VT_NAMES[vt], "err_vs_oracle_on_device_inputs": err,
                            "err_vs_fp64_oracle_original_inputs": rel_err(got, want64)})
            if not err <= TOL[vt]:
                failures.append(f"{vname}/{VT_NAMES[vt]}: {err:.3e}")
    if report:
        with open(report, "a") as fh:
            for r in records:
                fh.write(json.dumps(r) + "\n")
    assert not failures, failures
