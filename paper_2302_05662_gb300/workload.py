"""The benchmark workload: which kernel variants the format sweep runs.

Kept in the package so that the benchmark and the full-size parity tests run
exactly the same launch configurations.
"""
from __future__ import annotations

from . import binding as B

# (name, spmv_config fields) of the format sweep over the five matrices
SWEEP_VARIANTS = (
    ("csr", dict(format=B.FMT_CSR)),                                  # vector CSR, tpr from mean row length
    ("csr_split", dict(format=B.FMT_CSR, threads_per_row=B.TPR_SPLIT)),  # nnz-balanced CSR: warp chunks
    ("csr_tiles", dict(format=B.FMT_CSR, threads_per_row=B.TPR_SPLIT, hyb_ell_width=4096)),  # staged tiles
    ("ell", dict(format=B.FMT_ELL)),
    ("coo", dict(format=B.FMT_COO)),
    ("hyb", dict(format=B.FMT_HYB)),
    ("bsr", dict(format=B.FMT_BSR)),
    ("sell", dict(format=B.FMT_SELL)),
)


def variant_config(name: str):
    for n, kw in SWEEP_VARIANTS:
        if n == name:
            return B.make_config(**kw)
    raise KeyError(name)
