"""Seeded input generators: structure, sizes and value rounding."""
import numpy as np
import pytest

from paper_2302_05662_gb300 import matgen


def _sorted_unique(coo):
    key = coo.rows.astype(np.int64) * coo.n + coo.cols
    return bool(np.all(np.diff(key) > 0))


@pytest.mark.parametrize("fam", matgen.FAMILIES)
def test_families_sorted_unique_in_range(fam):
    for seed in range(3):
        coo = matgen.family_matrix(fam, 3000, seed, jitter=True)
        assert coo.nnz > 0 and _sorted_unique(coo)
        assert coo.rows.min() >= 0 and coo.rows.max() < coo.m
        assert coo.cols.min() >= 0 and coo.cols.max() < coo.n


def test_seeded_reproducible():
    a = matgen.family_matrix("rmat", 5000, 3)
    b = matgen.family_matrix("rmat", 5000, 3)
    assert np.array_equal(a.cols, b.cols) and np.array_equal(a.vals, b.vals)


def test_rmat_power_law_and_poisson_mean():
    r = matgen.rmat(14, 16, np.random.default_rng(0))
    lens = np.bincount(r.rows, minlength=r.m)
    assert lens.max() > 20 * lens.mean()          # heavy head
    assert (lens == 0).mean() > 0.05               # many empty rows
    p = matgen.poisson_rows(1 << 14, 16.0, np.random.default_rng(0))
    assert abs(p.nnz / p.m - 16.0) < 0.2


def test_small_workload_shapes():
    names = [n for n, _ in matgen.workload_matrices("small")]
    assert len(names) == 5


def test_bf16_rounding_ties_to_even():
    v = np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 / 3.0, -2.5,
                  1.0 + 2.0 ** -8 + 2.0 ** -30])
    r = matgen.round_to_bf16(v)
    assert r[0] == 1.0                              # tie -> even (down)
    assert r[1] == 1.0 + 2.0 ** -6                  # tie -> even (up)
    assert matgen.bf16_bits(r)[2] == 0x3EAB         # 1/3 in bf16
    assert r[3] == -2.5
    assert r[4] == 1.0 + 2.0 ** -7                  # just above the tie
    assert np.array_equal(matgen.round_to_f32(np.array([0.1])),
                          np.array([np.float32(0.1)], dtype=np.float64))


def test_batched_workload_families_sizes_and_seeds():
    """The batch cycles through the families with n log-uniform in
    [10^3, 2*10^5] (after each family's snapping) and is reproducible."""
    import itertools
    first = list(itertools.islice(matgen.batched_workload(), 10))
    again = list(itertools.islice(matgen.batched_workload(), 10))
    for (i, a), (j, b) in zip(first, again):
        assert i == j and a.name == b.name and np.array_equal(a.cols, b.cols) and np.array_equal(a.vals, b.vals)
    for i, coo in first:
        assert coo.name == f"batch{i}_{matgen.FAMILIES[i % 5]}"
        assert 500 <= coo.m <= 300_000 and coo.nnz > 0 and _sorted_unique(coo)
    assert len(list(itertools.islice(matgen.batched_workload(count=3), 10))) == 3


def test_column_contiguity_separates_scattered_from_banded_families():
    """The fp64 SELL layout default takes column-major when fewer than a
    quarter of consecutive stored entries have consecutive columns: on the
    generated families that threshold puts Poisson rows and R-MAT below and
    every stencil (5-, 7-, 27-point), band and block-diagonal above."""
    def contig(coo):
        o = np.lexsort((coo.cols, coo.rows))
        c = coo.cols[o].astype(np.int64)
        return float(np.mean(c[1:] == c[:-1] + 1))
    for fam in matgen.FAMILIES:
        for seed in range(4):
            f = contig(matgen.family_matrix(fam, 20000, seed=seed, jitter=True))
            if fam in ("poisson", "rmat"):
                assert f < 0.2, (fam, seed, f)
            else:
                assert f > 0.27, (fam, seed, f)
