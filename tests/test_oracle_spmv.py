"""Pins for the fp64 SpMV oracle (Section 2.2: Y = A X, with alpha/beta).

Each test checks the oracle against something other than itself: dense
brute force, exact closed forms (Laplacian eigenpairs), identity and
permutation matrices, exactly-rounded sums.  A dropped term, a wrong sign,
a swapped row/column index or a transposed operand fails at least one.
"""
import math

import numpy as np
import pytest

from paper_2302_05662_gb300 import matgen


def dense_of(m, n, rows, cols, vals):
    A = np.zeros((m, n))
    np.add.at(A, (rows.astype(np.int64), cols.astype(np.int64)), vals)
    return A


@pytest.mark.parametrize("seed", range(6))
def test_dense_bruteforce_integer_exact(oracle, seed):
    rng = np.random.default_rng(seed)
    m, n = int(rng.integers(1, 65)), int(rng.integers(1, 65))
    coo = matgen.random_coo(m, n, int(rng.integers(0, m * n + 1)), rng,
                            integer_values=8)
    x = matgen.dense_vector(n, seed + 100, integer_values=8)
    y = matgen.dense_vector(m, seed + 200, integer_values=8)
    A = dense_of(m, n, coo.rows, coo.cols, coo.vals)
    for alpha, beta in ((1.0, 0.0), (3.0, -2.0), (-1.0, 1.0)):
        got = oracle.spmv_coo_obj(coo, x, alpha, beta, y)
        want = alpha * (A @ x) + beta * y
        assert np.array_equal(got, want)


def test_rectangular_not_transposed(oracle):
    # m != n and a non-symmetric pattern: a transposed operand changes shape
    rng = np.random.default_rng(7)
    coo = matgen.random_coo(5, 9, 20, rng, integer_values=5)
    x = matgen.dense_vector(9, 1, integer_values=5)
    got = oracle.spmv_coo_obj(coo, x)
    assert got.shape == (5,)
    assert np.array_equal(got, dense_of(5, 9, coo.rows, coo.cols, coo.vals) @ x)


@pytest.mark.parametrize("seed", range(3))
def test_dense_bruteforce_real(oracle, seed):
    rng = np.random.default_rng(seed)
    m, n = 50, 40
    coo = matgen.random_coo(m, n, 600, rng)
    x = matgen.dense_vector(n, seed)
    y = matgen.dense_vector(m, seed + 1)
    got = oracle.spmv_coo_obj(coo, x, 0.75, -1.25, y)
    want = 0.75 * (dense_of(m, n, coo.rows, coo.cols, coo.vals) @ x) - 1.25 * y
    assert np.linalg.norm(got - want) <= 1e-14 * np.linalg.norm(want)


def test_row_sums(oracle):
    rng = np.random.default_rng(3)
    coo = matgen.random_coo(300, 200, 4000, rng, integer_values=100)
    got = oracle.spmv_coo_obj(coo, np.ones(200))
    want = np.bincount(coo.rows, weights=coo.vals, minlength=300)
    assert np.array_equal(got, want)


def test_identity_bit_exact(oracle):
    n = 1000
    idx = np.arange(n, dtype=np.int32)
    x = matgen.dense_vector(n, 11)
    y = matgen.dense_vector(n, 12)
    alpha, beta = 0.3, 1.7
    got = oracle.spmv_coo(n, n, idx, idx, np.ones(n), x, alpha, beta, y)
    assert np.array_equal(got, alpha * x + beta * y)


def test_permutation_bit_exact(oracle):
    n = 777
    pi = np.random.default_rng(5).permutation(n).astype(np.int32)
    x = matgen.dense_vector(n, 13)
    got = oracle.spmv_coo(n, n, np.arange(n, dtype=np.int32), pi, np.ones(n),
                          x, -2.5)
    assert np.array_equal(got, -2.5 * x[pi])


def test_unsorted_and_duplicate_triplets(oracle):
    rng = np.random.default_rng(9)
    coo = matgen.random_coo(40, 30, 500, rng, duplicates=True, shuffle=True,
                            integer_values=6)
    x = matgen.dense_vector(30, 4, integer_values=6)
    got = oracle.spmv_coo_obj(coo, x)
    assert np.array_equal(got, dense_of(40, 30, coo.rows, coo.cols, coo.vals) @ x)


@pytest.mark.parametrize("N", [1, 2, 17, 300])
def test_laplacian_1d_sine_modes(oracle, N):
    """tridiag(-1,2,-1) v_j = 4 sin^2(j pi / (2(N+1))) v_j,
    v_j(i) = sin(i j pi/(N+1)), i = 1..N."""
    coo = matgen.laplacian_1d(N)
    i = np.arange(1, N + 1)
    for j in sorted({1, 2, max(1, N // 2), N}):
        # reduce i*j exactly modulo the period 2(N+1) before scaling by pi
        v = np.sin(((i * j) % (2 * (N + 1))) * np.pi / (N + 1))
        lam = 4.0 * np.sin(j * np.pi / (2 * (N + 1))) ** 2
        got = oracle.spmv_coo_obj(coo, v)
        assert np.max(np.abs(got - lam * v)) <= 1e-13


def test_laplacian_2d_sine_modes_and_size(oracle):
    """5-point Dirichlet Laplacian on 64x64: nnz = 5*4096 - 4*64 = 20224 and
    A (sin(a p pi/(N+1)) sin(b q pi/(N+1))) = (4 - 2cos(p pi/(N+1))
    - 2cos(q pi/(N+1))) times the same grid function."""
    N = 64
    coo = matgen.laplacian_2d(N)
    assert coo.m == 4096 and coo.nnz == 5 * 4096 - 4 * 64 == 20224
    a = np.arange(1, N + 1)[:, None]
    b = np.arange(1, N + 1)[None, :]
    h = np.pi / (N + 1)
    for p, q in ((1, 1), (3, 7), (64, 2), (33, 64)):
        P = 2 * (N + 1)
        v = (np.sin(((a * p) % P) * h) * np.sin(((b * q) % P) * h)).reshape(-1)
        lam = 4 - 2 * np.cos(p * h) - 2 * np.cos(q * h)
        got = oracle.spmv_coo_obj(coo, v)
        assert np.max(np.abs(got - lam * v)) <= 1e-13


def test_beta_zero_ignores_y_and_beta_uses_y(oracle):
    coo = matgen.laplacian_2d(8)
    x = matgen.dense_vector(64, 1)
    y = np.full(64, np.nan)
    assert np.all(np.isfinite(oracle.spmv_coo_obj(coo, x, 2.0, 0.0, y)))
    y2 = matgen.dense_vector(64, 2)
    base = oracle.spmv_coo_obj(coo, x, 2.0, 0.0)
    assert np.allclose(oracle.spmv_coo_obj(coo, x, 2.0, 0.5, y2),
                       base + 0.5 * y2, rtol=0, atol=1e-15)


def test_empty_cases(oracle):
    assert oracle.spmv_coo(0, 5, [], [], [], np.ones(5)).shape == (0,)
    got = oracle.spmv_coo(4, 3, [], [], [], np.ones(3), 1.0, 2.0,
                          np.arange(4.0))
    assert np.array_equal(got, 2.0 * np.arange(4.0))


def test_out_of_range_rejected(oracle):
    with pytest.raises(ValueError):
        oracle.spmv_coo(3, 3, [0, 3], [0, 0], [1.0, 1.0], np.ones(3))
    with pytest.raises(ValueError):
        oracle.spmv_coo(3, 3, [0], [-1], [1.0], np.ones(3))


def test_compensated_sum_within_two_ulps(oracle):
    """A single row of 200k positive products: the compensated sum stays
    within a few ulps of the exactly rounded sum (math.fsum); plain
    left-to-right summation drifts by hundreds of ulps here."""
    rng = np.random.default_rng(21)
    k = 200_000
    vals = rng.random(k)
    x = rng.random(k)
    got = oracle.spmv_coo(1, k, np.zeros(k, np.int32),
                          np.arange(k, dtype=np.int32), vals, x)[0]
    exact = math.fsum((vals * x).tolist())
    assert abs(got - exact) <= 4 * math.ulp(exact)
    naive = 0.0
    for p in (vals * x).tolist():
        naive += p
    assert abs(naive - exact) > 4 * math.ulp(exact)   # the test can tell


def test_csr_from_coo_matches_dense(oracle):
    rng = np.random.default_rng(31)
    coo = matgen.random_coo(30, 25, 300, rng, duplicates=True, shuffle=True,
                            integer_values=9)
    rp, ci, cv = oracle.csr_from_coo(30, 25, coo.rows, coo.cols, coo.vals)
    A = np.zeros((30, 25))
    for r in range(30):
        seg = slice(rp[r], rp[r + 1])
        assert np.all(np.diff(ci[seg]) > 0)          # sorted, unique columns
        A[r, ci[seg]] = cv[seg]
    assert np.array_equal(A, dense_of(30, 25, coo.rows, coo.cols, coo.vals))
