"""Pins for the oracle's conjugate-gradient solver (the iterative setting of
Section 7.5, method of Hestenes and Stiefel).

Each test checks the oracle against something other than itself: closed-form
eigenpairs, finite termination on few distinct eigenvalues, a dense direct
solve, the steepest-descent first step, the orthogonality / conjugacy the
method guarantees, and monotone decrease of the energy-norm error.  A wrong
sign in alpha or beta, a swapped residual update or a stale rho breaks one.
"""
import numpy as np

from paper_2302_05662_gb300 import matgen


def dense(coo):
    A = np.zeros((coo.m, coo.n))
    np.add.at(A, (coo.rows.astype(np.int64), coo.cols.astype(np.int64)), coo.vals)
    return A


def diag_coo(d):
    n = len(d)
    i = np.arange(n, dtype=np.int32)
    return matgen.Coo(n, n, i, i.copy(), np.asarray(d, np.float64))


def run(oracle, coo, b, **kw):
    return oracle.cg(coo.m, coo.rows, coo.cols, coo.vals, b, **kw)


def test_eigenvector_rhs_converges_in_one_step(oracle):
    # 1D Laplacian tridiag(-1, 2, -1): v_j(i) = sin(i j pi/(N+1)), lambda_j = 4 sin^2(j pi/(2(N+1)))
    N, j = 40, 7
    coo = matgen.laplacian_1d(N)
    i = np.arange(1, N + 1)
    v = np.sin(i * j * np.pi / (N + 1))
    lam = 4 * np.sin(j * np.pi / (2 * (N + 1))) ** 2
    out = run(oracle, coo, v, tol=1e-12)
    assert out["iterations"] == 1 and out["converged"]
    np.testing.assert_allclose(out["x"], v / lam, rtol=0, atol=1e-13 * np.abs(v / lam).max())


def test_finite_termination_on_three_distinct_eigenvalues(oracle):
    d = np.tile([1.0, 2.0, 5.0], 30)
    coo = diag_coo(d)
    b = matgen.dense_vector(len(d), 3)
    out = run(oracle, coo, b, tol=1e-13)
    assert out["iterations"] == 3 and out["converged"]
    np.testing.assert_allclose(out["x"], b / d, rtol=1e-12)


def test_matches_dense_direct_solve(oracle):
    coo = matgen.laplacian_2d(16)
    b = matgen.dense_vector(coo.m, 11)
    out = run(oracle, coo, b, tol=1e-13, maxit=coo.m)
    want = np.linalg.solve(dense(coo), b)
    assert out["converged"] and out["iterations"] < coo.m
    np.testing.assert_allclose(out["x"], want, rtol=0, atol=1e-11 * np.abs(want).max())
    # the recursively updated residual agrees with the true one
    r_true = b - dense(coo) @ out["x"]
    assert np.sqrt(r_true @ r_true) <= 2e-13 * np.sqrt(b @ b)


def test_first_step_is_exact_line_search(oracle):
    coo = matgen.laplacian_2d(8)
    A = dense(coo)
    b = matgen.dense_vector(coo.m, 5)
    x0 = matgen.dense_vector(coo.m, 6)
    out = run(oracle, coo, b, x0=x0, maxit=1)
    r0 = b - A @ x0
    x1 = x0 + (r0 @ r0) / (r0 @ A @ r0) * r0
    assert out["iterations"] == 1
    np.testing.assert_allclose(out["x"], x1, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(out["rho"][0], r0 @ r0, rtol=1e-13)


def test_residuals_orthogonal_and_directions_conjugate(oracle):
    coo = matgen.stencil_3d(6, 7, values="laplace")
    A = dense(coo)
    b = matgen.dense_vector(coo.m, 9)
    out = run(oracle, coo, b, maxit=10, tol=0.0, record=True)
    R, P = out["r"], out["p"]
    assert len(R) == 11
    for i in range(8):
        for j in range(i + 1, 8):
            assert abs(R[i] @ R[j]) <= 1e-9 * np.linalg.norm(R[i]) * np.linalg.norm(R[j])
            assert abs(P[i] @ A @ P[j]) <= 1e-9 * np.sqrt((P[i] @ A @ P[i]) * (P[j] @ A @ P[j]))
    for k, r in enumerate(R):
        np.testing.assert_allclose(out["rho"][k], r @ r, rtol=1e-12)


def test_energy_norm_error_decreases(oracle):
    coo = matgen.laplacian_2d(12)
    A = dense(coo)
    b = matgen.dense_vector(coo.m, 13)
    xs = np.linalg.solve(A, b)
    prev = np.inf
    for k in range(1, 25):
        x = run(oracle, coo, b, maxit=k, tol=0.0)["x"]
        e = x - xs
        en = e @ A @ e
        assert en <= prev * (1 + 1e-12)
        prev = en
    assert prev < 1e-2 * (xs @ A @ xs)


def test_zero_rhs_and_exact_start_take_no_step(oracle):
    coo = matgen.laplacian_1d(10)
    out = run(oracle, coo, np.zeros(10))
    assert out["iterations"] == 0 and out["converged"] and not out["breakdown"]
    xs = np.arange(1.0, 11.0)
    b = dense(coo) @ xs          # integer entries: exact
    out = run(oracle, coo, b, x0=xs)
    assert out["iterations"] == 0 and out["rho"] == [0.0]
    np.testing.assert_array_equal(out["x"], xs)


def test_indefinite_matrix_breaks_down(oracle):
    coo = diag_coo([1.0, -1.0])
    out = run(oracle, coo, np.array([1.0, 1.0]))
    assert out["breakdown"] and out["iterations"] == 0 and not out["converged"]


def test_maxit_limits_products(oracle):
    coo = matgen.laplacian_2d(16)
    b = matgen.dense_vector(coo.m, 2)
    out = run(oracle, coo, b, maxit=5, tol=1e-14)
    assert out["iterations"] == 5 and not out["converged"] and len(out["rho"]) == 6
