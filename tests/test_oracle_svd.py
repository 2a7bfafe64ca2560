"""Pins of the oracle's one-sided Jacobi SVD (Alg. 2 with Sec. 2.1's SVD
preconditioner) against what the mathematics fixes: singular values built
into a matrix in double-double, LAPACK's SVD, orthogonality of both factors,
the residual, the 2x2 closed form, and the preconditioner's effect."""
import numpy as np
import pytest

import oracle
import pjac_inputs as pin


def _two_cluster_sigma(n, rng):
    h = n // 2
    return np.concatenate([1.0 + 1e-9 * rng.uniform(-1, 1, h), np.linspace(2.0, 3.0, n - h)])


@pytest.mark.parametrize("pivot", ["gap", "greedy", "cyclic"])
def test_svd_known_singular_values(pivot):
    rng = np.random.default_rng(4)
    sig = _two_cluster_sigma(48, rng)
    p = pin.svd_problem(70, 48, sig, seed=4)
    r = oracle.svd_jacobi(p.b, pivot=pivot, tol=1e-15)
    assert r["status"] == 0
    nb = np.max(p.sigma)
    assert np.max(np.abs(r["sigma"] - p.sigma)) <= 1e-13 * nb
    assert np.all(np.diff(r["sigma"]) <= 0)
    u, v = r["u"], r["v_sorted"]
    assert np.linalg.norm(u.T @ u - np.eye(48)) <= 1e-12
    assert np.linalg.norm(v.T @ v - np.eye(48)) <= 1e-12
    assert np.linalg.norm(p.b @ v - u * r["sigma"]) <= 1e-13 * np.linalg.norm(p.b)


def test_svd_matches_lapack_and_unpreconditioned():
    rng = np.random.default_rng(9)
    b = rng.standard_normal((90, 60))
    ref = np.linalg.svd(b, compute_uv=False)
    r = oracle.svd_jacobi(b, pivot="gap", tol=1e-15)
    r0 = oracle.svd_jacobi(b, pivot="gap", tol=1e-15, precondition_vectors=False)
    assert np.max(np.abs(r["sigma"] - ref)) <= 1e-13 * ref[0]
    assert np.max(np.abs(r0["sigma"] - ref)) <= 1e-13 * ref[0]
    # the low-precision preconditioner leaves far fewer rotations
    assert r["rotations"] < 0.5 * r0["rotations"]


def test_svd_two_columns_closed_form():
    """Two columns: one rotation makes them orthogonal; the singular values
    are the square roots of the 2x2 Gram matrix's eigenvalues (closed form,
    evaluated in 50-digit arithmetic)."""
    import mpmath
    rng = np.random.default_rng(2)
    b = rng.standard_normal((5, 2))
    r = oracle.svd_jacobi(b, pivot="gap", tol=1e-15, precondition_vectors=False)
    with mpmath.workdps(50):
        g = [[sum(mpmath.mpf(b[k, i]) * mpmath.mpf(b[k, j]) for k in range(5)) for j in range(2)] for i in range(2)]
        tr = g[0][0] + g[1][1]
        det = g[0][0] * g[1][1] - g[0][1] * g[1][0]
        disc = mpmath.sqrt(tr * tr / 4 - det)
        s = [float(mpmath.sqrt(tr / 2 + disc)), float(mpmath.sqrt(tr / 2 - disc))]
    assert r["rotations"] == 1
    assert np.max(np.abs(r["sigma"] - np.array(s))) <= 4e-16 * s[0]
    assert abs(r["u"][:, 0] @ r["u"][:, 1]) <= 1e-15


def test_column_norms_scaled_sum():
    x = np.array([[3e200, 1e-200, 0.0], [4e200, 0.0, 0.0]])
    assert np.allclose(oracle.column_norms(x), [5e200, 1e-200, 0.0], rtol=1e-15)


def test_hilbert_cholesky_closed_form():
    """The closed-form Cholesky factor of Sec. 4.2 reproduces the Hilbert
    matrix to rounding."""
    n = 14
    c = pin.hilbert_cholesky(n)
    h = 1.0 / (np.arange(1, n + 1)[:, None] + np.arange(1, n + 1)[None, :] - 1)
    assert np.allclose(np.tril(c), c)
    assert np.max(np.abs(c @ c.T - h)) <= 4e-16
