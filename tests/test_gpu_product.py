"""The working-precision product of the preconditioner (Sec. 2.1: the
Newton--Schulz steps and Q^T A Q) on the tensor cores, through the C ABI
(pjac_product with PJAC_TRANSFORM_SPLIT_BF16).

Two kinds of checks:
  * exactness: inputs whose entries have at most two 6-bit digits below
    their row (column) maximum make every slice product an integer matrix
    the tensor cores must sum without rounding, and the FP64 recombination
    of three diagonals in fixed point is exact too; the result must equal the exact
    product bit for bit.  The all-63-digit case puts the FP32 partial sums
    within 3% of 2^24, the limit of exact accumulation.
  * accuracy: on dense inputs (normal entries, rows scaled by powers of two
    up to 2^+-30, and a case with a 2^+-8 spread inside every row) the error
    against a double-double product stays within the bound of the splitting,
    |C - AB|_ij <= 2^(e_i + f_j) (k (S+3) 2^-bS + T 2^-(2b+38)) + u |C|, over ragged shapes,
    both transposes, alpha and beta, k at the b = 6 limit and beyond it
    (b = 5).
"""
import numpy as np
import pytest
import torch

import oracle
import pjac_inputs as pin

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pj():
    from paper_2607_23187_b300 import pjac
    pjac.load()
    return pjac


@pytest.fixture(scope="module")
def h(pj):
    hd = pj.Handle(transform="split_bf16")
    yield hd
    hd.close()


def gpu_product(pj, h, a, b, ta=False, tb=False, alpha=1.0, beta=0.0, c=None):
    A = torch.tensor(np.ascontiguousarray(a), device="cuda")
    B = torch.tensor(np.ascontiguousarray(b), device="cuda")
    C = None if c is None else torch.tensor(np.ascontiguousarray(c), device="cuda")
    out = pj.pjac_product(h, A, B, ta, tb, alpha, beta, C)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def exp_above(x):
    """e with 2^(e-1) <= x < 2^e (0 for x = 0)."""
    e = np.zeros(x.shape, np.int64)
    nz = x > 0
    e[nz] = np.frexp(x[nz])[1]
    return e


def split_params(k):
    b = 6 if k * 63 * 63 <= 2 ** 24 else 5
    return b, (54 + b - 1) // b


def bound(a_op, b_op, alpha=1.0):
    k = a_op.shape[1]
    b, S = split_params(k)
    ea = exp_above(np.abs(a_op).max(axis=1))
    eb = exp_above(np.abs(b_op).max(axis=0))
    scale = np.ldexp(1.0, ea[:, None] + eb[None, :])
    c = np.abs(alpha * (a_op @ b_op))
    # T slice products (s, t) with b (s + t) > 37 are rounded to 37
    # fractional bits in the fixed-point sum, each by at most half a unit
    T = sum(d + 1 for d in range(S) if b * d > 37)
    return abs(alpha) * scale * (k * (S + 3) * 2.0 ** (-b * S) + T * 2.0 ** -(2 * b + 38)) + 2.0 ** -53 * c


def two_digit_matrix(rng, rows, cols, maxdigits=False):
    """Integer matrix I with |I| < 4096 (two 6-bit digits) whose every row
    has an entry with leading digit >= 32 (so that its row maximum fixes
    the digit grid), and a power-of-two row scale."""
    if maxdigits:
        I = np.full((rows, cols), 63 * 64 + 63, dtype=np.int64)
    else:
        I = rng.integers(0, 4096, size=(rows, cols))
        I[:, 0] = rng.integers(2048, 4096, size=rows)
        I *= rng.choice([-1, 1], size=(rows, cols))
    return I


@pytest.mark.parametrize("m,k,n,maxdig", [(200, 2048, 136, True), (130, 1024, 70, True),
                                          (257, 513, 129, False), (64, 4096, 64, True),
                                          (5, 3, 7, False)])
def test_exact_on_digit_inputs(pj, h, m, k, n, maxdig):
    rng = np.random.default_rng(m * 7 + k)
    IA = two_digit_matrix(rng, m, k, maxdig)
    IBt = two_digit_matrix(rng, n, k, maxdig)          # columns of B as rows
    ra = rng.integers(-30, 30, size=m)
    rb = rng.integers(-30, 30, size=n)
    a = np.ldexp(IA.astype(np.float64), (ra - 12)[:, None])
    b = np.ldexp(IBt.astype(np.float64), (rb - 12)[:, None]).T.copy()
    # exact: integer products summed in FP64 (|sum| < 2^36, no rounding)
    exact = np.ldexp((IA.astype(np.float64) @ IBt.T.astype(np.float64)), (ra[:, None] + rb[None, :] - 24))
    got = gpu_product(pj, h, a, b)
    np.testing.assert_array_equal(got, exact)


def dense_case(rng, m, k, n, spread):
    a = rng.standard_normal((m, k)) * np.ldexp(1.0, rng.integers(-30, 30, size=(m, 1)))
    b = rng.standard_normal((k, n)) * np.ldexp(1.0, rng.integers(-30, 30, size=(1, n)))
    if spread:
        a *= np.ldexp(1.0, rng.integers(-8, 8, size=(m, k)))
        b *= np.ldexp(1.0, rng.integers(-8, 8, size=(k, n)))
    return a, b


@pytest.mark.parametrize("m,k,n,spread", [(1, 1, 1, False), (3, 7, 5, True), (130, 200, 70, False),
                                          (256, 1024, 256, True), (300, 4100, 200, False),
                                          (64, 5000, 72, True), (1024, 1024, 1024, False)])
def test_error_within_bound(pj, h, m, k, n, spread):
    rng = np.random.default_rng(m + 3 * k + 5 * n)
    a, b = dense_case(rng, m, k, n, spread)
    got = gpu_product(pj, h, a, b)
    hi, lo = oracle.exact_matmul(a, b)
    err = np.abs((got - hi) - lo)
    assert np.all(err <= bound(a, b)), float((err / bound(a, b)).max())


@pytest.mark.parametrize("ta,tb", [(False, True), (True, False), (True, True)])
def test_transposes_alpha_beta(pj, h, ta, tb):
    rng = np.random.default_rng(11)
    m, k, n = 150, 333, 97
    a, b = dense_case(rng, m, k, n, True)
    c0 = rng.standard_normal((m, n))
    a_st = a.T.copy() if ta else a
    b_st = b.T.copy() if tb else b
    alpha, beta = -0.75, 0.5
    got = gpu_product(pj, h, a_st, b_st, ta, tb, alpha, beta, c0)
    hi, lo = oracle.exact_matmul(a, b)
    ref = alpha * hi + beta * c0
    tol = bound(a, b, alpha) + 2 * 2.0 ** -53 * (np.abs(alpha * hi) + np.abs(beta * c0))
    assert np.all(np.abs(got - ref) <= tol)


def gpu_product_sym(pj, h, a, b, ta=False, tb=False, alpha=1.0, beta=0.0, c=None):
    A = torch.tensor(np.ascontiguousarray(a), device="cuda")
    B = torch.tensor(np.ascontiguousarray(b), device="cuda")
    C = None if c is None else torch.tensor(np.ascontiguousarray(c), device="cuda")
    out = pj.pjac_product_symmetric(h, A, B, ta, tb, alpha, beta, C)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("n,k,form", [(300, 200, "gram"), (130, 7, "gram"), (700, 4100, "gram"),
                                      (520, 300, "sandwich"), (1024, 1024, "outer")])
def test_symmetric_product(pj, h, n, k, form):
    """pjac_product_symmetric (the tiles on and above the diagonal, mirrored):
    the result is exactly symmetric and every entry is within the bound of
    the splitting at the entry, (i, j) or (j, i), that was computed.  Cases:
    Gram matrices X^T X (one with k at the b = 5 digit width, one small
    enough to spread tiles over several CTAs), X^T (S X) with S symmetric and
    S X exact (small integers), and X X^T with alpha and beta."""
    rng = np.random.default_rng(n + 7 * k)
    alpha, beta, c0 = 1.0, 0.0, None
    if form == "sandwich":
        x = rng.integers(-1000, 1000, size=(k, n)).astype(np.float64)
        s = rng.integers(-50, 50, size=(k, k)).astype(np.float64)
        s = s + s.T
        a_op, b_op = x.T, s @ x            # exact: integers below 2^36
        a_st, b_st, ta, tb = x, s @ x, True, False
    else:
        x = rng.standard_normal((k, n)) * np.ldexp(1.0, rng.integers(-20, 20, size=(1, n)))
        if form == "gram":
            a_op, b_op = x.T, x
            a_st, b_st, ta, tb = x, x, True, False
        else:
            x = x.T.copy()                 # n x k, C = X X^T
            a_op, b_op = x, x.T
            a_st, b_st, ta, tb = x, x, False, True
            alpha, beta = 0.5, -1.5
            c0 = rng.standard_normal((n, n))
            c0 = c0 + c0.T
    got = gpu_product_sym(pj, h, a_st, b_st, ta, tb, alpha, beta, c0)
    assert np.array_equal(got, got.T)
    hi, lo = oracle.exact_matmul(a_op, b_op)
    bnd = bound(a_op, b_op, alpha)
    tol = np.maximum(bnd, bnd.T)
    if c0 is None:
        err = np.abs((got - alpha * hi) - alpha * lo)
    else:
        ref = alpha * hi + beta * c0
        err = np.abs(got - ref)
        tol = tol + 2 * 2.0 ** -53 * (np.abs(alpha * hi) + np.abs(beta * c0))
    assert np.all(err <= tol), float((err / tol).max())
    with pj.Handle(transform="fp64") as h64:
        g64 = gpu_product_sym(pj, h64, a_st, b_st, ta, tb, alpha, beta, c0)
    assert np.array_equal(g64, g64.T)


def test_fp64_option_matches_plain_product(pj):
    """The same entry point with the FP64 option is the CUDA-core product."""
    rng = np.random.default_rng(5)
    a, b = dense_case(rng, 70, 90, 40, False)
    with pj.Handle(transform="fp64") as h64:
        got = gpu_product(pj, h64, a, b)
    hi, lo = oracle.exact_matmul(a, b)
    assert np.all(np.abs(got - hi) <= 90 * 2.0 ** -52 * (np.abs(a) @ np.abs(b)))


def test_bad_arguments(pj, h):
    lib = pj.load()
    x = torch.zeros((4, 4), dtype=torch.float64, device="cuda")
    p = x.data_ptr()
    assert lib.pjac_product(h.h, 0, 0, 0, 4, 4, 1.0, p, 4, p, 4, 0.0, p, 4, None) == pj.PJAC_EINVAL
    assert lib.pjac_product(h.h, 2, 0, 4, 4, 4, 1.0, p, 4, p, 4, 0.0, p, 4, None) == pj.PJAC_EINVAL
    assert lib.pjac_product(h.h, 0, 0, 4, 4, 4, 1.0, p, 3, p, 4, 0.0, p, 4, None) == pj.PJAC_EINVAL
    assert lib.pjac_product(h.h, 0, 0, 4, 4, 4, 1.0, None, 4, p, 4, 0.0, p, 4, None) == pj.PJAC_EINVAL
    assert lib.pjac_product_symmetric(h.h, 0, 0, 0, 4, 1.0, p, 4, p, 4, 0.0, p, 4, None) == pj.PJAC_EINVAL
    assert lib.pjac_product_symmetric(h.h, 0, 2, 4, 4, 1.0, p, 4, p, 4, 0.0, p, 4, None) == pj.PJAC_EINVAL
    assert lib.pjac_product_symmetric(h.h, 0, 0, 4, 4, 1.0, p, 4, p, 4, 0.0, p, 3, None) == pj.PJAC_EINVAL


def test_launch_count(pj, h):
    lib = pj.load()
    assert lib.pjac_product_launch_count(h.h, 1000, 900, 800) in (3, 4)
    assert lib.pjac_product_launch_count(h.h, 0, 4, 4) == -1
    assert lib.pjac_product_launch_count(None, 4, 4, 4) == -1
    with pj.Handle(transform="fp64") as h64:
        assert lib.pjac_product_launch_count(h64.h, 1000, 900, 800) == 1


def test_preconditioner_with_split_product(pj, h):
    """Sec. 2.1 with the tensor-core products: same Q0, the A1 of the split
    product and of the FP64 product agree to the transform's error, and
    Q is orthogonal to working precision."""
    p = pin.config_problem("cfg1", n=256)
    q0 = oracle.q0_fp32(p.a)
    a = torch.tensor(p.a, device="cuda")
    q0t = torch.tensor(q0, device="cuda")
    h.set_opts(transform="split_bf16")
    qs, a1s = pj.pjac_precondition(h, a, q0t)
    with pj.Handle(transform="fp64") as h64:
        qd, a1d = pj.pjac_precondition(h64, a, q0t)
    qs, a1s, qd, a1d = (t.cpu().numpy() for t in (qs, a1s, qd, a1d))
    n = p.a.shape[0]
    assert np.linalg.norm(qs.T @ qs - np.eye(n)) < 1e-13
    nrm = np.linalg.norm(p.a, 2)
    assert np.abs(a1s - a1d).max() < 64 * n * 2.0 ** -53 * nrm
    exact = oracle.transform_exact(p.a, qs)
    assert np.abs(a1s - exact).max() < 16 * n * 2.0 ** -53 * nrm


@pytest.mark.parametrize("cfg,n", [("cfg1", 512), ("cfg2", 256)])
def test_full_solve_split_product(pj, h, cfg, n):
    """End to end with the tensor-core transform: eigenvalues within
    1e-13 ||A|| of the known spectrum, V orthogonal, small residual."""
    p = pin.config_problem(cfg, n=n)
    h.set_opts(transform="split_bf16")
    a = torch.tensor(p.a, device="cuda")
    w, v, info, st = pj.pjac_solve(h, a, "gap", 1e-15)
    w, v = w.cpu().numpy(), v.cpu().numpy()
    assert st == 0
    assert np.max(np.abs(w - p.lam)) <= 1e-13 * p.norm2
    assert np.linalg.norm(p.a @ v - v * w) / np.linalg.norm(p.a) <= 1e-12
    assert np.linalg.norm(v.T @ v - np.eye(p.n)) <= 1e-12
    assert info["off_rel"] <= 1e-15
