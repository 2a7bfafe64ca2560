"""GPU parity of the Jacobi iteration and the preconditioner against the
CPU oracle, through the C ABI.

The Jacobi kernel evaluates every FP64 operation of Algorithm 1 with the
same rounding as the oracle (rotation, row updates, scores), and selects the
exact argmax of the FP64 scores with the same tie rule.  Given the same A1
and V0, the two therefore produce the same pivot sequence and bit-identical
final A1, W and V; the tests assert exactly that.  The only operation that
is not bit-identical is the off-mass sum of the stopping test (a different
summation order), which could move the stop by one test period only if
off(A) fell within a rounding error of the threshold.
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
    hd = pj.Handle(transform="fp64")
    yield hd
    hd.close()


_cache = {}


def oracle_run(key, a1, v0, pivot, tol, **kw):
    k = (key, pivot, tol, tuple(sorted(kw.items())))
    if k not in _cache:
        r = oracle.jacobi(a1, v0, pivot=pivot, tol=tol, **kw)
        w, v = oracle.readout(r["a"], r["v"])
        _cache[k] = (r, w, v)
    return _cache[k]


def gpu_run(pj, h, a1, v0, pivot, tol, **opts):
    h.set_opts(transform="fp64", **opts)
    a = torch.tensor(np.ascontiguousarray(a1), device="cuda")
    v = None if v0 is None else torch.tensor(np.ascontiguousarray(v0), device="cuda")
    w, V, info, st = pj.pjac_solve_preconditioned(h, a, v, pivot, tol, allow=(0, -4, -5))
    torch.cuda.synchronize()
    return w.cpu().numpy(), V.cpu().numpy(), a.cpu().numpy(), info, st


def preconditioned(cfg, n=None):
    p = pin.config_problem(cfg, n=n)
    q0 = oracle.q0_fp32(p.a)
    q, a1 = oracle.precondition(p.a, q0)
    return p, q0, q, a1


def assert_bit_parity(r, w, v, gw, gv, ga, info):
    assert info["rotations"] == r["rotations"]
    assert np.array_equal(ga, r["a"]), np.max(np.abs(ga - r["a"]))
    assert np.array_equal(gw, w)
    assert np.array_equal(gv, v)


@pytest.mark.parametrize("pivot", ["gap", "greedy", "cyclic"])
def test_worked_example_parity(pj, h, pivot):
    a = pin.worked_example()
    r, w, v = oracle_run("worked", a, None, pivot, 1e-18)
    gw, gv, ga, info, st = gpu_run(pj, h, a, None, pivot, 1e-18)
    assert st == 0
    assert_bit_parity(r, w, v, gw, gv, ga, info)


@pytest.mark.parametrize("pivot", ["gap", "greedy", "cyclic"])
def test_cfg1_parity(pj, h, pivot):
    p, q0, q, a1 = preconditioned("cfg1")
    r, w, v = oracle_run("cfg1", a1, q, pivot, 1e-15)
    gw, gv, ga, info, st = gpu_run(pj, h, a1, q, pivot, 1e-15)
    assert st == 0 and r["status"] == 0
    assert_bit_parity(r, w, v, gw, gv, ga, info)
    assert np.max(np.abs(gw - p.lam)) <= 1e-13 * p.norm2


@pytest.mark.parametrize("pivot", ["gap", "greedy"])
def test_unpreconditioned_random_parity(pj, h, pivot):
    """Large rotation angles and many ties-free rescans: a random symmetric
    matrix of a ragged order (n=77), no preconditioner."""
    rng = np.random.default_rng(21)
    b = rng.standard_normal((77, 77))
    a = b + b.T
    r, w, v = oracle_run("rand77", a, None, pivot, 1e-14)
    gw, gv, ga, info, st = gpu_run(pj, h, a, None, pivot, 1e-14)
    assert st == 0
    assert_bit_parity(r, w, v, gw, gv, ga, info)


@pytest.mark.parametrize("cluster", [1, 2, 4])
@pytest.mark.parametrize("pivot", ["gap", "greedy"])
def test_cluster_parity_n300(pj, h, pivot, cluster):
    """n=300 (config 2's recipe, 9 clusters of 32 + a ragged 12) on 1, 2
    and 4 cooperating CTAs: 300/4 = 75 indices per CTA."""
    p, q0, q, a1 = preconditioned("cfg2", n=300)
    r, w, v = oracle_run("cfg2_300", a1, q, pivot, 1e-15)
    gw, gv, ga, info, st = gpu_run(pj, h, a1, q, pivot, 1e-15, cluster_size=cluster)
    assert st == 0
    assert_bit_parity(r, w, v, gw, gv, ga, info)


@pytest.mark.parametrize("cluster,pivot", [(8, "gap"), (16, "gap"), (16, "greedy")])
def test_cluster_parity_n520(pj, h, pivot, cluster):
    p, q0, q, a1 = preconditioned("cfg2", n=520)
    r, w, v = oracle_run("cfg2_520", a1, q, pivot, 1e-15)
    gw, gv, ga, info, st = gpu_run(pj, h, a1, q, pivot, 1e-15, cluster_size=cluster)
    assert st == 0
    assert_bit_parity(r, w, v, gw, gv, ga, info)
    assert np.max(np.abs(gw - p.lam)) <= 1e-13 * p.norm2


def ties_matrix(kind, n):
    """Matrices whose scores tie exactly, so that the tie rule (smallest
    (i, j)) and the exact evaluation of near-equal keys decide the pivots:
    equal off-diagonals over an equal diagonal (every initial score equal),
    small integers (many equal |a_ij| and equal gaps), and the constant
    tridiagonal (every nonzero score equal at the start)."""
    if kind == "equal":
        return 2.0 * np.eye(n) + 0.5 * (np.ones((n, n)) - np.eye(n))
    if kind == "int":
        rng = np.random.default_rng(17)
        u = np.triu(rng.integers(-2, 3, size=(n, n)).astype(np.float64), 1)
        return u + u.T + np.diag(rng.integers(-3, 4, size=n).astype(np.float64))
    a = np.zeros((n, n))
    i = np.arange(n - 1)
    a[i, i + 1] = a[i + 1, i] = 1.0
    return a


@pytest.mark.parametrize("pivot", ["gap", "greedy"])
@pytest.mark.parametrize("kind,n,cluster", [("equal", 70, 1), ("equal", 70, 2), ("int", 130, 1),
                                            ("int", 130, 4), ("tridiag", 130, 2)])
def test_exact_ties_parity(pj, h, kind, n, cluster, pivot):
    a = ties_matrix(kind, n)
    r, w, v = oracle_run(("ties", kind, n), a, None, pivot, 1e-15)
    gw, gv, ga, info, st = gpu_run(pj, h, a, None, pivot, 1e-15, cluster_size=cluster)
    assert st == 0 and r["status"] == 0
    assert_bit_parity(r, w, v, gw, gv, ga, info)


def test_cyclic_cluster_parity(pj, h):
    p, q0, q, a1 = preconditioned("cfg2", n=200)
    r, w, v = oracle_run("cfg2_200", a1, q, "cyclic", 1e-15)
    gw, gv, ga, info, st = gpu_run(pj, h, a1, q, "cyclic", 1e-15, cluster_size=4)
    assert st == 0
    assert_bit_parity(r, w, v, gw, gv, ga, info)


def test_max_rotations_and_libound(pj, h):
    p, q0, q, a1 = preconditioned("cfg1")
    # rotation budget: status ENOCONV, same partial state as the oracle
    r, w, v = oracle_run("cfg1", a1, q, "gap", 1e-15, max_rot=37)
    gw, gv, ga, info, st = gpu_run(pj, h, a1, q, "gap", 1e-15, max_rotations=37)
    assert st == -4 and info["status"] == -4 and r["status"] == 1
    assert_bit_parity(r, w, v, gw, gv, ga, info)
    # Theorem 1 stop
    r, w, v = oracle_run("cfg1", a1, q, "gap", 1e-11, stop="libound")
    gw, gv, ga, info, st = gpu_run(pj, h, a1, q, "gap", 1e-11, stop="libound")
    assert st == 0
    assert_bit_parity(r, w, v, gw, gv, ga, info)


def test_edge_cases(pj, h):
    h.set_opts(transform="fp64")
    # n = 1
    a = torch.tensor([[3.5]], dtype=torch.float64, device="cuda")
    w, V, info, st = pj.pjac_solve(h, a)
    assert w.item() == 3.5 and V.item() == 1.0
    # n = 2
    a2 = np.array([[2.0, 1e-3], [1e-3, 1.0]])
    gw, gv, ga, info, st = gpu_run(pj, h, a2, None, "gap", 1e-15)
    r, w2, v2 = oracle_run("n2", a2, None, "gap", 1e-15)
    assert_bit_parity(r, w2, v2, gw, gv, ga, info)
    # already diagonal and all-zero: no rotation
    d = np.diag([3.0, 1.0, 2.0, 2.0, -1.0])
    gw, gv, ga, info, st = gpu_run(pj, h, d, None, "gap", 1e-15)
    assert info["rotations"] == 0 and np.array_equal(gw, np.sort(np.diag(d)))
    z = np.zeros((6, 6))
    gw, gv, ga, info, st = gpu_run(pj, h, z, None, "greedy", 1e-15)
    assert info["rotations"] == 0 and np.array_equal(gw, np.zeros(6))
    assert np.array_equal(gv, np.eye(6))
    # invalid inputs are rejected before any compute
    bad = torch.tensor(np.array([[1.0, np.nan], [np.nan, 2.0]]), device="cuda")
    with pytest.raises(pj.PjacError) as e:
        pj.pjac_solve(h, bad)
    assert e.value.status == -1
    asym = torch.tensor(np.array([[1.0, 2.0], [2.5, 2.0]]), device="cuda")
    with pytest.raises(pj.PjacError):
        pj.pjac_solve(h, asym)
    # device time budget: the kernel gives up cleanly with ETIMEOUT
    p, q0, q, a1 = preconditioned("cfg2", n=300)
    gw, gv, ga, info, st = gpu_run(pj, h, a1, q, "gap", 1e-15, time_budget_s=1e-7)
    assert st == -5 and info["status"] == -5
    h.set_opts(transform="fp64")


def test_precondition_parity(pj, h):
    """Sec. 2.1 on the GPU (FP64 products) against the oracle's
    Newton--Schulz + FP64 transform, same Q0."""
    h.set_opts(transform="fp64")
    for cfg, n in (("cfg1", None), ("cfg2", 300)):
        p = pin.config_problem(cfg, n=n)
        q0 = oracle.q0_fp32(p.a)
        q, a1 = oracle.precondition(p.a, q0)
        gq, ga1 = pj.pjac_precondition(h, torch.tensor(p.a, device="cuda"), torch.tensor(q0, device="cuda"))
        gq, ga1 = gq.cpu().numpy(), ga1.cpu().numpy()
        assert np.max(np.abs(gq - q)) <= 1e-14
        assert np.max(np.abs(ga1 - a1)) <= 1e-14 * np.abs(p.a).max()
        assert np.array_equal(ga1, ga1.T)


@pytest.mark.parametrize("cfg,n", [("cfg1", None), ("cfg2", 300), ("cfg2", None)])
def test_full_solve_known_spectrum(pj, h, cfg, n):
    """End to end (GPU FP32 diagonaliser, Newton--Schulz, transform,
    Jacobi, readout) against the spectrum the matrix was built from."""
    h.set_opts(transform="fp64")
    p = pin.config_problem(cfg, n=n)
    a = torch.tensor(p.a, device="cuda")
    for pivot in ("gap", "greedy"):
        w, V, info, st = pj.pjac_solve(h, a, pivot, 1e-15)
        w, V = w.cpu().numpy(), V.cpu().numpy()
        assert st == 0
        assert np.max(np.abs(w - p.lam)) <= 1e-13 * p.norm2
        assert np.linalg.norm(p.a @ V - V * w) / np.linalg.norm(p.a) <= 1e-12
        assert np.linalg.norm(V.T @ V - np.eye(p.n)) <= 1e-12
        assert info["off_rel"] <= 1e-15


@pytest.mark.parametrize("n,cluster,seed", [(32, 1, 99), (300, 4, 7), (77, 2, 0)])
def test_random_pivot_parity(pj, h, n, cluster, seed):
    """Sec. 4.2's randomized comparator: both sides draw the same pairs from
    the counter-based SplitMix64 sequence, so the results are bit-identical."""
    if n == 32:
        p, q0, q, a1 = preconditioned("cfg1")
    elif n == 300:
        p, q0, q, a1 = preconditioned("cfg2", n=300)
    else:
        rng = np.random.default_rng(21)
        b = rng.standard_normal((77, 77))
        a1, q = b + b.T, None
    r, w, v = oracle_run(("rand", n, seed), a1, q, "random", 1e-15, seed=seed)
    gw, gv, ga, info, st = gpu_run(pj, h, a1, q, "random", 1e-15, cluster_size=cluster, seed=seed)
    assert st == 0 and r["status"] == 0
    assert_bit_parity(r, w, v, gw, gv, ga, info)


def test_solve_without_preconditioner(pj, h):
    """opts.no_precondition: Algorithm 1 directly on A with V0 = I (the
    setting of Sec. 4.2), bit-identical to the oracle on A itself."""
    rng = np.random.default_rng(5)
    b = rng.standard_normal((150, 150))
    a = b @ b.T + 150 * np.eye(150)
    a = 0.5 * (a + a.T)
    r, w, v = oracle_run("noprec150", a, None, "gap", 1e-15)
    h.set_opts(transform="fp64", no_precondition=1)
    gw, gv, info, st = pj.pjac_solve(h, torch.tensor(a, device="cuda"), "gap", 1e-15)
    h.set_opts(transform="fp64")
    assert st == 0 and info["rotations"] == r["rotations"]
    assert np.array_equal(gw.cpu().numpy(), w)
    assert np.array_equal(gv.cpu().numpy(), v)


@pytest.mark.parametrize("K,ratio,pivot", [(1, 0.0, "gap"), (4, 0.0, "gap"), (16, 0.0, "gap"), (32, 0.0, "gap"),
                                           (16, 0.01, "gap"), (16, 0.0, "greedy")])
def test_multi_pivot_parity(pj, h, K, ratio, pivot):
    """The multi-pivot variant: the same accepted pivot sets, rotations,
    crossing-block updates and cache updates as the oracle, bit for bit;
    K = 1 is Algorithm 1."""
    p, q0, q, a1 = preconditioned("cfg2", n=300)
    r = oracle.jacobi_multi(a1, q, pivot=pivot, tol=1e-15, K=K, ratio=ratio)
    w, v = oracle.readout(r["a"], r["v"])
    gw, gv, ga, info, st = gpu_run(pj, h, a1, q, pivot, 1e-15, multi_pivot=max(K, 2) if K > 1 else 0,
                                   multi_ratio=ratio)
    if K == 1:
        r1, w1, v1 = oracle_run("cfg2_300", a1, q, pivot, 1e-15)
        assert r["rotations"] == r1["rotations"] and np.array_equal(r["a"], r1["a"])
    assert st == 0 and r["status"] == 0
    assert info["steps"] == r["steps"]
    assert_bit_parity(r, w, v, gw, gv, ga, info)


@pytest.mark.parametrize("kind,n", [("equal", 70), ("int", 130), ("tridiag", 130)])
def test_multi_pivot_ties_parity(pj, h, kind, n):
    a = ties_matrix(kind, n)
    r = oracle.jacobi_multi(a, None, pivot="gap", tol=1e-15, K=16)
    w, v = oracle.readout(r["a"], r["v"])
    gw, gv, ga, info, st = gpu_run(pj, h, a, None, "gap", 1e-15, multi_pivot=16)
    assert st == 0 and info["steps"] == r["steps"]
    assert_bit_parity(r, w, v, gw, gv, ga, info)
