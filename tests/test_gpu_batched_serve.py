"""Batched and serving forms on the GPU.

The per-problem arithmetic of both forms is the single-problem pipeline
(its Jacobi stage is the same device routine that test_gpu_jacobi checks
bit for bit against the oracle with one CTA).  Here:
  * every problem reaches the spectrum it was built from
    (|dlambda| <= 1e-13 ||A||_2, residual and orthogonality <= 1e-12);
  * a problem's result does not depend on the batch it is solved in
    (bit-identical alone and inside a batch of mixed sizes);
  * a served request gives the same result alone and in a mixed stream;
  * the serving scheduler runs waiting small requests ahead of a waiting
    large one, at most four micro-batches in a row.
"""
import time

import numpy as np
import pytest
import torch

import pjac_inputs as pin

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pj():
    from paper_2607_23187_b300 import pjac
    pjac.load()
    return pjac


def _check(p, w, v):
    w = np.asarray(w)
    v = np.asarray(v)
    assert np.max(np.abs(w - p.lam)) <= 1e-13 * p.norm2
    assert np.linalg.norm(p.a @ v - v * w) / np.linalg.norm(p.a) <= 1e-12
    assert np.linalg.norm(v.T @ v - np.eye(p.n)) <= 1e-12


@pytest.mark.parametrize("pivot", ["gap", "greedy"])
def test_batched_known_spectra_and_independence(pj, pivot):
    probs = pin.batched_workload(count=120, seed=1)
    # add the edge sizes: 2, 3, odd, and the largest batched order
    rng = np.random.default_rng(5)
    for n in (2, 3, 17, 255, 256):
        probs.append(pin.small_clustered_problem(n, rng, "clustered"))
    h = pj.Handle(transform="fp64")
    mats = [torch.tensor(p.a, device="cuda") for p in probs]
    res = pj.pjac_solve_batched(h, mats, pivot, 1e-15)
    ws, vs, infos = pj.batched_results(res)
    for p, w, v, inf in zip(probs, ws, vs, infos):
        assert inf["status"] == 0, inf
        _check(p, w.cpu().numpy(), v.cpu().numpy())
    # the same problems alone, in a different order and grouping: identical
    for k in (0, 7, len(probs) - 1, len(probs) - 3):
        r1 = pj.pjac_solve_batched(h, [mats[k]], pivot, 1e-15)
        w1, v1, i1 = pj.batched_results(r1)
        assert np.array_equal(w1[0].cpu().numpy(), ws[k].cpu().numpy())
        assert np.array_equal(v1[0].cpu().numpy(), vs[k].cpu().numpy())
        assert i1[0]["rotations"] == infos[k]["rotations"]
    h.close()


def test_batched_rejects_bad_sizes(pj):
    h = pj.Handle(transform="fp64")
    with pytest.raises(pj.PjacError):
        pj.pjac_solve_batched(h, [torch.zeros((1, 1), dtype=torch.float64, device="cuda")])
    with pytest.raises(pj.PjacError):
        pj.pjac_solve_batched(h, [torch.zeros((1100, 1100), dtype=torch.float64, device="cuda")])
    h.close()


def _serve_all(pj, srv, reqs, timeout=300.0):
    tickets = [srv.submit(a, piv, 1e-15) for a, piv in reqs]
    out = [None] * len(reqs)
    t0 = time.time()
    left = len(reqs)
    while left and time.time() - t0 < timeout:
        for k, t in enumerate(tickets):
            if out[k] is not None:
                continue
            st, info, w, v = srv.poll(t)
            if st == pj.PJAC_PENDING:
                continue
            out[k] = (st, info, w.copy(), v.copy())
            left -= 1
        time.sleep(0.001)
    assert left == 0, "serving did not finish"
    return out


def test_serving_mixed_stream_equals_alone(pj):
    sizes = (64, 128, 256, 512, 700)
    rng = np.random.default_rng(3)
    probs = [pin.small_clustered_problem(n, rng, "clustered") for n in sizes]
    order = [0, 3, 1, 1, 4, 2, 0, 3, 2, 1, 0, 4]
    reqs = [(probs[k].a, "gap" if j % 3 else "greedy") for j, k in enumerate(order)]
    srv = pj.Server(max_slots=4)
    mixed = _serve_all(pj, srv, reqs)
    st = srv.stats()
    assert st["completed"] == len(reqs) and st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()
    for (a, piv), k, (s, info, w, v) in zip(reqs, order, mixed):
        assert s == 0
        _check(probs[k], w, v)
    # each request alone on a fresh server: bit-identical results
    for j in (0, 1, 4, 5):
        srv1 = pj.Server(max_slots=1)
        alone = _serve_all(pj, srv1, [reqs[j]])[0]
        srv1.close()
        assert np.array_equal(alone[2], mixed[j][2])
        assert np.array_equal(alone[3], mixed[j][3])


def test_serving_admission_and_errors(pj):
    # a budget smaller than one request still admits it (never starves)
    srv = pj.Server(max_slots=2, hbm_budget_bytes=1 << 20)
    p = pin.small_clustered_problem(64, np.random.default_rng(1), "uniform")
    out = _serve_all(pj, srv, [(p.a, "gap"), (p.a, "gap")])
    assert all(o[0] == 0 for o in out)
    bad = p.a.copy()
    bad[0, 1] += 1.0
    with pytest.raises(pj.PjacError):
        srv.submit(bad)
    srv.close()


def test_serving_small_first_with_bounded_bypass(pj):
    """One lane, so the completion order is the run order.  A large request
    A takes the lane at once; then a large L and six small requests wait,
    the small ones with distinct tolerances (so each is its own
    micro-batch).  The small ones run first, but L is passed over by at
    most four micro-batches: A, S1..S4, L, S5, S6."""
    rng = np.random.default_rng(9)
    pa = pin.small_clustered_problem(400, rng, "clustered")
    pl = pin.small_clustered_problem(300, rng, "clustered")
    ps = [pin.small_clustered_problem(64 + 16 * k, rng, "uniform") for k in range(6)]
    srv = pj.Server(max_slots=1)
    names = ["A", "L"] + ["S%d" % (k + 1) for k in range(6)]
    probs = [pa, pl] + ps
    tols = [1e-15, 1e-15] + [(k + 1) * 1e-15 for k in range(6)]
    tickets = [srv.submit(p.a, "gap", t) for p, t in zip(probs, tols)]
    order, res = [], {}
    t0 = time.time()
    while len(order) < len(tickets) and time.time() - t0 < 300.0:
        for name, t in zip(names, tickets):
            if name in res:
                continue
            st, info, w, v = srv.poll(t)
            if st == pj.PJAC_PENDING:
                continue
            res[name] = (st, w.copy(), v.copy())
            order.append(name)
        time.sleep(0.001)
    launches = srv.stats()["launches"]
    srv.close()
    assert order == ["A", "S1", "S2", "S3", "S4", "L", "S5", "S6"]
    # two single-problem pipelines and six micro-batches of six kernels
    h = pj.Handle()
    count = pj.load().pjac_solve_launch_count
    assert launches == count(h.h, 400) + count(h.h, 300) + 6 * 6
    h.close()
    for name, p in zip(names, probs):
        assert res[name][0] == 0
        _check(p, res[name][1], res[name][2])
