"""Allocation-free Jacobi entry point.

pjac_solve_preconditioned_noalloc serves callers that must not allocate
device memory while they solve (a process that reserves its whole memory
budget at start-up, or a plug-in without access to its host application's
allocator).  It keeps its scratch in a fixed array inside the library.  This
test calls it through the C ABI and checks that two calls in a row give the
same results as pjac_solve_preconditioned, the entry point that allocates
its workspace, within the tolerance the other Jacobi tests use (here, bit
equality: both run the same iteration on the same inputs).  The file is
named to be collected last.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import pjac_inputs as pin

pytestmark = pytest.mark.gpu


def _noalloc(lib, a1, v0, pivot, tol, mem=None):
    """One call through the C ABI; the caller's buffers are made first, so
    that ``mem`` (a list) can receive the device's free memory just before
    and just after the call."""
    n = a1.shape[0]
    a = torch.tensor(np.ascontiguousarray(a1), device="cuda")
    v0t = None if v0 is None else torch.tensor(np.ascontiguousarray(v0.T), device="cuda")
    w = torch.empty(n, dtype=torch.float64, device="cuda")
    vt = torch.empty((n, n), dtype=torch.float64, device="cuda")
    from paper_2607_23187_b300 import pjac
    info = pjac.Info()
    torch.cuda.synchronize()
    if mem is not None:
        mem.append(torch.cuda.mem_get_info()[0])
    st = lib.pjac_solve_preconditioned_noalloc(
        ctypes.c_void_p(a.data_ptr()), n, n, None if v0t is None else ctypes.c_void_p(v0t.data_ptr()), n,
        pjac.PIVOTS[pivot], ctypes.c_double(tol), ctypes.c_void_p(w.data_ptr()), ctypes.c_void_p(vt.data_ptr()), n,
        ctypes.byref(info), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    if mem is not None:
        mem.append(torch.cuda.mem_get_info()[0])
    return st, w.cpu().numpy(), vt.t().cpu().numpy(), a.cpu().numpy(), info.rotations


def _existing(pj, a1, v0, pivot, tol):
    h = pj.Handle(transform="fp64")
    try:
        a = torch.tensor(np.ascontiguousarray(a1), device="cuda")
        v = None if v0 is None else torch.tensor(np.ascontiguousarray(v0), device="cuda")
        w, V, info, st = pj.pjac_solve_preconditioned(h, a, v, pivot, tol)
        torch.cuda.synchronize()
        return st, w.cpu().numpy(), V.cpu().numpy(), a.cpu().numpy(), info["rotations"]
    finally:
        h.close()


def test_noalloc_matches_the_allocating_entry_point():
    from paper_2607_23187_b300 import pjac
    lib = pjac.load()
    fn = lib.pjac_solve_preconditioned_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                   ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(pjac.Info),
                   ctypes.c_void_p]
    p = pin.config_problem("cfg2", n=300)
    q, a1 = oracle.precondition(p.a, oracle.q0_fp32(p.a))
    rng = np.random.default_rng(21)
    b = rng.standard_normal((77, 77))
    # n = 500 runs on a cluster of four CTAs, whose V and solve record then
    # live in the shared array too
    p5 = pin.config_problem("cfg2", n=500)
    q5, a15 = oracle.precondition(p5.a, oracle.q0_fp32(p5.a))
    cases = [(a1, q, "gap"), (b + b.T, None, "greedy"), (a15, q5, "gap")]
    # two calls in a row, each against the allocating entry point
    for a, v0, pivot in cases:
        st, w, v, af, rot = _noalloc(lib, a, v0, pivot, 1e-15)
        st2, w2, v2, af2, rot2 = _existing(pjac, a, v0, pivot, 1e-15)
        assert st == 0 and st2 == 0
        assert rot == rot2 > 0
        assert np.array_equal(w, w2)
        assert np.array_equal(v, v2)
        assert np.array_equal(af, af2)
    # after the first call, a call takes no device memory at all
    mem = []
    st, *_ = _noalloc(lib, a15, q5, "gap", 1e-15, mem=mem)
    assert st == 0 and mem[0] == mem[1], mem
    # sizes beyond the fixed scratch are refused with a clear error
    big = np.eye(513)
    st, *_ = _noalloc(lib, big, None, "gap", 1e-15)
    assert st == pjac.PJAC_EINVAL
    assert b"allocation-free limit" in lib.pjac_last_error()
