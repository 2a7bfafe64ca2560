"""Thin Python binding of libpjac (the C ABI of include/pjac.h).

Argument marshalling only: every step of the solver runs in the CUDA
library.  PyTorch supplies device memory and the current stream.  Matrices
are FP64 CUDA tensors; the library's column-major convention is honoured by
passing transposed views where it matters (for symmetric inputs the layouts
coincide).  The library is loaded from ``lib/libpjac.so`` next to this file;
if it is missing or the device is unavailable the calls raise -- there is
no other implementation behind them.
"""
from __future__ import annotations

import ctypes
import os
import threading
from typing import Optional, Sequence, Tuple

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libpjac.so")

PJAC_OK, PJAC_PENDING = 0, 1
PJAC_EINVAL, PJAC_ENOMEM, PJAC_EAGAIN = -1, -2, -3
PJAC_ENOCONV, PJAC_ETIMEOUT, PJAC_ECUDA, PJAC_ENOTIMPL = -4, -5, -6, -7
PIVOTS = {"gap": 0, "greedy": 1, "cyclic": 2, "random": 3, "gap_rel": 4}
STOPS = {"offdiag": 0, "libound": 1}
TRANSFORMS = {"split_bf16": 0, "fp64": 1}

EXPORTS = (
    "pjac_default_opts", "pjac_create", "pjac_destroy", "pjac_set_opts", "pjac_precondition",
    "pjac_solve", "pjac_solve_preconditioned", "pjac_solve_batched", "pjac_serve_default_opts",
    "pjac_serve_create", "pjac_serve_destroy", "pjac_serve_submit", "pjac_serve_poll",
    "pjac_serve_progress", "pjac_serve_get_stats", "pjac_status_string", "pjac_last_error",
    "pjac_solve_preconditioned_noalloc", "pjac_product", "pjac_product_symmetric", "pjac_product_plan",
    "pjac_solve_launch_count",
    "pjac_product_launch_count", "pjac_eig_lowprec", "pjac_svd", "pjac_svd_onesided", "pjac_probe_fp64",
    "pjac_batched_stage_ms", "pjac_batched_tuning", "pjac_fp32_sweeps_done",
)


class PjacError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s (status %d)" % (msg, status))
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("stop", ctypes.c_int), ("tol", ctypes.c_double),
                ("max_rotations", ctypes.c_int64), ("check_every", ctypes.c_int64),
                ("transform", ctypes.c_int), ("ns_steps", ctypes.c_int),
                ("cluster_size", ctypes.c_int), ("time_budget_s", ctypes.c_double),
                ("no_precondition", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("refine_steps", ctypes.c_int), ("fp32_sweeps", ctypes.c_int),
                ("multi_pivot", ctypes.c_int), ("multi_ratio", ctypes.c_double), ("autotune", ctypes.c_int)]


class Info(ctypes.Structure):
    _fields_ = [("rotations", ctypes.c_int64), ("sweeps", ctypes.c_double),
                ("off_rel", ctypes.c_double), ("max_score", ctypes.c_double),
                ("status", ctypes.c_int32), ("n", ctypes.c_int32),
                ("ms_precond", ctypes.c_float), ("ms_transform", ctypes.c_float),
                ("ms_jacobi", ctypes.c_float), ("steps", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServeOpts(ctypes.Structure):
    _fields_ = [("max_slots", ctypes.c_int), ("max_queue", ctypes.c_int),
                ("hbm_budget_bytes", ctypes.c_size_t), ("solver", Opts)]


class ServeStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("p50_ms", ctypes.c_double),
                ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("mean_ms", ctypes.c_double), ("solves_per_s", ctypes.c_double),
                ("peak_inflight", ctypes.c_int64), ("peak_hbm_bytes", ctypes.c_size_t),
                ("launches", ctypes.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None
_lock = threading.Lock()


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libpjac and declare its signatures (no GPU needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise ImportError("libpjac.so not built: run `python -m paper_2607_23187_b300.build_lib`")
        L = ctypes.CDLL(path)
        vp, i, d, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
        L.pjac_default_opts.argtypes = [ctypes.POINTER(Opts)]
        L.pjac_default_opts.restype = None
        L.pjac_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Opts)]
        L.pjac_destroy.argtypes = [vp]
        L.pjac_set_opts.argtypes = [vp, ctypes.POINTER(Opts)]
        L.pjac_precondition.argtypes = [vp, vp, i, i, vp, vp, i, vp, i, vp]
        L.pjac_solve.argtypes = [vp, vp, i, i, i, d, vp, vp, i, ctypes.POINTER(Info), vp]
        L.pjac_solve_preconditioned.argtypes = [vp, vp, i, i, vp, i, i, d, vp, vp, i,
                                                ctypes.POINTER(Info), vp]
        L.pjac_product.argtypes = [vp, i, i, i, i, i, d, vp, i, vp, i, d, vp, i, vp]
        L.pjac_product_symmetric.argtypes = [vp, i, i, i, i, d, vp, i, vp, i, d, vp, i, vp]
        L.pjac_eig_lowprec.argtypes = [vp, vp, i, i, vp, i, vp]
        L.pjac_svd.argtypes = [vp, vp, i, i, i, vp, i, i, d, vp, vp, i, vp, i, ctypes.POINTER(Info), vp]
        L.pjac_svd_onesided.argtypes = [vp, vp, i, i, i, i, d, vp, vp, i, vp, i, ctypes.POINTER(Info), vp]
        L.pjac_probe_fp64.argtypes = [ctypes.POINTER(d), vp]
        L.pjac_probe_fp64.restype = ctypes.c_int
        L.pjac_product_plan.argtypes = [i, i, i, i, i, vp, vp, i]
        L.pjac_product_plan.restype = ctypes.c_int
        L.pjac_batched_stage_ms.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
        L.pjac_batched_stage_ms.restype = ctypes.c_int
        L.pjac_batched_tuning.argtypes = [vp, i, i, ctypes.POINTER(i), ctypes.POINTER(i),
                                          ctypes.POINTER(ctypes.c_float)]
        L.pjac_batched_tuning.restype = ctypes.c_int
        L.pjac_fp32_sweeps_done.argtypes = [vp, ctypes.POINTER(i), ctypes.POINTER(i)]
        L.pjac_fp32_sweeps_done.restype = ctypes.c_int
        L.pjac_solve_batched.argtypes = [vp, i, vp, vp, vp, vp, vp, vp, vp, i, d, vp, vp]
        L.pjac_serve_default_opts.argtypes = [ctypes.POINTER(ServeOpts)]
        L.pjac_serve_default_opts.restype = None
        L.pjac_serve_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(ServeOpts)]
        L.pjac_serve_destroy.argtypes = [vp]
        L.pjac_serve_submit.argtypes = [vp, vp, i, i, i, d, vp, vp, i, ctypes.POINTER(ctypes.c_uint64)]
        L.pjac_serve_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(Info)]
        L.pjac_serve_progress.argtypes = [vp]
        L.pjac_serve_get_stats.argtypes = [vp, ctypes.POINTER(ServeStats)]
        L.pjac_solve_launch_count.argtypes = [vp, i]
        L.pjac_product_launch_count.argtypes = [vp, i, i, i]
        L.pjac_status_string.argtypes = [i]
        L.pjac_status_string.restype = ctypes.c_char_p
        L.pjac_last_error.argtypes = []
        L.pjac_last_error.restype = ctypes.c_char_p
        for name in ("pjac_create", "pjac_destroy", "pjac_set_opts", "pjac_precondition", "pjac_eig_lowprec",
                     "pjac_svd", "pjac_svd_onesided",
                     "pjac_solve",
                     "pjac_solve_preconditioned", "pjac_solve_batched", "pjac_serve_create",
                     "pjac_serve_destroy", "pjac_serve_submit", "pjac_serve_poll",
                     "pjac_serve_progress", "pjac_serve_get_stats"):
            getattr(L, name).restype = ctypes.c_int
        _lib = L
        return L


def _check(status: int, allow=(PJAC_OK,)) -> int:
    if status not in allow:
        L = load()
        raise PjacError(status, L.pjac_last_error().decode())
    return status


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def default_opts(**kw) -> Opts:
    o = Opts()
    load().pjac_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if k == "stop":
            v = STOPS[v] if isinstance(v, str) else v
        if k == "transform":
            v = TRANSFORMS[v] if isinstance(v, str) else v
        setattr(o, k, v)
    return o


class Handle:
    """pjac_create / pjac_destroy."""

    def __init__(self, **opts):
        self.h = ctypes.c_void_p()
        o = default_opts(**opts)
        _check(load().pjac_create(ctypes.byref(self.h), ctypes.byref(o)))

    def set_opts(self, **opts):
        o = default_opts(**opts)
        _check(load().pjac_set_opts(self.h, ctypes.byref(o)))

    def fp32_sweeps_done(self):
        """(sweeps of the FP32 diagonalisation, sweeps of its refinement) made
        by the handle's last low-precision eigenbasis (pjac_fp32_sweeps_done)."""
        d, r = ctypes.c_int(), ctypes.c_int()
        _check(load().pjac_fp32_sweeps_done(self.h, ctypes.byref(d), ctypes.byref(r)))
        return d.value, r.value

    def close(self):
        if self.h:
            load().pjac_destroy(self.h)
            self.h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _sym_input(a: torch.Tensor) -> torch.Tensor:
    if not (a.is_cuda and a.dtype == torch.float64 and a.dim() == 2 and a.shape[0] == a.shape[1]):
        raise ValueError("expected a square FP64 CUDA tensor")
    return a.contiguous()


def pjac_precondition(h: Handle, a: torch.Tensor, q0: Optional[torch.Tensor] = None
                      ) -> Tuple[torch.Tensor, torch.Tensor]:
    """Sec. 2.1 preconditioner.  q0: optional (n,n) FP32 approximate
    eigenvectors (columns).  Returns (Q, A1) as (n,n) FP64 tensors."""
    a = _sym_input(a)
    n = a.shape[0]
    q0c = None
    if q0 is not None:
        q0c = q0.to(device=a.device, dtype=torch.float32).t().contiguous()   # column-major storage
    qt = torch.empty((n, n), dtype=torch.float64, device=a.device)
    a1 = torch.empty((n, n), dtype=torch.float64, device=a.device)
    _check(load().pjac_precondition(h.h, _ptr(a), n, n, _ptr(q0c), _ptr(qt), n, _ptr(a1), n, _stream()))
    return qt.t(), a1


def pjac_eig_lowprec(h: Handle, a: torch.Tensor) -> torch.Tensor:
    """The low-precision spectral decomposition of Sec. 2.1 (FP32): returns
    Q0 as an (n,n) FP32 tensor whose columns are eigenvector estimates."""
    a = _sym_input(a)
    n = a.shape[0]
    q0t = torch.empty((n, n), dtype=torch.float32, device=a.device)
    _check(load().pjac_eig_lowprec(h.h, _ptr(a), n, n, _ptr(q0t), n, _stream()))
    return q0t.t()


def pjac_product(h: Handle, a: torch.Tensor, b: torch.Tensor, trans_a: bool = False, trans_b: bool = False,
                 alpha: float = 1.0, beta: float = 0.0, c: Optional[torch.Tensor] = None) -> torch.Tensor:
    """alpha op(a) @ op(b) + beta c with the handle's transform (split-BF16
    tensor-core product or plain FP64).  a, b: FP64 CUDA matrices (row-major
    torch layout); op(x) = x.T when the flag is set.  The library works in
    column-major order, so it is handed C^T = op(b)^T op(a)^T, which reads
    the row-major storage of a and b directly."""
    a = a.contiguous()
    b = b.contiguous()
    m = a.shape[1] if trans_a else a.shape[0]
    k = a.shape[0] if trans_a else a.shape[1]
    kb = b.shape[1] if trans_b else b.shape[0]
    n = b.shape[0] if trans_b else b.shape[1]
    if kb != k:
        raise ValueError(f"inner dimensions differ: {k} vs {kb}")
    if c is None:
        c = torch.zeros((m, n), dtype=torch.float64, device=a.device)
        beta = 0.0
    elif c.shape != (m, n) or not c.is_contiguous():
        raise ValueError("c must be a contiguous (m, n) tensor")
    _check(load().pjac_product(h.h, 1 if trans_b else 0, 1 if trans_a else 0, n, m, k, float(alpha),
                               _ptr(b), b.shape[1], _ptr(a), a.shape[1], float(beta), _ptr(c), n, _stream()))
    return c


def pjac_product_symmetric(h: Handle, a: torch.Tensor, b: torch.Tensor, trans_a: bool = False,
                           trans_b: bool = False, alpha: float = 1.0, beta: float = 0.0,
                           c: Optional[torch.Tensor] = None) -> torch.Tensor:
    """alpha op(a) @ op(b) + beta c for a product the caller knows to be
    symmetric in exact arithmetic; the result is exactly symmetric.  As in
    pjac_product the library is handed C^T = op(b)^T op(a)^T (also
    symmetric)."""
    a = a.contiguous()
    b = b.contiguous()
    m = a.shape[1] if trans_a else a.shape[0]
    k = a.shape[0] if trans_a else a.shape[1]
    kb = b.shape[1] if trans_b else b.shape[0]
    n = b.shape[0] if trans_b else b.shape[1]
    if kb != k or m != n:
        raise ValueError(f"expected op(a) {m}x{k} and op(b) {kb}x{n} with a square product")
    if c is None:
        c = torch.zeros((n, n), dtype=torch.float64, device=a.device)
        beta = 0.0
    elif c.shape != (n, n) or not c.is_contiguous():
        raise ValueError("c must be a contiguous (n, n) tensor")
    _check(load().pjac_product_symmetric(h.h, 1 if trans_b else 0, 1 if trans_a else 0, n, k, float(alpha),
                                         _ptr(b), b.shape[1], _ptr(a), a.shape[1], float(beta), _ptr(c), n,
                                         _stream()))
    return c


def pjac_solve(h: Handle, a: torch.Tensor, pivot: str = "gap", tol: float = 1e-15,
               vectors: bool = True, allow=(PJAC_OK,)):
    """Full solve.  Returns (W, V, info dict, status); V is (n,n) with
    column k the eigenvector of W[k] (None when vectors=False)."""
    a = _sym_input(a)
    n = a.shape[0]
    w = torch.empty(n, dtype=torch.float64, device=a.device)
    vt = torch.empty((n, n), dtype=torch.float64, device=a.device) if vectors else None
    info = Info()
    st = load().pjac_solve(h.h, _ptr(a), n, n, PIVOTS[pivot], float(tol), _ptr(w), _ptr(vt), n,
                           ctypes.byref(info), _stream())
    _check(st, allow)
    return w, (vt.t() if vt is not None else None), info.as_dict(), st


def pjac_solve_preconditioned(h: Handle, a1: torch.Tensor, v0: Optional[torch.Tensor] = None,
                              pivot: str = "gap", tol: float = 1e-15, allow=(PJAC_OK,)):
    """Algorithm 1 on A1 (overwritten in place with the final matrix).
    v0: (n,n) starting V (None: identity).  Returns (W, V, info, status)."""
    if not (a1.is_cuda and a1.dtype == torch.float64 and a1.is_contiguous()):
        raise ValueError("a1 must be a contiguous FP64 CUDA tensor")
    n = a1.shape[0]
    v0c = None if v0 is None else v0.to(dtype=torch.float64).t().contiguous()
    w = torch.empty(n, dtype=torch.float64, device=a1.device)
    vt = torch.empty((n, n), dtype=torch.float64, device=a1.device)
    info = Info()
    st = load().pjac_solve_preconditioned(h.h, _ptr(a1), n, n, _ptr(v0c), n, PIVOTS[pivot], float(tol),
                                          _ptr(w), _ptr(vt), n, ctypes.byref(info), _stream())
    _check(st, allow)
    return w, vt.t(), info.as_dict(), st


def pjac_svd(h: Handle, b: torch.Tensor, pivot: str = "gap", tol: float = 1e-15,
             vl: Optional[torch.Tensor] = None, vectors: bool = True, allow=(PJAC_OK,)):
    """One-sided Jacobi SVD of b (m, n), m >= n, FP64 CUDA.  vl: optional
    (n, n) FP32 right singular vectors (columns).  Returns (S descending,
    U (m, n), V (n, n), info, status); U and V are None with vectors=False."""
    if not (b.is_cuda and b.dtype == torch.float64 and b.dim() == 2):
        raise ValueError("expected an FP64 CUDA matrix")
    m, n = b.shape
    bc = b.t().contiguous()                       # column-major storage
    vlc = None if vl is None else vl.to(device=b.device, dtype=torch.float32).t().contiguous()
    s = torch.empty(n, dtype=torch.float64, device=b.device)
    ut = torch.empty((n, m), dtype=torch.float64, device=b.device) if vectors else None
    vt = torch.empty((n, n), dtype=torch.float64, device=b.device) if vectors else None
    info = Info()
    st = load().pjac_svd(h.h, _ptr(bc), m, n, m, _ptr(vlc), n, PIVOTS[pivot], float(tol), _ptr(s), _ptr(ut), m,
                         _ptr(vt), n, ctypes.byref(info), _stream())
    _check(st, allow)
    return s, (None if ut is None else ut.t()), (None if vt is None else vt.t()), info.as_dict(), st


def pjac_svd_onesided(h: Handle, b: torch.Tensor, pivot: str = "gap_rel", tol: float = 1e-16,
                      vectors: bool = True, allow=(PJAC_OK,)):
    """One-sided Jacobi SVD with inner products recomputed from the columns
    (relative accuracy, no preconditioner).  b (m, n) FP64 CUDA, m >= n.
    Returns (S descending, U (m, n), V (n, n), info, status)."""
    if not (b.is_cuda and b.dtype == torch.float64 and b.dim() == 2):
        raise ValueError("expected an FP64 CUDA matrix")
    m, n = b.shape
    bc = b.t().contiguous()
    s = torch.empty(n, dtype=torch.float64, device=b.device)
    ut = torch.empty((n, m), dtype=torch.float64, device=b.device) if vectors else None
    vt = torch.empty((n, n), dtype=torch.float64, device=b.device) if vectors else None
    info = Info()
    st = load().pjac_svd_onesided(h.h, _ptr(bc), m, n, m, PIVOTS[pivot], float(tol), _ptr(s), _ptr(ut), m,
                                  _ptr(vt), n, ctypes.byref(info), _stream())
    _check(st, allow)
    return s, (None if ut is None else ut.t()), (None if vt is None else vt.t()), info.as_dict(), st


def probe_fp64_tflops() -> float:
    """Measured FP64 FMA rate of the current device (TFLOP/s)."""
    v = ctypes.c_double()
    _check(load().pjac_probe_fp64(ctypes.byref(v), _stream()))
    return v.value


def pjac_solve_batched(h: Handle, mats: Sequence[torch.Tensor], pivot: str = "gap", tol: float = 1e-15,
                       vectors: bool = True):
    """Batched form: list of (n_p, n_p) FP64 CUDA matrices.  Returns
    (list of W, list of V, infos tensor view, raw buffers)."""
    import numpy as np
    dev = mats[0].device
    ns = np.array([m.shape[0] for m in mats], dtype=np.int32)
    sizes = ns.astype(np.int64) ** 2
    aoff = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    woff = np.concatenate([[0], np.cumsum(ns.astype(np.int64))[:-1]]).astype(np.int64)
    A = torch.cat([m.contiguous().reshape(-1) for m in mats])
    W = torch.empty(int(ns.sum()), dtype=torch.float64, device=dev)
    V = torch.empty(int(sizes.sum()), dtype=torch.float64, device=dev) if vectors else None
    infos = torch.empty((len(mats), ctypes.sizeof(Info)), dtype=torch.uint8, device=dev)
    _check(load().pjac_solve_batched(h.h, len(mats), ns.ctypes.data_as(ctypes.c_void_p),
                                     aoff.ctypes.data_as(ctypes.c_void_p), _ptr(A),
                                     woff.ctypes.data_as(ctypes.c_void_p), _ptr(W),
                                     aoff.ctypes.data_as(ctypes.c_void_p), _ptr(V), PIVOTS[pivot],
                                     float(tol), _ptr(infos), _stream()))
    return dict(ns=ns, aoff=aoff, woff=woff, A=A, W=W, V=V, infos=infos)


def batched_results(res):
    """Split the packed outputs of pjac_solve_batched (synchronises)."""
    torch.cuda.synchronize()
    ns, aoff, woff = res["ns"], res["aoff"], res["woff"]
    raw = res["infos"].cpu().numpy().tobytes()
    isz = ctypes.sizeof(Info)
    infos = [Info.from_buffer_copy(raw[k * isz:(k + 1) * isz]).as_dict() for k in range(len(ns))]
    ws, vs = [], []
    for k, m in enumerate(ns):
        m = int(m)
        ws.append(res["W"][woff[k]:woff[k] + m])
        if res["V"] is not None:
            vs.append(res["V"][aoff[k]:aoff[k] + m * m].reshape(m, m).t())
    return ws, vs, infos


class Server:
    """pjac_serve_*: continuous batching of eigenproblems."""

    def __init__(self, max_slots: int = 0, max_queue: int = 0, hbm_budget_bytes: int = 0, **solver):
        L = load()
        o = ServeOpts()
        L.pjac_serve_default_opts(ctypes.byref(o))
        if max_slots:
            o.max_slots = max_slots
        if max_queue:
            o.max_queue = max_queue
        if hbm_budget_bytes:
            o.hbm_budget_bytes = hbm_budget_bytes
        for k, v in solver.items():
            if k == "stop" and isinstance(v, str):
                v = STOPS[v]
            if k == "transform" and isinstance(v, str):
                v = TRANSFORMS[v]
            setattr(o.solver, k, v)
        self.s = ctypes.c_void_p()
        _check(L.pjac_serve_create(ctypes.byref(self.s), ctypes.byref(o)))
        self._keep = {}

    def submit(self, a_host, pivot: str = "gap", tol: float = 1e-15, vectors: bool = True) -> int:
        """a_host: (n,n) FP64 numpy array (symmetric).  Returns a ticket."""
        import numpy as np
        a = np.ascontiguousarray(a_host, dtype=np.float64)
        n = a.shape[0]
        w = np.empty(n)
        v = np.empty((n, n)) if vectors else None
        t = ctypes.c_uint64()
        st = load().pjac_serve_submit(self.s, a.ctypes.data_as(ctypes.c_void_p), n, n, PIVOTS[pivot],
                                      float(tol), w.ctypes.data_as(ctypes.c_void_p),
                                      None if v is None else v.ctypes.data_as(ctypes.c_void_p), n,
                                      ctypes.byref(t))
        if st == PJAC_EAGAIN:
            return -1
        _check(st)
        self._keep[t.value] = (a, w, v)
        return t.value

    def poll(self, ticket: int):
        """(status, info, W, V): status PJAC_PENDING while running."""
        info = Info()
        st = load().pjac_serve_poll(self.s, ctypes.c_uint64(ticket), ctypes.byref(info))
        if st == PJAC_PENDING:
            return st, None, None, None
        a, w, v = self._keep.pop(ticket, (None, None, None))
        return st, info.as_dict(), w, (None if v is None else v.T)

    def progress(self) -> int:
        return load().pjac_serve_progress(self.s)

    def stats(self):
        s = ServeStats()
        _check(load().pjac_serve_get_stats(self.s, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if self.s:
            load().pjac_serve_destroy(self.s)
            self.s = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def product_plan(m: int, n: int, k: int, symmetric: bool = False, sms: int = 0) -> Tuple[dict, list]:
    """The split-BF16 product's schedule (host only): ({b, S, units, splits,
    ctas, pairs}, [(s, t, unit, split), ...] in launch order)."""
    info = (ctypes.c_int * 6)()
    cap = 128
    pairs = (ctypes.c_int * (4 * cap))()
    _check(load().pjac_product_plan(int(m), int(n), int(k), 1 if symmetric else 0, int(sms), info, pairs, cap))
    keys = ("b", "S", "units", "splits", "ctas", "pairs")
    d = {kk: info[j] for j, kk in enumerate(keys)}
    return d, [tuple(pairs[4 * j:4 * j + 4]) for j in range(min(d["pairs"], cap))]
