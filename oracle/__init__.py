"""CPU FP64 oracle of the preconditioned Jacobi eigensolver.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg use it to check and time the CUDA
path.  Nothing in the product imports it, and it imports nothing from the
product.  It shares only the seeded input generators (``pjac_inputs``).

Layers (each cites the passage of Shao & Nakatsukasa it follows):

* ``pjac_oracle.c`` -- Algorithm 1 with the gap rule of Eq. (1.1), Jacobi's
  greedy rule and cyclic sweeps (Sec. 1, Sec. 2), the O(n) score update of
  Sec. 3.2 and the Theorem 1 stopping rule (Sec. 3.1), in plain FP64 C.
* this module -- the mixed-precision preconditioner of Sec. 2.1: a
  low-precision (FP32) spectral decomposition, reorthogonalisation to FP64 by
  Householder QR (the choice of the Sec. 4 experiments) or Newton--Schulz,
  and the preconditioned matrix V^T A V; plus the eigenvalue readout.
  Library routines (LAPACK eigh/qr, BLAS matmul, numpy sort) serve as steps.

Readings where the paper is silent are listed in ``pjac_oracle.c``'s header.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from typing import Dict, Optional, Tuple

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pjac_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

PIVOTS = {"gap": 0, "greedy": 1, "cyclic": 2, "random": 3, "gap_rel": 4}
STOPS = {"offdiag": 0, "libound": 1}


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, -O2 -ffp-contract=off, OpenMP)."""
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Info(ctypes.Structure):
    _fields_ = [("rotations", ctypes.c_longlong), ("sweeps", ctypes.c_longlong),
                ("checks", ctypes.c_longlong), ("norm_f", ctypes.c_double),
                ("off_final", ctypes.c_double), ("max_score_final", ctypes.c_double),
                ("status", ctypes.c_int), ("reserved", ctypes.c_int),
                ("first_rot_eig_ok", ctypes.c_longlong),
                ("eig_err_max_final", ctypes.c_double), ("eig_err_sum_final", ctypes.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            dp = ctypes.POINTER(ctypes.c_double)
            L.or_gap_score.restype = ctypes.c_double
            L.or_gap_score.argtypes = [ctypes.c_double] * 3
            L.or_greedy_score.restype = ctypes.c_double
            L.or_greedy_score.argtypes = [ctypes.c_double]
            L.or_rotation.restype = None
            L.or_rotation.argtypes = [ctypes.c_double] * 3 + [dp] * 3
            L.or_rotate.restype = None
            L.or_rotate.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                    ctypes.c_int, dp]
            L.or_offmass.restype = ctypes.c_double
            L.or_offmass.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double]
            L.or_frobenius.restype = ctypes.c_double
            L.or_frobenius.argtypes = [ctypes.c_void_p, ctypes.c_int]
            L.or_jacobi.restype = ctypes.c_int
            L.or_jacobi.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_double, ctypes.c_longlong,
                                    ctypes.c_longlong, ctypes.c_int, ctypes.c_void_p,
                                    ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p,
                                    ctypes.c_uint64, ctypes.POINTER(_Info)]
            L.or_splitmix64.restype = ctypes.c_uint64
            L.or_splitmix64.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
            L.or_gap_rel_score.restype = ctypes.c_double
            L.or_gap_rel_score.argtypes = [ctypes.c_double] * 3
            L.or_svd_onesided.restype = ctypes.c_int
            L.or_svd_onesided.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_uint64,
                                          ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong),
                                          ctypes.POINTER(ctypes.c_int)]
            L.or_jacobi_multi.restype = ctypes.c_int
            L.or_jacobi_multi.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_double, ctypes.c_longlong, ctypes.c_longlong,
                                          ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_longlong),
                                          ctypes.POINTER(_Info)]
            L.or_random_pair.restype = None
            L.or_random_pair.argtypes = [ctypes.c_uint64, ctypes.c_longlong, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
            L.or_jacobi_many.restype = ctypes.c_int
            L.or_jacobi_many.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                         ctypes.c_longlong, ctypes.c_void_p, ctypes.c_void_p]
            _lib = L
    return _lib


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


# ----------------------------------------------------------------------------
# scalar pieces
# ----------------------------------------------------------------------------
def gap_score(aii: float, ajj: float, aij: float) -> float:
    """Eq. (1.1): L_ij = 2|a_ij|^2 / (|a_ii-a_jj| + sqrt(|a_ii-a_jj|^2 + 4|a_ij|^2))."""
    return lib().or_gap_score(float(aii), float(ajj), float(aij))


def greedy_score(aij: float) -> float:
    """Jacobi's classical score |a_ij| (Sec. 1)."""
    return lib().or_greedy_score(float(aij))


def rotation(aii: float, ajj: float, aij: float) -> Tuple[float, float, float]:
    """(c, s, t) with G = [[c,-s],[s,c]] making G^T [[aii,aij],[aij,ajj]] G
    diagonal (Sec. 2), |theta| <= pi/4."""
    c, s, t = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    lib().or_rotation(float(aii), float(ajj), float(aij), ctypes.byref(c), ctypes.byref(s), ctypes.byref(t))
    return c.value, s.value, t.value


def rotate(a: np.ndarray, i: int, j: int, v: Optional[np.ndarray] = None) -> float:
    """Apply A <- G^T A G (and V <- V G) in place for pivot (i,j); returns t."""
    assert a.flags.c_contiguous and a.dtype == np.float64
    t = ctypes.c_double()
    lib().or_rotate(_ptr(a), a.shape[0], _ptr(v), int(i), int(j), ctypes.byref(t))
    return t.value


def offmass(a: np.ndarray, ref: Optional[float] = None) -> float:
    """off(A) = sqrt(sum_{k != l} a_kl^2)."""
    a = np.ascontiguousarray(a, dtype=np.float64)
    if ref is None:
        ref = frobenius(a)
    return lib().or_offmass(_ptr(a), a.shape[0], float(ref))


def frobenius(a: np.ndarray) -> float:
    a = np.ascontiguousarray(a, dtype=np.float64)
    return lib().or_frobenius(_ptr(a), a.shape[0])


# ----------------------------------------------------------------------------
# Algorithm 1
# ----------------------------------------------------------------------------
def jacobi(a1: np.ndarray, v0: Optional[np.ndarray] = None, pivot: str = "gap",
           stop: str = "offdiag", tol: float = 1e-15, max_rot: Optional[int] = None,
           check_every: Optional[int] = None, select: str = "cache",
           lam: Optional[np.ndarray] = None, eig_tol: float = 0.0,
           log_len: int = 0, hist_cap: int = 0, seed: int = 0) -> Dict:
    """Run Algorithm 1 on a copy of ``a1`` (symmetric FP64), accumulating
    V <- V0 G (identity when v0 is None).

    Returns a dict with the final matrix ``a``, ``v``, ``rotations``,
    ``status`` (0 converged, 1 budget reached), ``pivots`` (first log_len
    (i,j)), ``scores``, ``off_final``, ``norm_f``, ``first_rot_eig_ok`` and
    the convergence history when ``hist_cap`` > 0.
    """
    a = np.array(a1, dtype=np.float64, order="C", copy=True)
    n = a.shape[0]
    v = np.eye(n) if v0 is None else np.array(v0, dtype=np.float64, order="C", copy=True)
    if max_rot is None:
        max_rot = 50 * n * (n - 1) // 2 + 1
    if check_every is None:
        check_every = max(n, 1)
    lam_s = None if lam is None else np.ascontiguousarray(np.sort(lam), dtype=np.float64)
    piv = np.zeros(2 * max(log_len, 1), dtype=np.int32)
    sc = np.zeros(max(log_len, 1), dtype=np.float64)
    hr = np.zeros(max(hist_cap, 1), dtype=np.int64)
    he = np.zeros(max(hist_cap, 1), dtype=np.float64)
    ho = np.zeros(max(hist_cap, 1), dtype=np.float64)
    hl = ctypes.c_longlong(0)
    info = _Info()
    lib().or_jacobi(_ptr(a), n, _ptr(v), PIVOTS[pivot], STOPS[stop], float(tol), int(max_rot),
                    int(check_every), 1 if select == "cache" else 0, _ptr(lam_s), float(eig_tol),
                    _ptr(piv), _ptr(sc), int(log_len), _ptr(hr), _ptr(he), _ptr(ho), int(hist_cap),
                    ctypes.byref(hl), ctypes.c_uint64(seed), ctypes.byref(info))
    nl = min(log_len, info.rotations)
    return {
        "a": a, "v": v, "rotations": int(info.rotations), "sweeps": int(info.sweeps),
        "checks": int(info.checks), "status": int(info.status), "norm_f": info.norm_f,
        "off_final": info.off_final, "max_score_final": info.max_score_final,
        "pivots": piv[:2 * nl].reshape(-1, 2).copy(), "scores": sc[:nl].copy(),
        "first_rot_eig_ok": int(info.first_rot_eig_ok),
        "eig_err_max_final": info.eig_err_max_final, "eig_err_sum_final": info.eig_err_sum_final,
        "hist_rot": hr[:hl.value].copy(), "hist_err": he[:hl.value].copy(),
        "hist_off": ho[:hl.value].copy(),
    }


def splitmix64(seed: int, k: int) -> int:
    """Step k's 64-bit draw of the randomized pivot rule (SplitMix64's
    output function on the counter seed + (k+1) * 0x9e3779b97f4a7c15)."""
    return int(lib().or_splitmix64(ctypes.c_uint64(seed), ctypes.c_uint64(k)))


def random_pair(seed: int, k: int, n: int) -> Tuple[int, int]:
    """The pivot (i, j), i < j, of step k of the randomized rule (Sec. 4.2's
    comparator: every pair equally likely)."""
    i, j = ctypes.c_int(), ctypes.c_int()
    lib().or_random_pair(ctypes.c_uint64(seed), int(k), int(n), ctypes.byref(i), ctypes.byref(j))
    return i.value, j.value


def readout(a: np.ndarray, v: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Eigenvalues = diag(A) ascending (stable on ties), V's columns
    permuted the same way (Sec. 2: the diagonal approximates the spectrum)."""
    d = np.diag(a).copy()
    p = np.argsort(d, kind="stable")
    return d[p], v[:, p]


# ----------------------------------------------------------------------------
# Sec. 2.1: the mixed-precision preconditioner
# ----------------------------------------------------------------------------
def q0_fp32(a: np.ndarray) -> np.ndarray:
    """Low-precision spectral decomposition (u_l = single, Sec. 4):
    eigenvectors of fl32(A) computed in FP32 (LAPACK ssyevd)."""
    _, q0 = np.linalg.eigh(np.asarray(a, dtype=np.float32))
    return np.ascontiguousarray(q0.astype(np.float32))


def reorth_qr(q0: np.ndarray) -> np.ndarray:
    """Householder QR reorthogonalisation in FP64 (the Sec. 4 choice); the
    signs are fixed so that diag(R) > 0, which keeps Q close to Q0."""
    q, r = np.linalg.qr(np.asarray(q0, dtype=np.float64))
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return q * d[None, :]


def reorth_ns(q0: np.ndarray, steps: int = 3) -> np.ndarray:
    """Newton--Schulz reorthogonalisation (Sec. 2.1):
    X <- X (3I - X^T X) / 2, in FP64."""
    x = np.asarray(q0, dtype=np.float64).copy()
    n = x.shape[1]
    eye3 = 3.0 * np.eye(n)
    for _ in range(steps):
        x = 0.5 * (x @ (eye3 - x.T @ x))
    return x


def transform(a: np.ndarray, q: np.ndarray) -> np.ndarray:
    """The preconditioned matrix V^T A V (Sec. 2.1) in FP64, symmetrised
    as (A1 + A1^T)/2 (the paper does not say whether to symmetrise)."""
    a1 = q.T @ (np.asarray(a, dtype=np.float64) @ q)
    return 0.5 * (a1 + a1.T)


def _split_rows(x: np.ndarray, bits: int, nslices: int):
    rest = x.copy()
    out = []
    for _ in range(nslices):
        mu = np.max(np.abs(rest), axis=1, keepdims=True)
        e = np.ceil(np.log2(np.where(mu > 0, mu, 1.0)))
        sigma = np.ldexp(np.ones_like(mu), (e + (53 - bits)).astype(np.int64))
        hi = np.where(mu > 0, (rest + sigma) - sigma, 0.0)
        out.append(hi)
        rest = rest - hi
    if np.any(rest != 0):
        out.append(rest)
    return out


def exact_matmul(x: np.ndarray, y: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """X @ Y as an unevaluated sum hi + lo accurate to about 2^-100 relative
    (error-free slice products after Ozaki, Ogita, Oishi & Rump 2012, summed
    with Knuth's TwoSum).  Used only to measure the transform's error."""
    k = x.shape[1]
    bits = (53 - int(np.ceil(np.log2(max(k, 2))))) // 2
    ns = int(np.ceil(53 / bits))
    xs = _split_rows(np.asarray(x, dtype=np.float64), bits, ns)
    ys = _split_rows(np.asarray(y, dtype=np.float64).T.copy(), bits, ns)
    hi = np.zeros((x.shape[0], y.shape[1]))
    lo = np.zeros_like(hi)
    for xa in xs:
        for yb in ys:
            p = xa @ yb.T
            s = hi + p
            bb = s - hi
            lo += (hi - (s - bb)) + (p - bb)
            hi = s
    return hi, lo


def transform_exact(a: np.ndarray, q: np.ndarray) -> np.ndarray:
    """Q^T A Q to about double-double accuracy, rounded to FP64 and
    symmetrised like ``transform`` -- the reference for the error of A1."""
    th, tl = exact_matmul(np.asarray(a, dtype=np.float64), q)
    qt = np.ascontiguousarray(q.T)
    h1, l1 = exact_matmul(qt, th)
    h2, l2 = exact_matmul(qt, tl)
    a1 = h1 + (l1 + (h2 + l2))
    return 0.5 * (a1 + a1.T)


REFINE_TAU = 0.01          # pairs with |a_ij| > tau |a_jj - a_ii| are left to Jacobi
REFINE_MAX_ROWSUM = 0.25   # max_i sum_j |D_ij| (>= ||D||_2) is scaled down to at most this
REFINE_NS_STEPS = 5         # at most; fewer when ||D||_2 is small (refine_ns_count)


def refine_ns_count(rho: float) -> int:
    """Newton--Schulz steps that take Z = I + D (D antisymmetric, ||D||_2 <=
    rho <= 1/4) to orthogonality: the defect R = Z^T Z - I = D^T D starts at
    ||R|| <= rho^2 and one step maps r to 3/4 r^2 + 1/4 r^3 <= r^2, so k steps
    leave at most rho^(2^(k+1)); the count is the least k >= 1 with
    rho^(2^(k+1)) <= 2^-56, at most REFINE_NS_STEPS."""
    if rho <= 0.0:
        return 0
    bits = -np.log2(rho)                 # rho = 2^-bits, bits >= 2
    k = 1
    while k < REFINE_NS_STEPS and (2.0 ** (k + 1)) * bits < 56.0:
        k += 1
    return k


def refine_step(a1: np.ndarray, q: np.ndarray, tau: float = REFINE_TAU) -> Tuple[np.ndarray, np.ndarray]:
    """One first-order refinement of the preconditioned pair (A1, Q), an
    EXTENSION beyond the paper (a simplified step of Ogita and Aishima's
    iterative refinement for the symmetric eigenvalue problem, 2018): for
    A1 = diag(d) + E nearly diagonal, the first-order eigenvector correction
    is I + D with D_ij = e_ij / (d_j - d_i) (antisymmetric, D_ii = 0); pairs
    with |e_ij| > tau |d_j - d_i| (near-degenerate) get D_ij = 0 and are left
    to the Jacobi iteration.  D is scaled so that its largest absolute row
    sum (an upper bound of ||D||_2 for antisymmetric D) is at most 1/4, Z is
    I + D made orthogonal by Newton--Schulz (refine_ns_count(||D||) steps:
    4 from ||Z^T Z - I||_2 = ||D||_2^2 <= 1/16, fewer for a small D),
    and the pair becomes (Z^T A1 Z symmetrised, Q Z) -- an exact orthogonal
    similarity up to rounding, so the spectrum is unchanged."""
    a1 = np.asarray(a1, dtype=np.float64)
    d = np.diag(a1)
    delta = d[None, :] - d[:, None]            # d_j - d_i at (i, j)
    e = a1 - np.diag(d)
    keep = np.abs(e) <= tau * np.abs(delta)
    with np.errstate(divide="ignore", invalid="ignore"):
        dm = np.where(keep, e / np.where(keep, delta, 1.0), 0.0)
    np.fill_diagonal(dm, 0.0)
    nrm = np.max(np.sum(np.abs(dm), axis=1))
    if nrm == 0.0:
        return a1, np.asarray(q, dtype=np.float64)   # nothing to refine
    if nrm > REFINE_MAX_ROWSUM:
        dm = dm * (REFINE_MAX_ROWSUM / nrm)
    z = reorth_ns(np.eye(a1.shape[0]) + dm, refine_ns_count(min(nrm, REFINE_MAX_ROWSUM)))
    a2 = z.T @ (a1 @ z)
    return 0.5 * (a2 + a2.T), np.asarray(q, dtype=np.float64) @ z


def precondition(a: np.ndarray, q0: Optional[np.ndarray] = None, reorth: str = "ns",
                 ns_steps: int = 3, refine_steps: int = 0) -> Tuple[np.ndarray, np.ndarray]:
    """Sec. 2.1: returns (Q, A1) with Q the FP64-orthogonal preconditioner
    and A1 = Q^T A Q; refine_steps > 0 adds that many ``refine_step``
    (an extension beyond the paper)."""
    if q0 is None:
        q0 = q0_fp32(a)
    q = reorth_qr(q0) if reorth == "qr" else reorth_ns(q0, ns_steps)
    a1 = transform(a, q)
    for _ in range(refine_steps):
        a1, q = refine_step(a1, q)
    return q, a1


def solve(a: np.ndarray, pivot: str = "gap", tol: float = 1e-15, q0: Optional[np.ndarray] = None,
          reorth: str = "ns", ns_steps: int = 3, refine_steps: int = 0, **kw) -> Dict:
    """Preconditioned Jacobi: Sec. 2.1 preconditioner, then Algorithm 1 on
    A1 with V0 = Q, then the readout."""
    q, a1 = precondition(a, q0, reorth, ns_steps, refine_steps)
    r = jacobi(a1, q, pivot=pivot, tol=tol, **kw)
    w, v = readout(r["a"], r["v"])
    r.update({"w": w, "v_sorted": v, "q": q, "a1": a1})
    return r


def jacobi_many(mats, pivot: str = "gap", stop: str = "offdiag", tol: float = 1e-15,
                max_rot_per_n2: int = 25):
    """Algorithm 1 on independent problems (list of (n,n) arrays), threads
    over problems.  Returns (list of final A, list of V, rotations, status)."""
    ns = np.array([m.shape[0] for m in mats], dtype=np.int32)
    sizes = ns.astype(np.int64) ** 2
    off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    A = np.concatenate([np.ascontiguousarray(m, dtype=np.float64).ravel() for m in mats])
    V = np.concatenate([np.eye(int(m)).ravel() for m in ns])
    rots = np.zeros(len(mats), dtype=np.int64)
    st = np.zeros(len(mats), dtype=np.int32)
    lib().or_jacobi_many(len(mats), _ptr(ns), _ptr(off), _ptr(A), _ptr(off), _ptr(V),
                         PIVOTS[pivot], STOPS[stop], float(tol), int(max_rot_per_n2),
                         _ptr(rots), _ptr(st))
    outa = [A[o:o + s].reshape(m, m) for o, s, m in zip(off, sizes, ns)]
    outv = [V[o:o + s].reshape(m, m) for o, s, m in zip(off, sizes, ns)]
    return outa, outv, rots, st


# ----------------------------------------------------------------------------
# Alg. 2 with Sec. 2.1's SVD preconditioner: one-sided Jacobi SVD
# ----------------------------------------------------------------------------
def right_vectors_fp32(b: np.ndarray) -> np.ndarray:
    """Low-precision right singular vectors V_l of B (Sec. 2.1, SVD
    paragraph, u_l = single): LAPACK's FP32 SVD of fl32(B)."""
    _, _, vt = np.linalg.svd(np.asarray(b, dtype=np.float32), full_matrices=False)
    return np.ascontiguousarray(vt.T.astype(np.float32))


def column_norms(x: np.ndarray) -> np.ndarray:
    """||x_k||_2 of every column, each summed in row order after scaling by
    the exact power of two 2^-e, e = ilogb(max_r |x_rk|), so that squares
    neither overflow nor underflow."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros(x.shape[1])
    for k in range(x.shape[1]):
        m = np.max(np.abs(x[:, k]))
        if m == 0.0:
            continue
        e = int(np.frexp(m)[1]) - 1
        acc = 0.0
        for v in np.ldexp(x[:, k], -e):
            acc += v * v
        out[k] = np.ldexp(np.sqrt(acc), e)
    return out


def svd_jacobi(b: np.ndarray, pivot: str = "gap", tol: float = 1e-15, vl: Optional[np.ndarray] = None,
               precondition_vectors: bool = True, ns_steps: int = 3, **kw) -> Dict:
    """One-sided Jacobi SVD of B (m x n, m >= n) with the paper's pivoting
    (Alg. 2; Sec. 2.1's SVD paragraph).

    Preconditioner: V_l, the FP32 right singular vectors (``vl`` or
    ``right_vectors_fp32``), made orthogonal by Newton--Schulz: V.  Jacobi
    then runs on B1 = BV, whose columns are orthogonal up to O(u_l ||B||).
    As Sec. 2.1 prescribes, the pivot rule is applied to A = (BV)^T BV: each
    rotation (c, s) is the one that makes columns i, j of B1 orthogonal as
    far as A records their inner products, A is updated two-sided
    (A <- G^T A G, exactly Algorithm 1) and the same rotation multiplies the
    columns of V.  The rotated matrix B1 G_1 G_2 ... equals B V_final, which
    is formed once at the end; the singular values are its column norms,
    sorted descending, U its normalised columns.  Without the preconditioner
    V = I.  Returns sigma, U, V (columns in sigma's order), rotations,
    status and the final A.
    """
    b = np.asarray(b, dtype=np.float64)
    m, n = b.shape
    if precondition_vectors:
        if vl is None:
            vl = right_vectors_fp32(b)
        v0 = reorth_ns(vl, ns_steps)
    else:
        v0 = np.eye(n)
    b1 = b @ v0
    a = b1.T @ b1
    a = 0.5 * (a + a.T)
    r = jacobi(a, v0, pivot=pivot, tol=tol, **kw)
    bf = b @ r["v"]
    sig = column_norms(bf)
    order = np.argsort(-sig, kind="stable")
    sig = sig[order]
    v = r["v"][:, order]
    u = bf[:, order] / np.where(sig > 0, sig, 1.0)[None, :]
    r.update({"sigma": sig, "u": u, "v_sorted": v, "v0": v0, "a0": a})
    return r


def gap_rel_score(aii: float, ajj: float, aij: float) -> float:
    """Sec. 4.2's relative score (1/a_ii + 1/a_jj) L_ij for SPD matrices."""
    return lib().or_gap_rel_score(float(aii), float(ajj), float(aij))


def svd_onesided(b: np.ndarray, pivot: str = "gap_rel", tol: float = 1e-15,
                 max_rot: Optional[int] = None, seed: int = 0) -> Dict:
    """One-sided Jacobi SVD with the inner products recomputed from the
    rotated columns after every rotation (Alg. 2; Sec. 4.2's setting, no
    preconditioner); see ``or_svd_onesided``.  Returns sigma (descending,
    sqrt of the final Gram diagonal), U (normalised columns), V, rotations,
    status, and the final B and Gram matrix."""
    b = np.asarray(b, dtype=np.float64)
    m, n = b.shape
    bc = np.asfortranarray(b).copy(order="F")
    v = np.eye(n)                      # column k at v[:, k]: Fortran order
    v = np.asfortranarray(v)
    g = np.zeros((n, n))
    if max_rot is None:
        max_rot = 50 * n * (n - 1) // 2 + 1
    rot = ctypes.c_longlong(0)
    st = ctypes.c_int(0)
    lib().or_svd_onesided(bc.ctypes.data_as(ctypes.c_void_p), m, n, v.ctypes.data_as(ctypes.c_void_p),
                          PIVOTS[pivot], float(tol), int(max_rot), ctypes.c_uint64(seed), _ptr(g),
                          ctypes.byref(rot), ctypes.byref(st))
    sig_u = np.sqrt(np.maximum(np.diag(g), 0.0))
    order = np.argsort(-sig_u, kind="stable")
    sig = sig_u[order]
    u = bc[:, order] / np.where(sig > 0, sig, 1.0)[None, :]
    return {"sigma": sig, "u": u, "v": np.ascontiguousarray(v[:, order]), "rotations": int(rot.value),
            "status": int(st.value), "b": np.ascontiguousarray(bc), "g": g, "order": order}


def jacobi_multi(a1: np.ndarray, v0: Optional[np.ndarray] = None, pivot: str = "gap", stop: str = "offdiag",
                 tol: float = 1e-15, K: int = 8, ratio: float = 0.0, max_rot: Optional[int] = None,
                 check_every: Optional[int] = None) -> Dict:
    """The multi-pivot variant (see ``or_jacobi_multi``): up to K
    non-conflicting pivots per step, taken greedily from the K best row
    heads; K = 1 is Algorithm 1.  Returns the final matrix, V, rotations,
    steps and status."""
    a = np.array(a1, dtype=np.float64, order="C", copy=True)
    n = a.shape[0]
    v = np.eye(n) if v0 is None else np.array(v0, dtype=np.float64, order="C", copy=True)
    if max_rot is None:
        max_rot = 50 * n * (n - 1) // 2 + 1
    if check_every is None:
        check_every = max(n, 1)
    steps = ctypes.c_longlong(0)
    info = _Info()
    lib().or_jacobi_multi(_ptr(a), n, _ptr(v), PIVOTS[pivot], STOPS[stop], float(tol), int(max_rot),
                          int(check_every), int(K), float(ratio), ctypes.byref(steps), ctypes.byref(info))
    return {"a": a, "v": v, "rotations": int(info.rotations), "steps": int(steps.value),
            "status": int(info.status), "off_final": info.off_final, "norm_f": info.norm_f}
