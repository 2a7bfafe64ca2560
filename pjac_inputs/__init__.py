"""Seeded synthetic inputs for the preconditioned Jacobi eigensolver.

This module is shared by the CPU oracle (``oracle/``), the tests and the
benchmark.  It holds no arithmetic of the method itself: it only builds
symmetric matrices with a known spectrum, ``A = Q diag(lam) Q^T`` with ``Q``
Haar-orthogonal, and the workload descriptions (batched problem sizes,
serving arrival streams).

``A`` is formed from the exact product ``Q diag(lam) Q^T`` rounded once to
FP64.  The exact product is obtained with error-free transformations:
Dekker's TwoProduct for ``Q diag(lam)`` and the error-free matrix-product
splitting of Ozaki, Ogita, Oishi and Rump (2012) for the GEMM, whose slice
products are exact in FP64 and are summed in double-double (Knuth's TwoSum).
The eigenvalues of the rounded ``A`` then differ from ``lam`` by at most the
rounding of ``A`` (Weyl: <= u/2 * ||A||_F) plus the departure of the
floating-point ``Q`` from orthogonality.
"""
from __future__ import annotations

import dataclasses
import hashlib
import os
from typing import List, Optional, Sequence, Tuple

import numpy as np

__all__ = [
    "haar", "exact_sym_product", "sym_from_spectrum", "worked_example",
    "spectrum_clustered", "spectrum_cfg1", "spectrum_cfg2", "spectrum_cfg3",
    "spectrum_p1", "batched_workload", "serving_workload", "Problem",
    "config_problem", "exact_product", "svd_problem", "SvdProblem", "hilbert_cholesky",
]


# ----------------------------------------------------------------------------
# error-free building blocks (input construction only)
# ----------------------------------------------------------------------------
def _two_sum(a: np.ndarray, b: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Knuth's TwoSum: s + e == a + b exactly."""
    s = a + b
    bb = s - a
    e = (a - (s - bb)) + (b - bb)
    return s, e


def _veltkamp_split(a: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    c = a * 134217729.0  # 2**27 + 1
    hi = c - (c - a)
    return hi, a - hi


def _two_prod(a: np.ndarray, b: np.ndarray) -> Tuple[np.ndarray, np.ndarray]:
    """Dekker's TwoProduct: p + e == a * b exactly (no overflow assumed)."""
    p = a * b
    ah, al = _veltkamp_split(a)
    bh, bl = _veltkamp_split(b)
    e = ((ah * bh - p) + ah * bl + al * bh) + al * bl
    return p, e


def _ozaki_slices(x: np.ndarray, bits: int, nslices: int) -> List[np.ndarray]:
    """Split the rows of x into slices of at most `bits` significant bits
    relative to each row's largest magnitude (extraction by adding and
    subtracting a power of two), so that x == sum(slices) exactly."""
    rest = x.copy()
    out = []
    for _ in range(nslices):
        mu = np.max(np.abs(rest), axis=-1, keepdims=True)
        with np.errstate(divide="ignore"):
            e = np.where(mu > 0, np.ceil(np.log2(np.where(mu > 0, mu, 1.0))), 0.0)
        sigma = np.ldexp(np.ones_like(mu), (e + (53 - bits)).astype(np.int64))
        hi = (rest + sigma) - sigma
        hi = np.where(mu > 0, hi, 0.0)
        out.append(hi)
        rest = rest - hi
    if np.any(rest != 0):
        out.append(rest)
    return out


def exact_sym_product(q: np.ndarray, lam: np.ndarray) -> np.ndarray:
    """Return fl(Q diag(lam) Q^T): the exact product rounded to FP64.

    Works on a single (n, n) matrix.  The result is made exactly symmetric
    by mirroring its lower triangle.
    """
    q = np.ascontiguousarray(q, dtype=np.float64)
    lam = np.asarray(lam, dtype=np.float64)
    n = q.shape[0]
    # B = Q diag(lam) exactly as bh + bl
    bh, bl = _two_prod(q, lam[None, :])
    k = max(1, int(np.ceil(np.log2(max(n, 2)))))
    bits = (53 - k) // 2
    ns = int(np.ceil(53 / bits))
    bs = _ozaki_slices(bh, bits, ns)      # rows of B
    qs = _ozaki_slices(q, bits, ns)       # rows of Q == columns of Q^T
    hi = np.zeros((n, n))
    lo = np.zeros((n, n))
    for bsl in bs:
        for qsl in qs:
            p = bsl @ qsl.T               # exact: every partial sum fits in 53 bits
            hi, e = _two_sum(hi, p)
            lo = lo + e
    lo = lo + bl @ q.T                    # second-order part, FP64 accuracy suffices
    a = hi + lo
    a = np.tril(a) + np.tril(a, -1).T
    return a


def exact_product(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    """fl(X Y) for rectangular X (m x k) and Y (k x n): the exact product
    (Ozaki--Ogita--Oishi--Rump slices, summed in double-double with Knuth's
    TwoSum) rounded once to FP64."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.float64)
    k = x.shape[1]
    kk = max(1, int(np.ceil(np.log2(max(k, 2)))))
    bits = (53 - kk) // 2
    ns = int(np.ceil(53 / bits))
    xs = _ozaki_slices(x, bits, ns)
    ys = _ozaki_slices(np.ascontiguousarray(y.T), bits, ns)
    hi = np.zeros((x.shape[0], y.shape[1]))
    lo = np.zeros_like(hi)
    for xa in xs:
        for yb in ys:
            hi, e = _two_sum(hi, xa @ yb.T)
            lo = lo + e
    return hi + lo


@dataclasses.dataclass
class SvdProblem:
    b: np.ndarray            # (m, n) FP64
    sigma: np.ndarray        # the singular values it was built from, descending
    name: str


def svd_problem(m: int, n: int, sigma: np.ndarray, seed: int = 0) -> SvdProblem:
    """B = fl(U diag(sigma) V^T) with U the first n columns of a Haar (m x m)
    matrix and V Haar (n x n), the product exact before its one rounding."""
    rng = np.random.default_rng(seed)
    u = haar(m, rng)[:, :n]
    v = haar(n, rng)
    sig = np.asarray(sigma, dtype=np.float64)
    uh, ul = _two_prod(u, sig[None, :])
    b = exact_product(uh, v.T) + ul @ v.T
    return SvdProblem(b=b, sigma=np.sort(sig)[::-1], name="svd_%dx%d_s%d" % (m, n, seed))


def hilbert_cholesky(n: int) -> np.ndarray:
    """The Cholesky factor C_n of the Hilbert matrix H_n = C_n C_n^T in closed
    form (Sec. 4.2): c_ij = sqrt(2j-1) ((i-1)!)^2 / ((i+j-1)! (i-j)!) for
    i >= j (1-based), evaluated in 60-digit arithmetic and rounded once."""
    import mpmath
    c = np.zeros((n, n))
    with mpmath.workdps(60):
        for i in range(1, n + 1):
            for j in range(1, i + 1):
                v = mpmath.sqrt(2 * j - 1) * mpmath.factorial(i - 1) ** 2 / (
                    mpmath.factorial(i + j - 1) * mpmath.factorial(i - j))
                c[i - 1, j - 1] = float(v)
    return c


def haar(n: int, rng: np.random.Generator) -> np.ndarray:
    """Haar-distributed orthogonal Q: Householder QR of an N(0,1) matrix,
    columns sign-fixed so that diag(R) > 0."""
    g = rng.standard_normal((n, n))
    qm, r = np.linalg.qr(g)
    d = np.sign(np.diag(r))
    d[d == 0] = 1.0
    return qm * d[None, :]


def sym_from_spectrum(lam: np.ndarray, rng: np.random.Generator) -> np.ndarray:
    q = haar(len(lam), rng)
    return exact_sym_product(q, lam)


# ----------------------------------------------------------------------------
# spectra
# ----------------------------------------------------------------------------
def spectrum_clustered(n: int, nclusters: int, spread: float,
                       rng: np.random.Generator,
                       centres: Optional[np.ndarray] = None) -> np.ndarray:
    """n eigenvalues in `nclusters` clusters; centres U[-1,1] unless given;
    each eigenvalue offset by U[-spread, spread]."""
    if centres is None:
        centres = rng.uniform(-1.0, 1.0, nclusters)
    sizes = [n // nclusters + (1 if c < n % nclusters else 0) for c in range(nclusters)]
    lam = np.concatenate([centres[c] + rng.uniform(-spread, spread, sizes[c])
                          for c in range(nclusters)])
    return lam


def spectrum_cfg1(rng: np.random.Generator) -> np.ndarray:
    """n=32: 4 clusters of 8 around 1, 2, 3, 4, offsets U[-1e-6, 1e-6]."""
    return spectrum_clustered(32, 4, 1e-6, rng, centres=np.array([1.0, 2.0, 3.0, 4.0]))


def spectrum_cfg2(rng: np.random.Generator) -> np.ndarray:
    """n=1024: 32 clusters of 32, centres U[-1,1], spread 1e-8."""
    return spectrum_clustered(1024, 32, 1e-8, rng)


def spectrum_cfg3(rng: np.random.Generator, n: int = 4096) -> np.ndarray:
    """n=4096: half geometric 1 ... 1e-6, half in 64 clusters of 32 with
    spread 1e-10 and centres U[-1,1]."""
    h = n // 2
    geo = 10.0 ** (-6.0 * np.arange(h) / (h - 1))
    clu = spectrum_clustered(n - h, max(1, (n - h) // 32), 1e-10, rng)
    return np.concatenate([geo, clu])


def spectrum_p1(alpha: float, n: int = 1000) -> np.ndarray:
    """The clustered example of the paper's Sec. 4.1: 1 + exp(-alpha k) and
    2 + (k-1)/499 for k = 1..500 (n/2 of each)."""
    m = n // 2
    k = np.arange(1, m + 1, dtype=np.float64)
    return np.concatenate([1.0 + np.exp(-alpha * k), 2.0 + (k - 1.0) / (m - 1)])


def worked_example() -> np.ndarray:
    """The 4x4 block-diagonal example of the paper's introduction."""
    a = np.zeros((4, 4))
    a[0, 0], a[1, 1], a[0, 1], a[1, 0] = 1.0, 2.0, 1e-8, 1e-8
    a[2, 2], a[3, 3], a[2, 3], a[3, 2] = 1.0, 1.0 + 1e-10, 1e-9, 1e-9
    return a


# ----------------------------------------------------------------------------
# problems
# ----------------------------------------------------------------------------
@dataclasses.dataclass
class Problem:
    a: np.ndarray            # (n, n) FP64 symmetric
    lam: np.ndarray          # the spectrum it was built from, ascending
    name: str

    @property
    def n(self) -> int:
        return self.a.shape[0]

    @property
    def norm2(self) -> float:
        return float(np.max(np.abs(self.lam)))


def _cache_dir() -> Optional[str]:
    d = os.environ.get("PJAC_INPUT_CACHE")
    if d is None:
        d = os.path.join(os.path.expanduser("~"), ".cache", "pjac_inputs")
    try:
        os.makedirs(d, exist_ok=True)
    except OSError:
        return None
    return d


def _cached(key: str, build):
    d = _cache_dir()
    path = None
    if d is not None:
        path = os.path.join(d, hashlib.sha1(key.encode()).hexdigest()[:16] + ".npz")
        if os.path.exists(path):
            try:
                z = np.load(path)
                return z["a"], z["lam"]
            except Exception:
                pass
    a, lam = build()
    if path is not None:
        try:
            tmp = path + ".%d.tmp.npz" % os.getpid()
            np.savez(tmp, a=a, lam=lam)
            os.replace(tmp, path)
        except OSError:
            pass
    return a, lam


def config_problem(cfg: str, seed: int = 0, n: Optional[int] = None) -> Problem:
    """Build one of the named single-problem workloads.

    cfg1: n=32, 4 clusters x 8 (centres 1..4, spread 1e-6)
    cfg2: n=1024, 32 clusters x 32 (centres U[-1,1], spread 1e-8)
    cfg3: n=4096, half geometric 1..1e-6, half 64 clusters x 32 (spread 1e-10)
    p1a / p1b: the paper's Sec. 4.1 example with alpha = 0.01 / 1 (n=1000)
    The random stream draws the Gaussian matrix for Q first, then the spectrum.
    `n` overrides the order of cfg2/cfg3 (same recipe, smaller size).
    """
    def build():
        rng = np.random.default_rng(seed)
        if cfg == "cfg1":
            q = haar(32, rng)
            lam = spectrum_cfg1(rng)
        elif cfg == "cfg2":
            m = n or 1024
            q = haar(m, rng)
            lam = spectrum_clustered(m, max(1, m // 32), 1e-8, rng)
        elif cfg == "cfg3":
            m = n or 4096
            q = haar(m, rng)
            lam = spectrum_cfg3(rng, m)
        elif cfg in ("p1a", "p1b"):
            m = n or 1000
            q = haar(m, rng)
            lam = spectrum_p1(0.01 if cfg == "p1a" else 1.0, m)
        else:
            raise ValueError(cfg)
        a = exact_sym_product(q, lam)
        return a, np.sort(lam)

    a, lam = _cached("v1|%s|%d|%s" % (cfg, seed, n), build)
    return Problem(a=a, lam=lam, name=cfg if n is None else "%s_n%d" % (cfg, n))


def small_clustered_problem(n: int, rng: np.random.Generator, kind: str) -> Problem:
    """One problem of the batched workload: clustered (n/8 clusters, spread
    1e-8, centres U[-1,1]) or uniform U[-1,1]."""
    q = haar(n, rng)
    if kind == "clustered":
        lam = spectrum_clustered(n, max(1, n // 8), 1e-8, rng)
    else:
        lam = rng.uniform(-1.0, 1.0, n)
    a = exact_sym_product(q, lam)
    return Problem(a=a, lam=np.sort(lam), name="%s_n%d" % (kind, n))


def batched_sizes(count: int = 10000, seed: int = 1, nmin: int = 16,
                  nmax: int = 256) -> Tuple[np.ndarray, np.ndarray]:
    """Sizes n = round(exp(U[ln nmin, ln nmax])) and kinds (0 clustered,
    1 uniform, 50/50) of the batched workload."""
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(np.log(nmin), np.log(nmax), count))).astype(np.int64)
    kinds = rng.integers(0, 2, count)
    return ns, kinds


def batched_workload(count: int = 10000, seed: int = 1, nmin: int = 16,
                     nmax: int = 256) -> List[Problem]:
    """The batched workload: `count` independent problems."""
    ns, kinds = batched_sizes(count, seed, nmin, nmax)

    def build():
        rng = np.random.default_rng(seed + 1000)
        mats = [small_clustered_problem(int(m), rng, "clustered" if k == 0 else "uniform")
                for m, k in zip(ns, kinds)]
        flat_a = np.concatenate([p.a.ravel() for p in mats])
        flat_l = np.concatenate([p.lam for p in mats])
        return flat_a, flat_l

    flat_a, flat_l = _cached("v1|batched|%d|%d|%d|%d" % (count, seed, nmin, nmax), build)
    out = []
    oa = ol = 0
    for m, k in zip(ns, kinds):
        m = int(m)
        a = flat_a[oa:oa + m * m].reshape(m, m)
        lam = flat_l[ol:ol + m]
        oa += m * m
        ol += m
        out.append(Problem(a=a, lam=lam, name="%s_n%d" % ("clustered" if k == 0 else "uniform", m)))
    return out


SERVE_SIZES = (64, 128, 256, 512, 1024, 2048)
SERVE_PROBS = (0.30, 0.25, 0.20, 0.12, 0.08, 0.05)


def serving_workload(count: int = 20000, rate: float = 2000.0, seed: int = 2,
                     pool_per_size: int = 4,
                     sizes: Sequence[int] = SERVE_SIZES,
                     probs: Sequence[float] = SERVE_PROBS):
    """The serving stream: Poisson arrivals at `rate` per second (exponential
    inter-arrival times), sizes drawn from `sizes` with `probs`, clustered
    spectra as in the batched workload.  Matrices are drawn from a pool of
    `pool_per_size` distinct problems per size (20,000 distinct n<=2048
    matrices would not fit in host memory); request r uses pool entry
    r mod pool_per_size of its size.

    Returns (arrival_times_s, size_index_per_request, pool) where pool[s] is
    the list of Problems of size sizes[s].
    """
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / rate, count)
    t = np.cumsum(gaps) - gaps[0]
    sidx = rng.choice(len(sizes), size=count, p=np.asarray(probs) / np.sum(probs))
    prng = np.random.default_rng(seed + 1000)
    pool = []
    for m in sizes:
        pool.append([small_clustered_problem(int(m), prng, "clustered") for _ in range(pool_per_size)])
    return t, sidx, pool
