/*
 * pjac -- preconditioned Jacobi eigensolver with perturbation-inspired
 * (spectral-gap-weighted) pivoting, for NVIDIA B300 (sm_103a).
 *
 * Method: Shao & Nakatsukasa, "Accelerating preconditioned Jacobi methods
 * via perturbation-inspired pivoting".  A symmetric A is first brought close
 * to diagonal by a mixed-precision preconditioner (Sec. 2.1): an FP32
 * spectral decomposition Q0 ~ eig(fl32(A)), reorthogonalised to an
 * FP64-orthogonal Q, then A1 = Q^T A Q.  Jacobi's method (Algorithm 1,
 * Sec. 2) then annihilates the off-diagonal entries of A1 with one of three
 * pivot rules: the gap-weighted rule of Eq. (1.1),
 *     L_ij = 2|a_ij|^2 / (|a_ii-a_jj| + sqrt(|a_ii-a_jj|^2 + 4|a_ij|^2)),
 * Jacobi's classical greedy argmax|a_ij|, or cyclic sweeps (Sec. 1).  The
 * eigenvalues are the final diagonal; the eigenvectors are V = Q * prod G.
 *
 * Conventions for every call:
 *   - Matrices are DEVICE pointers to FP64 column-major storage with a
 *     leading dimension (>= n).  A symmetric input is read in full; the
 *     caller must pass an exactly symmetric matrix (A[i,j] == A[j,i]).
 *   - The caller owns every buffer it passes.  The handle owns its
 *     workspace (device memory sized on first use, grown on demand).
 *   - Calls are asynchronous on the given stream unless stated otherwise.
 *   - Every call returns a pjac_status; PJAC_OK is 0.  On failure a message
 *     is available from pjac_last_error() (per thread).
 *   - Sizes: 1 <= n <= PJAC_MAX_N.  n == 1 is trivial (W = A, V = 1).
 *   - Index pairs (i,j) are 0-based with i < j.
 */
#ifndef PJAC_H
#define PJAC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PJAC_MAX_N 16384

/* Status codes. */
typedef enum {
    PJAC_OK = 0,
    PJAC_PENDING = 1,      /* serving: request not finished yet */
    PJAC_EINVAL = -1,      /* bad argument (n, leading dimension, pointer, NaN/Inf input) */
    PJAC_ENOMEM = -2,      /* device allocation failed */
    PJAC_EAGAIN = -3,      /* serving: queue full, retry later */
    PJAC_ENOCONV = -4,     /* rotation budget reached; W, V are valid but not converged */
    PJAC_ETIMEOUT = -5,    /* a device-side time budget ran out; results partial */
    PJAC_ECUDA = -6,       /* a CUDA runtime call failed */
    PJAC_ENOTIMPL = -7     /* option not available */
} pjac_status;

/* Pivot rules (Sec. 1, Eq. (1.1)). */
typedef enum {
    PJAC_PIVOT_GAP = 0,     /* argmax L_ij of Eq. (1.1) */
    PJAC_PIVOT_GREEDY = 1,  /* argmax |a_ij| (Jacobi 1846) */
    PJAC_PIVOT_CYCLIC = 2,  /* row-cyclic sweeps (0,1),(0,2),...,(n-2,n-1) */
    /* Randomized comparator (Sec. 4.2): every pair equally likely.  Step k
     * takes z = SplitMix64 output function of (seed + (k+1)*0x9e3779b97f4a7c15)
     * (Steele, Lea and Flood's generator, used counter-based), i = (z mod 2^32)
     * mod n, j' = (z div 2^32) mod (n-1), j = j' + [j' >= i], ordered.  A draw
     * with a_ij == 0 applies the identity and still counts as a rotation.
     * Off-diagonal stop only. */
    PJAC_PIVOT_RANDOM = 3,
    /* Sec. 4.2's relative score (1/a_ii + 1/a_jj) L_ij for positive definite
     * matrices; pjac_svd_onesided only. */
    PJAC_PIVOT_GAP_REL = 4
} pjac_pivot;

/* Stopping rules. */
typedef enum {
    /* off(A1) = sqrt(sum_{i!=j} a_ij^2) <= tol * ||A1||_F, tested every n
     * rotations (gap, greedy) or before every sweep (cyclic). */
    PJAC_STOP_OFFDIAG = 0,
    /* Theorem 1 (Sec. 3.1): stop when max L_ij <= tol*||A1||_F/(2n(n-1)),
     * which guarantees |lambda_k - a_kk| <= tol*||A1||_F.  Eigenvalues only:
     * V is then NOT accurate to working precision. Gap rule only. */
    PJAC_STOP_LIBOUND = 1
} pjac_stop;

/* How A1 = Q^T A Q and the Newton--Schulz products are formed. */
typedef enum {
    PJAC_TRANSFORM_SPLIT_BF16 = 0, /* tensor cores: BF16 slices, FP32 accumulate, FP64 recombine */
    PJAC_TRANSFORM_FP64 = 1        /* plain FP64 products on the CUDA cores */
} pjac_transform;

typedef struct {
    pjac_stop stop;          /* default PJAC_STOP_OFFDIAG */
    double tol;              /* default 1e-15 */
    int64_t max_rotations;   /* 0: 50 * n(n-1)/2 */
    int64_t check_every;     /* 0: n (off-mass test period, gap/greedy) */
    pjac_transform transform;/* default PJAC_TRANSFORM_SPLIT_BF16 */
    int ns_steps;            /* Newton--Schulz steps, 0: 3 */
    int cluster_size;        /* CTAs cooperating on one single problem; 0: automatic */
    double time_budget_s;    /* device-side time budget per solve, 0: 600 s */
    /* 1: no preconditioner -- Algorithm 1 runs directly on A with V0 = I, as
     * in the paper's Sec. 4.2 experiment (a global orthogonal preconditioner
     * would spoil the relative accuracy sought there).  0 (default): the
     * Sec. 2.1 preconditioner runs first.  Applies to pjac_solve,
     * pjac_solve_batched and the serving calls. */
    int no_precondition;
    uint64_t seed;           /* PJAC_PIVOT_RANDOM's seed, default 0 */
    /* EXTENSION beyond the paper, default 0: first-order refinement steps
     * applied to (A1, Q) after the Sec. 2.1 preconditioner, each a
     * simplified step of Ogita and Aishima's iterative refinement for the
     * symmetric eigenproblem: with A1 = diag(d) + E, D_ij = e_ij/(d_j - d_i)
     * for pairs with |e_ij| <= 0.01 |d_j - d_i| (the rest are left to
     * Jacobi), D scaled so its largest absolute row sum is <= 1/4, Z = I + D
     * made orthogonal by Newton--Schulz steps, then A1 <- Z^T A1 Z,
     * Q <- Q Z.  The step count is the least k >= 1 with
     * rho^(2^(k+1)) <= 2^-56 for the row-sum bound rho of the scaled D, at
     * most 5, read back from the device (a step with D = 0 is skipped); the
     * serving lanes, which must not wait on the host, take 5.  Two products
     * per Newton--Schulz step and three more per refinement step; it
     * resolves the well-separated pairs on the tensor cores and leaves fewer
     * rotations to the Jacobi iteration.  0..8. */
    int refine_steps;
    /* Most sweeps of the parallel-order FP32 Jacobi pass of the low-precision
     * eigenbasis (it stops earlier once its off-diagonal mass stagnates);
     * 0: 40. */
    int fp32_sweeps;
    /* Multi-pivot variant (the parallel direction Sec. 5 names as future
     * work), for the gap and greedy rules, n <= 4096: 0 or 1 = off; K >= 2
     * (<= 64): every step ranks the rows by their best score, walks the K
     * best rows in order and accepts each head whose score is positive, at
     * least multi_ratio times the first one's and whose indices are still
     * free, then applies the accepted rotations in that order (they act on
     * disjoint index pairs).  K = 1 is Algorithm 1.  One CTA per problem,
     * exact FP64 scores. */
    int multi_pivot;
    double multi_ratio;      /* default 0 */
    /* pjac_solve_batched: 1 (default) tunes, per order bucket (n < 32, < 64,
     * < 128, <= 256, > 256) and pivot rule, the refinement steps (1..3) and
     * the FP32 sweep cap (12 or 40) on the first call outside a stream
     * capture that meets the bucket, by timing up to 32 of the call's own
     * problems with every candidate; the choice is cached in the handle.
     * 0: refinement 1 + refine_steps, sweep cap fp32_sweeps (or 40). */
    int autotune;
} pjac_opts;

/* Per-solve report. */
typedef struct {
    int64_t rotations;       /* rotations applied */
    double sweeps;           /* rotations / (n(n-1)/2), or sweeps for cyclic */
    double off_rel;          /* off(A_final) / ||A1||_F */
    double max_score;        /* last selected pivot score (L_ij or |a_ij|) */
    int32_t status;          /* pjac_status of this solve */
    int32_t n;
    float ms_precond;        /* FP32 diagonalisation + reorthogonalisation */
    float ms_transform;      /* Q^T A Q */
    float ms_jacobi;         /* Jacobi iteration + readout */
    int64_t steps;           /* selection steps (== rotations except for the multi-pivot variant) */
} pjac_info;

typedef struct pjac_handle pjac_handle;

/* Default options (stop OFFDIAG, tol 1e-15, split-BF16 transform, 3 NS steps). */
void pjac_default_opts(pjac_opts* o);

/* Create a handle bound to the current CUDA device.  o may be NULL.
 * Errors: PJAC_EINVAL (h NULL), PJAC_ECUDA. */
int pjac_create(pjac_handle** h, const pjac_opts* o);
/* Release the handle and its workspace (synchronises the device). */
int pjac_destroy(pjac_handle* h);
/* Replace the handle's options. */
int pjac_set_opts(pjac_handle* h, const pjac_opts* o);

/*
 * Mixed-precision preconditioner (Sec. 2.1).
 *   A   [in]  n x n symmetric, lda >= n.  Not modified.
 *   Q0  [in]  optional n x n FP32 approximate eigenvectors (column-major,
 *             leading dimension n).  NULL: computed on the device by an FP32
 *             parallel-order Jacobi diagonalisation of fl32(A).
 *   Q   [out] n x n FP64 orthogonal to working precision (Newton--Schulz
 *             X <- X(3I - X^T X)/2 from X = Q0), ldq >= n.
 *   A1  [out] Q^T A Q symmetrised ((A1 + A1^T)/2), lda1 >= n.
 * Errors: PJAC_EINVAL, PJAC_ENOMEM, PJAC_ECUDA.
 */
int pjac_precondition(pjac_handle* h, const double* A, int n, int lda, const float* Q0,
                      double* Q, int ldq, double* A1, int lda1, void* stream);

/*
 * The low-precision spectral decomposition of Sec. 2.1 on its own (the first
 * step of the preconditioner, u_l = single precision as in Sec. 4): the FP32
 * eigenvector estimate Q0 of fl32(A) that pjac_precondition computes when it
 * is given no Q0.  Computed on the device by a parallel-order FP32 Jacobi
 * pass on fl32(A), a Newton--Schulz step pair in working precision and a
 * refinement pass of the same FP32 Jacobi on X^T fl32(A) X; the result is
 * rounded to FP32.  Any Q0 with ||Q0^T Q0 - I|| = O(n u_32) and
 * off(Q0^T fl32(A) Q0) = O(n u_32 ||A||) serves the preconditioner.
 *   A   [in]  n x n symmetric, lda >= n.  Not modified.
 *   Q0  [out] n x n FP32, column-major, ldq0 >= n (column k: eigenvector
 *             estimate; the columns are in no particular order).
 * Synchronises the stream.  Errors: PJAC_EINVAL (bad sizes, NaN/Inf or
 * asymmetric input), PJAC_ENOMEM, PJAC_ETIMEOUT, PJAC_ECUDA.
 */
int pjac_eig_lowprec(pjac_handle* h, const double* A, int n, int lda, float* Q0, int ldq0, void* stream);

/*
 * Working-precision product C = alpha op(A) op(B) + beta C, computed the way
 * the preconditioner of Sec. 2.1 computes its products (the Newton--Schulz
 * steps and Q^T A Q), with the handle's transform option:
 *   PJAC_TRANSFORM_SPLIT_BF16: the operands are cut into 6-bit (5-bit for
 *     k > 4227) digit slices scaled per row of op(A) and per column of
 *     op(B); slice products run on the tensor cores in BF16 with exact FP32
 *     accumulation and are summed exactly in 64-bit fixed point (Ozaki, Ogita,
 *     Oishi and Rump's error-free splitting).  Error per entry at most
 *     |alpha| 2^(e_i+f_j) (k (S+3) 2^(-bS) + T 2^-(2b+38)) + 2^-53 |C_ij|,
 *     where 2^(e_i-1) <= max_l |op(A)_il| < 2^e_i, likewise f_j for op(B)'s
 *     column j, b S = 54 (b = 6, S = 9) or 55 (b = 5, S = 11), and T = 17
 *     (b = 6) or 30 (b = 5) slice products are rounded to 37 fractional bits
 *     in the fixed-point sum.
 *   PJAC_TRANSFORM_FP64: plain FP64 products on the CUDA cores.
 * All matrices are FP64, column-major, in device memory.
 *   transa, transb  0: op(X) = X, 1: op(X) = X^T.
 *   m, n, k         op(A) is m x k, op(B) is k x n, C is m x n; 1..PJAC_MAX_N.
 *   lda >= rows of A as stored (m, or k if transposed); likewise ldb; ldc >= m.
 *   beta == 0: C is not read.  C must not overlap A or B.  Entries of A
 *   and B must be finite.
 * Synchronises the stream (it reads the product's device status).
 * Errors: PJAC_EINVAL, PJAC_ENOMEM, PJAC_ENOTIMPL (k > 17458 with the split
 * product), PJAC_ETIMEOUT (a wait inside the tensor-core pipeline timed
 * out; C is unspecified), PJAC_ECUDA.
 */
int pjac_product(pjac_handle* h, int transa, int transb, int m, int n, int k, double alpha,
                 const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
                 void* stream);

/*
 * The products of Sec. 2.1 whose exact value is symmetric: X^T X in the
 * Newton--Schulz steps and X^T (A X) in the transform (n x n results).
 * Same arguments as pjac_product with m = n; the caller states that
 * op(A) op(B) is symmetric in exact arithmetic.  With the split product only
 * the 128 x 128 output tiles on and above the diagonal are computed and
 * entry (i, j), i <= j, is written to both (i, j) and (j, i): about half the
 * work, and C is exactly symmetric.  Each written pair carries the error
 * bound of pjac_product for entry (i, j).  With PJAC_TRANSFORM_FP64 the full
 * product is formed and then averaged with its transpose.  beta != 0 uses
 * C(i, j) and C(j, i) each for its own entry.
 * Synchronises the stream.  Errors as pjac_product.
 */
int pjac_product_symmetric(pjac_handle* h, int transa, int transb, int n, int k, double alpha,
                           const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
                           void* stream);

/*
 * Full solve: preconditioner, then Algorithm 1 on A1 with V0 = Q, then the
 * readout (W ascending, V's columns in the same order).
 *   A   [in]  n x n symmetric, not modified.
 *   W   [out] n eigenvalues ascending.
 *   V   [out] n x n eigenvectors (column k for W[k]), ldv >= n.
 *   info [out, host, nullable] filled after the solve; this call
 *        synchronises the stream when info != NULL.
 * Returns PJAC_OK, PJAC_ENOCONV, PJAC_ETIMEOUT or an error.
 */
int pjac_solve(pjac_handle* h, const double* A, int n, int lda, pjac_pivot pivot, double tol,
               double* W, double* V, int ldv, pjac_info* info, void* stream);

/*
 * Algorithm 1 on an already preconditioned A1 (overwritten with the final,
 * nearly diagonal matrix).  V0 [in] n x n (NULL: identity), ldv0 >= n;
 * V [out] the accumulated V0 * prod G with columns sorted like W.
 * Same returns as pjac_solve.
 */
int pjac_solve_preconditioned(pjac_handle* h, double* A1, int n, int lda1, const double* V0,
                              int ldv0, pjac_pivot pivot, double tol, double* W, double* V,
                              int ldv, pjac_info* info, void* stream);

/*
 * Allocation-free variant of pjac_solve_preconditioned.  The paper has no
 * counterpart: this entry point exists for callers that must not allocate
 * device memory at solve time -- a process that reserves its whole device
 * memory budget when it starts (its own allocator then holds all free
 * memory, so a cudaMalloc during a solve would fail or fragment it), or a
 * plug-in that runs inside a host application without access to that
 * application's allocator.  It needs no handle and allocates nothing: its
 * scratch lives in a fixed array of PJAC_NOALLOC_SCRATCH_BYTES in every
 * GPU's memory, kept there until the process exits.
 *   Arguments, layouts and results are those of pjac_solve_preconditioned
 *   with the default options (off-diagonal stop at tol).
 *   n must not exceed PJAC_NOALLOC_MAX_N; larger n returns PJAC_EINVAL.
 *   First call on a device: it looks up the array's device address and
 *   loads the kernels it launches.  Under CUDA's lazy module loading these
 *   are the moments the array and the kernels' code take device memory, so
 *   make the first call on each device (any small valid input will do)
 *   BEFORE reserving that device's memory; later calls take none.
 *   All calls share the one array: calls whose work overlaps on the GPU
 *   (other streams, other host threads) race on it and must be serialised
 *   by the caller.  The call synchronises the stream and copies its solve
 *   record to the host, so it cannot be recorded into a CUDA graph.
 */
#define PJAC_NOALLOC_MAX_N 512
#define PJAC_NOALLOC_SCRATCH_BYTES ((size_t)PJAC_NOALLOC_MAX_N * PJAC_NOALLOC_MAX_N * 8 + 8192)
int pjac_solve_preconditioned_noalloc(double* A1, int n, int lda1, const double* V0, int ldv0,
                                      pjac_pivot pivot, double tol, double* W, double* V, int ldv,
                                      pjac_info* info, void* stream);

/*
 * Batched form: nb independent problems of order n[p] (2 <= n[p] <= 1024)
 * packed in one device buffer.  Host arrays n, a_off, w_off, v_off give each
 * problem's order and its offsets (in doubles) into A, W and V; problem p is
 * column-major with leading dimension n[p].  A is not modified.  Each problem
 * is preconditioned and solved like pjac_solve.  infos [out, DEVICE] nb
 * records, written by the device.
 * Graph capture: called on a capturing stream, the call only records its
 * copies and kernels (no host synchronisation) and hands its pinned staging
 * buffer to the graph, which replays the same batch (the host arrays are
 * read at capture time).  The graph stays valid while the handle lives and
 * no later batched call on the handle needs a larger device workspace.
 * Outside a capture the call synchronises the stream once before it stages
 * the descriptors.
 * Returns PJAC_OK once the work is enqueued; per-problem status is in infos.
 */
int pjac_solve_batched(pjac_handle* h, int nb, const int* n, const int64_t* a_off,
                       const double* A, const int64_t* w_off, double* W, const int64_t* v_off,
                       double* V, pjac_pivot pivot, double tol, pjac_info* infos, void* stream);

/*
 * One-sided Jacobi SVD with the paper's pivoting (Alg. 2) and the
 * low-precision right-singular-vector preconditioner (Sec. 2.1, SVD
 * paragraph).  B = U diag(S) V^T.
 *   B   [in]  m x n, column-major, ldb >= m, 1 <= n <= m <= PJAC_MAX_N,
 *             m <= 17458 with the split-BF16 products.  Not modified.
 *   Vl  [in]  optional n x n FP32 right singular vectors of fl32(B)
 *             (column-major, ldvl >= n).  NULL: computed on the device as
 *             the FP32 eigenbasis of B^T B (see pjac_eig_lowprec).  Ignored
 *             with opts.no_precondition (then V0 = I).
 *   S   [out] n singular values, descending.
 *   U   [out, nullable] m x n left singular vectors, ldu >= m (a column is
 *             zero where its singular value is zero).
 *   V   [out, nullable] n x n right singular vectors, ldv >= n.
 * Steps: V0 = Newton--Schulz(Vl); B1 = B V0; A = B1^T B1 (symmetrised);
 * Algorithm 1 on A with the given pivot rule and stop (each rotation makes
 * columns i, j of B1 orthogonal as far as A records their inner products;
 * A is updated two-sided and V0's columns rotated: the pivot rule sees
 * (BV)^T BV as Sec. 2.1 prescribes); then the rotated B V is formed with
 * one product, its column norms (scaled by a power of two) are the singular
 * values.  Products use the handle's transform option.  Accuracy: absolute,
 * about u ||B||^2 / sigma for each sigma (the Gram matrix is formed once).
 * Synchronises the stream when info != NULL.  Returns like pjac_solve.
 */
int pjac_svd(pjac_handle* h, const double* B, int m, int n, int ldb, const float* Vl, int ldvl,
             pjac_pivot pivot, double tol, double* S, double* U, int ldu, double* V, int ldv, pjac_info* info,
             void* stream);

/*
 * One-sided Jacobi SVD for relative accuracy (Alg. 2 in the setting of
 * Sec. 4.2: no preconditioner, the pivot matrix G = B^T B of the CURRENT
 * columns).  G is formed once and, after each rotation (i,j), its rows and
 * columns i and j are recomputed from the rotated columns, every entry a dot
 * product summed in row order with fused multiply-adds.  The rotation is the
 * one that makes columns i, j orthogonal as G records them.  Pivot rules:
 *   PJAC_PIVOT_GAP_REL  Sec. 4.2's (1/g_ii + 1/g_jj) L_ij; stop when the
 *                       largest score is <= tol (a relative bound),
 *   PJAC_PIVOT_GAP      Eq. (1.1) on G; stop at largest score <= tol ||G0||_F,
 *   PJAC_PIVOT_GREEDY   |g_ij|; stop at largest score <= tol ||G0||_F,
 *   PJAC_PIVOT_RANDOM   uniform pairs (Sec. 4.2's comparator); stop tested
 *                       every n draws on the GAP_REL scores.
 * Rotation budget: opts.max_rotations (0: 50 n(n-1)/2) -> PJAC_ENOCONV.
 *   B   [in]  m x n, ldb >= m, 2 <= n <= 1024, n <= m <= PJAC_MAX_N; not
 *             modified.
 *   S   [out] n singular values sqrt(g_kk) of the final G, descending.
 *   U   [out, nullable] m x n, ldu >= m: the rotated columns / S.
 *   V   [out, nullable] n x n, ldv >= n: the accumulated rotations.
 * One CTA runs the iteration (the dependent chain of this small, accurate
 * form); O(mn) work per rotation.  Synchronises the stream when info != NULL.
 */
int pjac_svd_onesided(pjac_handle* h, const double* B, int m, int n, int ldb, pjac_pivot pivot, double tol,
                      double* S, double* U, int ldu, double* V, int ldv, pjac_info* info, void* stream);

/* The autotuner's choice for an order bucket (0: n < 32, 1: < 64, 2: < 128,
 * 3: <= 256, 4: > 256) and pivot rule of the batched form on h: refinement
 * steps, FP32 sweep cap and the tuning sample's solves/s.  PJAC_EINVAL when
 * that bucket has not been tuned on h. */
int pjac_batched_tuning(pjac_handle* h, int bucket, pjac_pivot pivot, int* refine, int* fp32_sweeps,
                        float* sample_solves_per_s);

/* Device milliseconds of the five stages of the last pjac_solve_batched call
 * made on h outside a stream capture: ms[0] FP32 eigenbases (or the copy-in
 * without the preconditioner), ms[1] Newton--Schulz and Q^T A Q, ms[2] the
 * refinement step(s), ms[3] the Jacobi iteration, ms[4] readout and report.
 * Synchronises on that call's completion.  Errors: PJAC_EINVAL when no such
 * call was made, PJAC_ECUDA. */
int pjac_batched_stage_ms(pjac_handle* h, float* ms);

/* ---------------------------------------------------------------------
 * Serving: continuous batching of eigenproblems of mixed sizes.  Requests
 * are admitted while their device footprint fits the memory budget and a
 * slot is free; admitted requests run concurrently on the device; finished
 * slots are recycled immediately for waiting requests.  Each slot has one
 * stream; an eighth of them (at least one, from two slots up) run at the
 * device's highest stream priority, the rest at its lowest.  Waiting
 * requests of order <= 256 go first, as one micro-batch, preferably on a
 * high-priority slot; otherwise the oldest larger request takes a
 * low-priority slot alone.  Larger requests together hold at most 7/8 of
 * the device's SMs, so small ones always find room, and the oldest larger
 * request is passed over by at most four micro-batches.
 * Streams beyond the CUDA_DEVICE_MAX_CONNECTIONS hardware queues (default
 * 8) share a queue, where work runs in submission order and a micro-batch
 * can wait behind another slot's large solve: set that variable to 32
 * before the process's first CUDA call and keep max_slots <= 32.
 * pjac_serve_create loads every kernel of the library on the current
 * device (under lazy module loading a first launch would load it, and that
 * load can wait for the solves already running).
 * ------------------------------------------------------------------- */
typedef struct pjac_server pjac_server;

typedef struct {
    int max_slots;            /* lanes (streams) running admitted work, <= 64; 0: 8 */
    int max_queue;            /* waiting (not yet admitted) requests, 0: 1 << 16 */
    size_t hbm_budget_bytes;  /* device bytes for admitted requests, 0: 8 GiB */
    pjac_opts solver;         /* options of every solve */
} pjac_serve_opts;

void pjac_serve_default_opts(pjac_serve_opts* o);
int pjac_serve_create(pjac_server** s, const pjac_serve_opts* o);
/* Waits for in-flight work, then frees everything. */
int pjac_serve_destroy(pjac_server* s);

/*
 * Submit one request (non-blocking).  A [in, HOST] n x n symmetric,
 * column-major, lda >= n; copied before the call returns.  W [out, HOST]
 * n doubles, V [out, HOST, nullable] n x n with ldv >= n: written when the
 * request completes and must stay valid until pjac_serve_poll returns a
 * terminal status for the ticket.  Returns PJAC_EAGAIN when the waiting
 * queue is full.
 */
int pjac_serve_submit(pjac_server* s, const double* A, int n, int lda, pjac_pivot pivot,
                      double tol, double* W, double* V, int ldv, uint64_t* ticket);

/* Progress the server and report on one ticket: PJAC_PENDING while queued
 * or running, else the request's final status (info filled, nullable). A
 * ticket can be polled to completion once. */
int pjac_serve_poll(pjac_server* s, uint64_t ticket, pjac_info* info);

/* Progress the server without asking about a ticket; returns the number of
 * requests still queued or running. */
int pjac_serve_progress(pjac_server* s);

/* Latency statistics (milliseconds from submit to completion) over the
 * completed requests so far. */
typedef struct {
    int64_t completed;
    double p50_ms, p99_ms, max_ms, mean_ms;
    double solves_per_s;      /* completed / (last completion - first submission) */
    int64_t peak_inflight;
    size_t peak_hbm_bytes;
    int64_t launches;         /* kernel launches of this library enqueued so far */
} pjac_serve_stats;
int pjac_serve_get_stats(pjac_server* s, pjac_serve_stats* st);

/* Number of kernel launches of this library that one pjac_solve of size n
 * makes with the handle's current options (preconditioner products,
 * element-wise steps, the Jacobi kernel, the readout).  With refine_steps
 * > 0 the Newton--Schulz steps of each refinement step depend on the size
 * of its correction: the count is that of the handle's last solve of order
 * n, or an upper bound before there is one.  A diagnostic for launch
 * accounting; returns -1 when h is NULL or n is out of range. */
int pjac_solve_launch_count(pjac_handle* h, int n);

/* The plan of the split-BF16 product of shape m x n x k (host only; no
 * device work, no handle): how the digit-slice pairs are scheduled.
 *   symmetric  1: the plan of pjac_product_symmetric (m == n).
 *   sms        SMs the plan is made for (0: the current device's count, 148
 *              when there is none).
 *   info [out, host, 6 ints] b (bits per digit), S (slices), units (blocks of
 *              up to 2 x 2 slice pairs sharing their operand tiles), splits
 *              (CTAs that share one output tile's pairs), CTAs of the
 *              product kernel, pairs in all (the pairs (s, t) with s + t < S).
 *   pairs [out, host, nullable] the pairs in launch order as quadruples
 *              (s, t, unit, split), at most pairs_cap of them.
 * A diagnostic of the schedule.  PJAC_EINVAL for invalid sizes (every k up
 * to PJAC_MAX_N has a plan: 5-bit digits reach k = 17458). */
int pjac_product_plan(int m, int n, int k, int symmetric, int sms, int* info, int* pairs, int pairs_cap);

/* Number of kernel launches of this library that one pjac_product of shape
 * m x n x k makes with the handle's current transform (split BF16: digit
 * split, slice products, reduction when the inner dimension is split; FP64:
 * one).  Returns -1 when h is NULL, a size is out of range, or the split
 * product does not support the shape. */
int pjac_product_launch_count(pjac_handle* h, int m, int n, int k);

/* Sweeps made by the two parallel-order FP32 Jacobi passes of the last
 * low-precision eigenbasis computed with h (the first pass on fl32(A), the
 * refinement pass on X^T fl32(A) X).  A diagnostic; synchronises the device. */
int pjac_fp32_sweeps_done(pjac_handle* h, int* diag, int* refine);

/* Measured FP64 fused multiply-add rate of the current device in TFLOP/s
 * (2 flops per FMA): eight independent chains per thread over a grid of
 * eight CTAs of 256 threads per SM, timed with CUDA events on the stream
 * after one warm-up launch.  A diagnostic for the roofline of the FP64-bound
 * kernels.  Synchronises the stream. */
int pjac_probe_fp64(double* tflops, void* stream);

/* Human-readable text for a status code (static storage). */
const char* pjac_status_string(int status);
/* Last error message of the calling thread (static per-thread storage). */
const char* pjac_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PJAC_H */
