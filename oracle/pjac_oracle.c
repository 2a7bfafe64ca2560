/*
 * CPU FP64 oracle for the preconditioned Jacobi eigensolver with
 * perturbation-inspired (spectral-gap-weighted) pivoting.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load it.  It shares no code with the
 * CUDA library.
 *
 * Compiled with -O2 -ffp-contract=off: every floating-point operation below
 * is rounded exactly as written (fma() is the IEEE fused multiply-add).
 *
 * What it follows (Shao & Nakatsukasa, "Accelerating preconditioned Jacobi
 * methods via perturbation-inspired pivoting"):
 *   - Algorithm 1 (Jacobi method for eigenvalue computation): loop of
 *     "find a pivot (i,j); compute c,s so that G_ij^T A_ij G_ij is diagonal;
 *     A <- G(c,s,i,j)^T A G(c,s,i,j)", Sec. 2.
 *   - The rotation G(c,s,i,j) = [[c,-s],[s,c]] embedded at rows/cols i,j
 *     (Sec. 2).  The paper does not print c and s; the textbook symmetric
 *     Schur 2x2 with |theta| <= pi/4 is used (see or_rotation).
 *   - The gap-weighted pivot of Eq. (1.1):
 *       L_ij = 2|a_ij|^2 / (|a_ii-a_jj| + sqrt(|a_ii-a_jj|^2 + 4|a_ij|^2)).
 *   - Jacobi's classical greedy pivot argmax |a_ij| and cyclic sweeps (Sec. 1).
 *   - The O(n) update of scores after a rotation (Sec. 3.2): only rows and
 *     columns i and j change, so a per-row best score is kept and only rows
 *     that lost their best entry are rescanned.
 *   - Theorem 1 stopping rule: once every L_ij <= eps, the diagonal is within
 *     2n(n-1)eps of the eigenvalues, so stopping at eps = tau/(2n(n-1))
 *     guarantees eigenvalue accuracy tau (Sec. 3.1).
 *
 * Readings where the paper is silent (every one also stated in the design
 * notes):
 *   - Ties between equal scores: the lexicographically smallest (i,j), i<j.
 *   - Cyclic order: row-cyclic (0,1),(0,2),...,(0,n-1),(1,2),...; a pair
 *     whose a_ij is exactly zero is skipped (no rotation is counted).
 *   - Rotation: d = a_ii - a_jj, den = |d| + sqrt(d*d + 4*(q*q)), q = a_ij;
 *     t = sign * 2|q|/den (sign negative iff d != 0 and d, q have opposite
 *     signs, read from the signs, not from the product d*q which can
 *     underflow), which is the smaller
 *     root of t^2 + 2 zeta t - 1 = 0, zeta = d/(2q), with sign(0) = +1;
 *     c = den / sqrt(den*den + 4*(q*q)) = 1/sqrt(1+t^2); s = t*c.
 *     a_ii' = fma(t,q,a_ii), a_jj' = fma(-t,q,a_jj), a_ij' = 0 exactly;
 *     x' = fma(c,x,s*y), y' = fma(c,y,-(s*x)) for (x,y) = (a_ki,a_kj) and
 *     for (v_ki,v_kj).
 *   - Magnitudes beyond 2^+-500 are scaled by an exact power of two before
 *     squaring (Eq. (1.1) is homogeneous of degree one, t and c of degree 0).
 *   - Convergence (Alg. 1 "Not convergent"): off(A) = sqrt(sum_{k!=l} a_kl^2)
 *     <= tol*||A||_F, tested before every `check_every`-th rotation (greedy,
 *     gap, random) or before every sweep (cyclic).
 *   - Randomized pivoting (the comparator of Sec. 4.2: every pair (i,j)
 *     drawn with equal probability): step k draws the 64-bit word
 *     z = SplitMix64(seed + (k+1)*0x9e3779b97f4a7c15) -- the mixing function
 *     of Steele, Lea and Flood's SplitMix64 generator, used counter-based so
 *     that any step's draw is known without the ones before it -- and takes
 *     i = (z mod 2^32) mod n, j' = (z div 2^32) mod (n-1), j = j' + [j' >= i],
 *     then orders the pair.  Every ordered pair, hence every unordered pair,
 *     has the same probability up to a bias below n/2^32.  A draw whose
 *     a_ij is exactly zero applies the identity rotation and still counts
 *     as a step.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_PIVOT_GAP 0
#define OR_PIVOT_GREEDY 1
#define OR_PIVOT_CYCLIC 2
#define OR_PIVOT_RANDOM 3
#define OR_STOP_OFFDIAG 0
#define OR_STOP_LIBOUND 1

static const double OR_BIG = 0x1p+500;
static const double OR_SMALL = 0x1p-500;

/* Shared piece of Eq. (1.1) and of the rotation: for d = a_ii - a_jj and
 * q = a_ij (already scaled), den = |d| + sqrt(d^2 + 4 q^2) and q2 = q*q. */
static double or_den(double d, double q, double* q2out) {
    double q2 = q * q;
    double r = sqrt(d * d + 4.0 * q2);
    *q2out = q2;
    return fabs(d) + r;
}

/* Exponent used to bring max(|d|,|q|) near 1 when it lies outside
 * [2^-500, 2^500]; 0 otherwise. */
static int or_scale_exp(double d, double q) {
    double m = fmax(fabs(d), fabs(q));
    if (m > OR_BIG || m < OR_SMALL) return ilogb(m);
    return 0;
}

/* Eq. (1.1): L_ij for diagonal entries aii, ajj and off-diagonal aij. */
double or_gap_score(double aii, double ajj, double aij) {
    if (aij == 0.0) return 0.0;
    double d = aii - ajj;
    double q = aij;
    int e = or_scale_exp(d, q);
    if (e != 0) { d = ldexp(d, -e); q = ldexp(q, -e); }
    double q2;
    double den = or_den(d, q, &q2);
    double l = (2.0 * q2) / den;
    if (e != 0) l = ldexp(l, e);
    return l;
}

/* Classical greedy score (Sec. 1): |a_ij|. */
double or_greedy_score(double aij) { return fabs(aij); }

/* c, s, t of the Jacobi rotation that diagonalises [[aii,aij],[aij,ajj]]
 * under A <- G^T A G with G = [[c,-s],[s,c]] (Sec. 2, Alg. 1 line 3). */
void or_rotation(double aii, double ajj, double aij, double* c, double* s, double* t) {
    if (aij == 0.0) { *c = 1.0; *s = 0.0; *t = 0.0; return; }
    double d = aii - ajj;
    double q = aij;
    int e = or_scale_exp(d, q);
    if (e != 0) { d = ldexp(d, -e); q = ldexp(q, -e); }
    double q2;
    double den = or_den(d, q, &q2);
    double tt = (2.0 * fabs(q)) / den;
    if (d != 0.0 && ((d < 0.0) != (q < 0.0))) tt = -tt;
    double cc = den / sqrt(den * den + 4.0 * q2);
    *t = tt;
    *c = cc;
    *s = tt * cc;
}

/* SplitMix64's output function applied to the counter seed + (k+1) gamma. */
uint64_t or_splitmix64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* The pair of step k of the randomized rule (see the header). */
void or_random_pair(uint64_t seed, long long k, int n, int* pi, int* pj) {
    uint64_t z = or_splitmix64(seed, (uint64_t)k);
    int i = (int)((uint32_t)z % (uint32_t)n);
    int j = (int)((uint32_t)(z >> 32) % (uint32_t)(n - 1));
    if (j >= i) j++;
    *pi = i < j ? i : j;
    *pj = i < j ? j : i;
}

static double or_score(int pivot, const double* A, int n, int k, int l) {
    if (pivot == OR_PIVOT_GREEDY) return or_greedy_score(A[(size_t)k * n + l]);
    return or_gap_score(A[(size_t)k * n + k], A[(size_t)l * n + l], A[(size_t)k * n + l]);
}

/* Apply the rotation for pivot (i,j) to A (row-major, symmetric, full
 * storage) and, when V != NULL, to the columns i,j of V (row-major). */
void or_rotate(double* A, int n, double* V, int i, int j, double* tout) {
    double aii = A[(size_t)i * n + i], ajj = A[(size_t)j * n + j], q = A[(size_t)i * n + j];
    double c, s, t;
    or_rotation(aii, ajj, q, &c, &s, &t);
    for (int k = 0; k < n; ++k) {
        if (k == i || k == j) continue;
        double x = A[(size_t)k * n + i];
        double y = A[(size_t)k * n + j];
        double xn = fma(c, x, s * y);
        double yn = fma(c, y, -(s * x));
        A[(size_t)k * n + i] = xn;
        A[(size_t)i * n + k] = xn;
        A[(size_t)k * n + j] = yn;
        A[(size_t)j * n + k] = yn;
    }
    A[(size_t)i * n + i] = fma(t, q, aii);
    A[(size_t)j * n + j] = fma(-t, q, ajj);
    A[(size_t)i * n + j] = 0.0;
    A[(size_t)j * n + i] = 0.0;
    if (V) {
        for (int k = 0; k < n; ++k) {
            double x = V[(size_t)k * n + i];
            double y = V[(size_t)k * n + j];
            V[(size_t)k * n + i] = fma(c, x, s * y);
            V[(size_t)k * n + j] = fma(c, y, -(s * x));
        }
    }
    if (tout) *tout = t;
}

/* off(A) = sqrt(sum_{k != l} a_kl^2), accumulated after scaling every entry
 * by the exact power of two 2^-e so that squares neither overflow nor
 * underflow for entries comparable to `ref`. */
double or_offmass(const double* A, int n, double ref) {
    int e = (ref > 0.0) ? ilogb(ref) : 0;
    double acc = 0.0;
    for (int k = 0; k < n; ++k)
        for (int l = 0; l < n; ++l) {
            if (k == l) continue;
            double x = ldexp(A[(size_t)k * n + l], -e);
            acc += x * x;
        }
    return ldexp(sqrt(acc), e);
}

double or_frobenius(const double* A, int n) {
    double m = 0.0;
    for (size_t p = 0; p < (size_t)n * n; ++p) m = fmax(m, fabs(A[p]));
    if (m == 0.0) return 0.0;
    int e = ilogb(m);
    double acc = 0.0;
    for (size_t p = 0; p < (size_t)n * n; ++p) {
        double x = ldexp(A[p], -e);
        acc += x * x;
    }
    return ldexp(sqrt(acc), e);
}

/* Is (v, k, l) better than (bv, bk, bl)?  Larger score first; among equal
 * scores, the lexicographically smaller (k, l). */
static int or_better(double v, int k, int l, double bv, int bk, int bl) {
    if (v > bv) return 1;
    if (v < bv) return 0;
    if (k != bk) return k < bk;
    return l < bl;
}

/* Brute-force pivot: argmax over i<j of the score, ties to the smallest
 * (i,j) (Eq. (1.1) for gap, Sec. 1 for greedy). */
static double or_select_brute(int pivot, const double* A, int n, int* pi, int* pj) {
    double best = -1.0;
    int bi = 0, bj = 1;
    for (int i = 0; i < n - 1; ++i)
        for (int j = i + 1; j < n; ++j) {
            double v = or_score(pivot, A, n, i, j);
            if (v > best) { best = v; bi = i; bj = j; }
        }
    *pi = bi;
    *pj = bj;
    return best;
}

/* Row-best cache (Sec. 3.2): bestv[k], bestc[k] = max over l != k of the
 * score of row k, ties to the smallest column. */
static void or_rescan_row(int pivot, const double* A, int n, int k, double* bestv, int* bestc) {
    double bv = -1.0;
    int bc = (k == 0) ? 1 : 0;
    for (int l = 0; l < n; ++l) {
        if (l == k) continue;
        double v = or_score(pivot, A, n, k, l);
        if (v > bv) { bv = v; bc = l; }
    }
    bestv[k] = bv;
    bestc[k] = bc;
}

static double or_select_cache(const double* bestv, const int* bestc, int n, int* pi, int* pj) {
    double bv = -1.0;
    int bk = 0;
    for (int k = 0; k < n; ++k)
        if (bestv[k] > bv) { bv = bestv[k]; bk = k; }
    int l = bestc[bk];
    *pi = bk < l ? bk : l;
    *pj = bk < l ? l : bk;
    return bv;
}

/* After rotating (i,j): rows i, j and rows whose best column was i or j are
 * rescanned; every other row compares its best with its new entries (k,i)
 * and (k,j), in increasing column order. */
static void or_update_cache(int pivot, const double* A, int n, int i, int j, double* bestv, int* bestc) {
    for (int k = 0; k < n; ++k) {
        if (k == i || k == j || bestc[k] == i || bestc[k] == j) {
            or_rescan_row(pivot, A, n, k, bestv, bestc);
            continue;
        }
        int cols[2] = {i < j ? i : j, i < j ? j : i};
        for (int m = 0; m < 2; ++m) {
            int l = cols[m];
            double v = or_score(pivot, A, n, k, l);
            if (or_better(v, k, l, bestv[k], k, bestc[k])) { bestv[k] = v; bestc[k] = l; }
        }
    }
}

static int cmp_double(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}

/* max_k |lam_k - d_k| and sum_k |lam_k - d_k| with both sorted ascending
 * (the paper's Sec. 4 error measure is the sum divided by ||A||). */
static void or_eig_error(const double* A, int n, const double* lam_sorted, double* tmp,
                         double* emax, double* esum) {
    for (int k = 0; k < n; ++k) tmp[k] = A[(size_t)k * n + k];
    qsort(tmp, n, sizeof(double), cmp_double);
    double m = 0.0, s = 0.0;
    for (int k = 0; k < n; ++k) {
        double e = fabs(tmp[k] - lam_sorted[k]);
        if (e > m) m = e;
        s += e;
    }
    *emax = m;
    *esum = s;
}

typedef struct {
    long long rotations;      /* rotations applied */
    long long sweeps;         /* cyclic: sweeps started; others: 0 */
    long long checks;         /* convergence tests performed */
    double norm_f;            /* ||A||_F at entry */
    double off_final;         /* off(A) at exit (absolute) */
    double max_score_final;   /* last selected score (gap/greedy) */
    int status;               /* 0 converged, 1 max_rot reached */
    int reserved;
    long long first_rot_eig_ok; /* first checked rotation count with max|dlam| <= eig_tol, or -1 */
    double eig_err_max_final;
    double eig_err_sum_final;
} or_info;

/*
 * Algorithm 1 on A (row-major n x n, symmetric, overwritten), accumulating
 * V <- V G (row-major n x n, may be NULL).
 *   pivot        OR_PIVOT_GAP / GREEDY / CYCLIC
 *   stop         OR_STOP_OFFDIAG: off(A) <= tol*||A||_F
 *                OR_STOP_LIBOUND (gap only): max L <= tol*||A||_F/(2n(n-1))
 *   max_rot      rotation budget (status 1 when reached)
 *   check_every  rotations between off-mass tests (gap/greedy)
 *   select_mode  0 brute force every step, 1 row-best cache
 *   lam_sorted   known eigenvalues ascending, or NULL; eig_tol absolute
 *   piv_log      first log_len pivots as (i,j) pairs, scores in score_log
 *   hist_*       at each convergence test: rotation count, sum|dlam|, off
 */
int or_jacobi(double* A, int n, double* V, int pivot, int stop, double tol,
              long long max_rot, long long check_every, int select_mode,
              const double* lam_sorted, double eig_tol,
              int* piv_log, double* score_log, long long log_len,
              long long* hist_rot, double* hist_err, double* hist_off, long long hist_cap,
              long long* hist_len, uint64_t seed, or_info* info) {
    memset(info, 0, sizeof(*info));
    info->first_rot_eig_ok = -1;
    if (hist_len) *hist_len = 0;
    if (n < 2) { info->status = 0; return 0; }
    double normf = or_frobenius(A, n);
    info->norm_f = normf;
    double thr = tol * normf;
    double eps_li = tol * normf / (2.0 * (double)n * (double)(n - 1));
    double* tmp = (double*)malloc(sizeof(double) * (size_t)n);
    double* bestv = NULL;
    int* bestc = NULL;
    long long rot = 0;
    int status = 1;
    double last_score = 0.0;
    if (check_every < 1) check_every = n;

#define OR_CHECK_AND_MAYBE_STOP()                                                    \
    do {                                                                             \
        double off_ = or_offmass(A, n, normf);                                       \
        info->checks++;                                                              \
        if (lam_sorted) {                                                            \
            double em_, es_;                                                         \
            or_eig_error(A, n, lam_sorted, tmp, &em_, &es_);                         \
            if (info->first_rot_eig_ok < 0 && em_ <= eig_tol) info->first_rot_eig_ok = rot; \
            if (hist_len && *hist_len < hist_cap) {                                  \
                hist_rot[*hist_len] = rot; hist_err[*hist_len] = es_;                \
                hist_off[*hist_len] = off_; (*hist_len)++;                           \
            }                                                                        \
        } else if (hist_len && *hist_len < hist_cap) {                               \
            hist_rot[*hist_len] = rot; hist_err[*hist_len] = -1.0;                   \
            hist_off[*hist_len] = off_; (*hist_len)++;                               \
        }                                                                            \
        if (stop == OR_STOP_OFFDIAG && off_ <= thr) { status = 0; goto done; }       \
    } while (0)

    if (pivot == OR_PIVOT_CYCLIC) {
        for (;;) {
            OR_CHECK_AND_MAYBE_STOP();
            info->sweeps++;
            int any = 0;
            for (int i = 0; i < n - 1; ++i)
                for (int j = i + 1; j < n; ++j) {
                    if (A[(size_t)i * n + j] == 0.0) continue;
                    if (rot >= max_rot) { status = 1; goto done; }
                    if (piv_log && rot < log_len) {
                        piv_log[2 * rot] = i; piv_log[2 * rot + 1] = j;
                        if (score_log) score_log[rot] = fabs(A[(size_t)i * n + j]);
                    }
                    or_rotate(A, n, V, i, j, NULL);
                    rot++;
                    any = 1;
                }
            if (!any) { status = 0; goto done; }
        }
    }

    if (pivot == OR_PIVOT_RANDOM) {
        for (;;) {
            if (rot % check_every == 0) OR_CHECK_AND_MAYBE_STOP();
            if (rot >= max_rot) { status = 1; goto done; }
            int i, j;
            or_random_pair(seed, rot, n, &i, &j);
            if (piv_log && rot < log_len) {
                piv_log[2 * rot] = i; piv_log[2 * rot + 1] = j;
                if (score_log) score_log[rot] = fabs(A[(size_t)i * n + j]);
            }
            or_rotate(A, n, V, i, j, NULL);
            rot++;
        }
    }

    if (select_mode == 1) {
        bestv = (double*)malloc(sizeof(double) * (size_t)n);
        bestc = (int*)malloc(sizeof(int) * (size_t)n);
        for (int k = 0; k < n; ++k) or_rescan_row(pivot, A, n, k, bestv, bestc);
    }
    for (;;) {
        if (rot % check_every == 0) OR_CHECK_AND_MAYBE_STOP();
        int i, j;
        double v = (select_mode == 1) ? or_select_cache(bestv, bestc, n, &i, &j)
                                      : or_select_brute(pivot, A, n, &i, &j);
        last_score = v;
        if (v == 0.0) { status = 0; goto done; }   /* all off-diagonals are zero */
        if (stop == OR_STOP_LIBOUND && v <= eps_li) { status = 0; goto done; }
        if (rot >= max_rot) { status = 1; goto done; }
        if (piv_log && rot < log_len) {
            piv_log[2 * rot] = i; piv_log[2 * rot + 1] = j;
            if (score_log) score_log[rot] = v;
        }
        or_rotate(A, n, V, i, j, NULL);
        rot++;
        if (select_mode == 1) or_update_cache(pivot, A, n, i, j, bestv, bestc);
    }
done:
    info->rotations = rot;
    info->status = status;
    info->max_score_final = last_score;
    info->off_final = or_offmass(A, n, normf);
    if (lam_sorted) or_eig_error(A, n, lam_sorted, tmp, &info->eig_err_max_final, &info->eig_err_sum_final);
    free(tmp);
    free(bestv);
    free(bestc);
    return 0;
#undef OR_CHECK_AND_MAYBE_STOP
}

/* Run the pivot rule to completion on k independent problems (packed,
 * row-major, offsets in doubles) — the oracle of the batched form.  The
 * problems are independent, so they are distributed over threads. */
int or_jacobi_many(int count, const int* ns, const long long* a_off, double* A,
                   const long long* v_off, double* V, int pivot, int stop, double tol,
                   long long max_rot_per_n2, long long* rotations, int* status) {
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1)
    for (int p = 0; p < count; ++p) {
        or_info inf;
        int n = ns[p];
        long long mr = max_rot_per_n2 * (long long)n * (long long)n;
        or_jacobi(A + a_off[p], n, V ? V + v_off[p] : NULL, pivot, stop, tol, mr, n, 1,
                  NULL, 0.0, NULL, NULL, 0, NULL, NULL, NULL, 0, NULL, 0, &inf);
        rotations[p] = inf.rotations;
        status[p] = inf.status;
    }
    return err;
}

/* ------------------------------------------------------------------------
 * One-sided Jacobi SVD with inner products recomputed from the columns
 * (Alg. 2, and Sec. 4.2's relative-accuracy setting: no preconditioner).
 *
 * B is m x n column-major (column k at B + k*m), overwritten by B G_1 G_2 ...
 * The pivot matrix is the Gram matrix G = B^T B of the CURRENT columns:
 * g_kl = sum_r b_rk b_rl, accumulated in row order with fma.  It is formed
 * once in full; after each rotation (i,j) the rows/columns i and j of G are
 * recomputed from the rotated columns (every other entry is unchanged).
 *   Rotation: (c, s, t) of or_rotation on (g_ii, g_jj, g_ij), which makes
 *   columns i, j orthogonal as far as G records them; b_i' = fma(c,b_i,s*b_j),
 *   b_j' = fma(c,b_j,-(s*b_i)), the same for V's columns.
 *   Scores: GAP, Eq. (1.1) on G; GREEDY |g_ij|; GAP_REL, Sec. 4.2's
 *   L^_ij = (1/g_ii + 1/g_jj) L_ij (0 when g_ii or g_jj is 0); RANDOM, the
 *   uniform comparator of Sec. 4.2 (or_random_pair).  Ties: smallest (i,j).
 *   Stop (status 0): the largest score is <= tol (GAP_REL: a relative
 *   bound; GAP, GREEDY: tol * ||G0||_F), tested before every rotation for
 *   the greedy-type rules and every n draws for RANDOM (on GAP_REL scores).
 *   Budget: max_rot rotations (status 1).
 * The singular values are sqrt(g_kk) of the final G; the caller sorts them.
 * ------------------------------------------------------------------------ */
#define OR_PIVOT_GAP_REL 4

static double or_dot(const double* x, const double* y, int m) {
    double acc = 0.0;
    for (int r = 0; r < m; ++r) acc = fma(x[r], y[r], acc);
    return acc;
}

/* Sec. 4.2's relative score. */
double or_gap_rel_score(double aii, double ajj, double aij) {
    if (aij == 0.0 || aii == 0.0 || ajj == 0.0) return 0.0;
    return (1.0 / aii + 1.0 / ajj) * or_gap_score(aii, ajj, aij);
}

static double or_os_score(int pivot, const double* G, int n, int k, int l) {
    double gkl = G[(size_t)k * n + l];
    if (pivot == OR_PIVOT_GREEDY) return fabs(gkl);
    double gkk = G[(size_t)k * n + k], gll = G[(size_t)l * n + l];
    if (pivot == OR_PIVOT_GAP) return or_gap_score(gkk, gll, gkl);
    return or_gap_rel_score(gkk, gll, gkl);
}

static void or_os_rescan(int pivot, const double* G, int n, int k, double* bv, int* bc) {
    double best = -1.0;
    int col = (k == 0) ? 1 : 0;
    for (int l = 0; l < n; ++l) {
        if (l == k) continue;
        double v = or_os_score(pivot, G, n, k, l);
        if (v > best) { best = v; col = l; }
    }
    bv[k] = best;
    bc[k] = col;
}

int or_svd_onesided(double* B, int m, int n, double* V, int pivot, double tol, long long max_rot,
                    uint64_t seed, double* G, long long* rot_out, int* status_out) {
    for (int k = 0; k < n; ++k)
        for (int l = 0; l <= k; ++l) {
            double g = or_dot(B + (size_t)k * m, B + (size_t)l * m, m);
            G[(size_t)k * n + l] = g;
            G[(size_t)l * n + k] = g;
        }
    double normg = or_frobenius(G, n);
    int score_pivot = (pivot == OR_PIVOT_RANDOM) ? OR_PIVOT_GAP_REL : pivot;
    double thr = (score_pivot == OR_PIVOT_GAP_REL) ? tol : tol * normg;
    double* bv = (double*)malloc(sizeof(double) * (size_t)n);
    int* bc = (int*)malloc(sizeof(int) * (size_t)n);
    for (int k = 0; k < n; ++k) or_os_rescan(score_pivot, G, n, k, bv, bc);
    long long rot = 0;
    int status = 1;
    for (;;) {
        int i, j;
        if (pivot == OR_PIVOT_RANDOM) {
            if (rot % n == 0) {
                double mx = 0.0;
                for (int k = 0; k < n; ++k) mx = fmax(mx, bv[k]);
                if (mx <= thr) { status = 0; break; }
            }
            if (rot >= max_rot) break;
            or_random_pair(seed, rot, n, &i, &j);
        } else {
            double best = -1.0;
            int bk = 0;
            for (int k = 0; k < n; ++k)
                if (bv[k] > best) { best = bv[k]; bk = k; }
            if (best <= thr || best == 0.0) { status = 0; break; }
            if (rot >= max_rot) break;
            i = bk < bc[bk] ? bk : bc[bk];
            j = bk < bc[bk] ? bc[bk] : bk;
        }
        double c, s, t;
        or_rotation(G[(size_t)i * n + i], G[(size_t)j * n + j], G[(size_t)i * n + j], &c, &s, &t);
        double* bi = B + (size_t)i * m;
        double* bj = B + (size_t)j * m;
        for (int r = 0; r < m; ++r) {
            double x = bi[r], y = bj[r];
            bi[r] = fma(c, x, s * y);
            bj[r] = fma(c, y, -(s * x));
        }
        if (V) {
            double* vi = V + (size_t)i * n;
            double* vj = V + (size_t)j * n;
            for (int r = 0; r < n; ++r) {
                double x = vi[r], y = vj[r];
                vi[r] = fma(c, x, s * y);
                vj[r] = fma(c, y, -(s * x));
            }
        }
        /* rows and columns i, j of G from the rotated columns */
        for (int k = 0; k < n; ++k) {
            double gi = or_dot(bi, B + (size_t)k * m, m);
            double gj = or_dot(bj, B + (size_t)k * m, m);
            G[(size_t)i * n + k] = gi; G[(size_t)k * n + i] = gi;
            G[(size_t)j * n + k] = gj; G[(size_t)k * n + j] = gj;
        }
        rot++;
        /* row-best cache (Sec. 3.2), as or_update_cache */
        for (int k = 0; k < n; ++k) {
            if (k == i || k == j || bc[k] == i || bc[k] == j) {
                or_os_rescan(score_pivot, G, n, k, bv, bc);
                continue;
            }
            int cols[2] = {i, j};
            for (int q = 0; q < 2; ++q) {
                int l = cols[q];
                double v = or_os_score(score_pivot, G, n, k, l);
                if (or_better(v, k, l, bv[k], k, bc[k])) { bv[k] = v; bc[k] = l; }
            }
        }
    }
    free(bv);
    free(bc);
    *rot_out = rot;
    *status_out = status;
    return 0;
}

/* ------------------------------------------------------------------------
 * Multi-pivot variant (the block/parallel direction Sec. 5 names as future
 * work; its rules here are readings, listed in the design notes).  Every
 * step
 *   1. ranks the rows by their best score (row-best cache of Sec. 3.2),
 *      larger first, ties to the smaller row, and takes the first K rows;
 *   2. walks those K rows in order and accepts the head (k, bestc[k]) as a
 *      pivot when its score is > 0, at least `ratio` times the first row's
 *      score, and neither index is taken by an accepted pivot;
 *   3. applies the accepted rotations one after another in that order
 *      (disjoint index pairs, so each one's (c, s) is that of the matrix
 *      before the step);
 *   4. rescans rows that are pivot indices or whose best column is one, and
 *      compares the new entries (k, x) of every other row, x over the pivot
 *      indices in increasing order (the or_update_cache rule).
 * With K = 1 this is Algorithm 1 with the row-best cache exactly.  Stop: the
 * off-diagonal test before the first step and then before every step at
 * which the rotation count has passed another multiple of check_every; the
 * Theorem 1 stop on the first row's score; a zero first score.  max_rot is
 * tested at the start of a step (status 1).  steps_out: steps taken.
 * ------------------------------------------------------------------------ */
int or_jacobi_multi(double* A, int n, double* V, int pivot, int stop, double tol, long long max_rot,
                    long long check_every, int K, double ratio, long long* steps_out, or_info* info) {
    memset(info, 0, sizeof(*info));
    info->first_rot_eig_ok = -1;
    *steps_out = 0;
    if (n < 2) return 0;
    if (K < 1) K = 1;
    if (check_every < 1) check_every = n;
    double normf = or_frobenius(A, n);
    info->norm_f = normf;
    double thr = tol * normf;
    double eps_li = tol * normf / (2.0 * (double)n * (double)(n - 1));
    double* bestv = (double*)malloc(sizeof(double) * (size_t)n);
    int* bestc = (int*)malloc(sizeof(int) * (size_t)n);
    int* taken = (int*)calloc((size_t)n, sizeof(int));
    int* cand = (int*)malloc(sizeof(int) * (size_t)K);
    int* pi = (int*)malloc(sizeof(int) * (size_t)K);
    int* pj = (int*)malloc(sizeof(int) * (size_t)K);
    char* inset = (char*)calloc((size_t)n, 1);
    int* idx = (int*)malloc(sizeof(int) * (size_t)(2 * K));
    for (int k = 0; k < n; ++k) or_rescan_row(pivot, A, n, k, bestv, bestc);
    long long rot = 0, steps = 0, next_check = 0;
    int status = 1;
    double last = 0.0;
    for (;;) {
        if (rot >= next_check) {
            double off = or_offmass(A, n, normf);
            info->checks++;
            if (stop == OR_STOP_OFFDIAG && off <= thr) { status = 0; break; }
            next_check = (rot / check_every + 1) * check_every;
        }
        /* the K best rows, larger score first, ties to the smaller row */
        int nc = 0;
        for (int q = 0; q < K && q < n; ++q) {
            double bv = -1.0;
            int bk = -1;
            for (int k = 0; k < n; ++k)
                if (!taken[k] && bestv[k] > bv) { bv = bestv[k]; bk = k; }
            if (bk < 0) break;
            taken[bk] = 1;
            cand[nc++] = bk;
        }
        for (int q = 0; q < nc; ++q) taken[cand[q]] = 0;
        double first = bestv[cand[0]];
        last = first;
        if (first == 0.0) { status = 0; break; }
        if (stop == OR_STOP_LIBOUND && first <= eps_li) { status = 0; break; }
        if (rot >= max_rot) { status = 1; break; }
        int na = 0;
        for (int q = 0; q < nc; ++q) {
            int k = cand[q], l = bestc[k];
            double v = bestv[k];
            if (!(v > 0.0) || v < ratio * first) break;
            int i = k < l ? k : l, j = k < l ? l : k;
            if (inset[i] || inset[j]) continue;
            inset[i] = inset[j] = 1;
            pi[na] = i;
            pj[na] = j;
            na++;
        }
        for (int p = 0; p < na; ++p) or_rotate(A, n, V, pi[p], pj[p], NULL);
        rot += na;
        steps++;
        /* the pivot indices in increasing order */
        int ni = 0;
        for (int p = 0; p < na; ++p) { idx[ni++] = pi[p]; idx[ni++] = pj[p]; }
        for (int a = 1; a < ni; ++a)
            for (int b = a; b > 0 && idx[b - 1] > idx[b]; --b) { int t = idx[b]; idx[b] = idx[b - 1]; idx[b - 1] = t; }
        for (int k = 0; k < n; ++k) {
            if (inset[k] || inset[bestc[k]]) {
                or_rescan_row(pivot, A, n, k, bestv, bestc);
                continue;
            }
            for (int q = 0; q < ni; ++q) {
                int l = idx[q];
                double v = or_score(pivot, A, n, k, l);
                if (or_better(v, k, l, bestv[k], k, bestc[k])) { bestv[k] = v; bestc[k] = l; }
            }
        }
        for (int q = 0; q < ni; ++q) inset[idx[q]] = 0;
    }
    info->rotations = rot;
    info->status = status;
    info->max_score_final = last;
    info->off_final = or_offmass(A, n, normf);
    *steps_out = steps;
    free(bestv); free(bestc); free(taken); free(cand); free(pi); free(pj); free(inset); free(idx);
    return 0;
}
