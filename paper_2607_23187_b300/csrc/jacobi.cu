// Jacobi iteration on the preconditioned matrix (Shao & Nakatsukasa,
// Algorithm 1, Sec. 2; pivot rules of Sec. 1 and Eq. (1.1); O(n) score
// update of Sec. 3.2; Theorem 1 stop of Sec. 3.1).
//
// One problem is solved by a cluster of P CTAs (P = 1 for small orders and
// for the batched form).  CTA c owns the index range K_c; for every rotation
// (i,j) it
//   1. rotates the entries (k,i),(k,j) and their mirrors (i,k),(j,k) for
//      k in K_c, and the entries (k,i),(k,j) of V,
//   2. scores the new entries: its own rows k update their cached entries
//      with (k,i),(k,j) (see the row cache below), and the new rows i and j
//      are scored over K_c,
//   3. publishes three candidates (its best own row, its part of row i, its
//      part of row j) and the two largest keys of its parts of rows i and j
//      in shared memory; one cluster barrier later every CTA reads all P
//      slots and makes the same selection.
//
// Row cache (Sec. 3.2's O(n) update, with fewer rescans): each owned row k
// keeps a list of up to two of its entries in exact score order and a key
// bound F_k: every entry of the row outside the list has a key <= F_k.  When
// (k,i),(k,j) change, list entries in those columns are dropped and the new
// entries are inserted if their keys exceed F_k (an entry pushed out of the
// list raises F_k to its own key).  The list head is the exact row maximum
// as long as it was not dropped; a new head is certified when its key
// exceeds F_k by the tie band.  Only an empty or uncertified list triggers a
// rescan.  Rows i and j get their new head from the cluster exchange, and
// as F the largest key among their other entries (from the two largest keys
// of every CTA's part).
// Scores are ranked by integer keys; entries whose keys are within the tie
// band are compared on their exact FP64 scores, so the pivot is the exact
// argmax of the FP64 scores with ties to the smallest (i,j).  The key of
// every entry is kept in the key matrix K (int32, n x n), updated with the
// rotated entries, so that a rescan reads keys instead of recomputing them.
// The convergence test (every check_every rotations) sums the squares of
// the strict upper triangle, rows taken cyclically by the cluster's CTAs.
//
// A is read and written with ld/st.global.cg (L2), because entries of a row
// are written by several CTAs between cluster barriers.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <cstdint>
#include <climits>
#include "devmath.cuh"
#include "internal.h"

namespace cg = cooperative_groups;

namespace pjac {

constexpr int NT = 256;     // threads per CTA
constexpr int MAXR = 4;     // owned indices per thread (m <= NT * MAXR); MR <= MAXR per kernel

struct Cand {
    int key, row, col, pad;
    double x;               // the entry a_row,col
    double ex;              // exact score (gap) if >= 0, else not yet computed
};

struct Slot {
    Cand cand[3];           // this CTA's best own row, its part of row i, of row j
    int ki[2], kj[2];       // the two largest keys of its parts of rows i and j
    double prm[3][3];       // (den, 4q^2, t) of each candidate's rotation (scaled; rot_cs gives c, s)
    double sum;
    int flags, pad;
};

struct Sh {
    int fij[2];             // key bounds F of the new rows i and j
    int wkk[NT / 32][4];    // per-warp two largest keys of rows i and j
    Cand ww[NT / 32][3];    // per-warp winners of the three selections
    int wkey[NT / 32];
    Cand wc[NT / 32];
    double wsum[NT / 32];
    Cand out;
    Slot slots[2];
    Slot inbox[2][16];      // slot of every cluster rank, pushed by the sender
    Slot stage;             // this CTA's slot before it is pushed
    Cand sel;
    Cand sel3[3];           // cta_select3: the warps' final selections (1 and 2 used)
    int rk[32], rc[32];     // rescan_row_keys: each warp's four largest keys and their columns
    Cand rs_b, rs_s;        // rescan_row_keys: the row's head and second entry
    int rs_f, rs_ok;        // rescan_row_keys: the key bound; 0 when the full rescan is needed
    int kk3[4];             // cta_select3: the merged keys of rows i and j
    int tflag, pad3;
    double c, s, t, dii, djj, q;
    double cs[48][2];       // (c, s) of every published candidate (3 per cluster rank)
    double old_di, old_dj;  // diagonal entries before the pending rotation
    double normf, thr, eps_li, scale;
    int scaled_sum;                // off-diagonal sums scale every entry (extreme ||A1||_F only)
    int pi, pj, nresc, decision;
    int win, pad4;          // inbox index of the pending pivot
    int key_eps, pad2;
#ifdef PJAC_PROFILE
    long long t_top;
#endif
};

// the key-based rescan merges four entries of each warp in one warp
static_assert((NT / 32) * 4 == 32, "rescan_row_keys expects eight warps");
// warps 5 and up finish (c, s) of the 3 candidates of each of up to 16 ranks
static_assert((NT / 32 - 5) * 32 >= 48, "too few warps for the cosines of the published candidates");

#ifdef PJAC_PROFILE
// Profiling build only: per-phase clock totals of CTA 0 and event counts.
__device__ unsigned long long g_prof[40];
__device__ unsigned long long g_rank[32];   // per cluster rank: loop top to arrive, arrive to wait done
#define PROF_ADD(k, v) atomicAdd(&g_prof[k], (unsigned long long)(v))
// exact evaluations made by this CTA (one counter per CTA)
__device__ __forceinline__ unsigned int& prof_exact() {
    __shared__ unsigned int s;
    return s;
}
#else
#define PROF_ADD(k, v) ((void)0)
#endif

// Scores are non-negative doubles (or a negative "not evaluated" sentinel);
// such values order like their bit patterns read as signed integers, so
// they are compared on the integer pipes (an FP64 compare waits on the
// FP64 pipe's long latency).
__device__ __forceinline__ long long sbits(double v) { return __double_as_longlong(v); }

__device__ __forceinline__ double ldcg(const double* p) { return __ldcg(p); }
__device__ __forceinline__ void stcg(double* p, double v) { __stcg(p, v); }

__device__ __forceinline__ Cand no_cand() {
    Cand c;
    c.key = KEY_NONE; c.row = -1; c.col = -1; c.pad = 0; c.x = 0.0; c.ex = -1.0;
    return c;
}

__device__ __forceinline__ int entry_key(int pivot, double x, double dd) {
    return pivot == PJAC_PIVOT_GREEDY ? greedy_key(x) : gap_key(x, dd);
}

// Exact score of a candidate (gap: Eq. (1.1) in FP64; greedy: |x|).
__device__ __forceinline__ double cand_value(Cand& c, int pivot, const double* diag) {
    if (pivot == PJAC_PIVOT_GREEDY) return fabs(c.x);
    if (sbits(c.ex) < 0) {   // not evaluated yet
        c.ex = gap_exact(diag[c.row], diag[c.col], c.x);
#ifdef PJAC_PROFILE
        if (c.x != 0.0) atomicAdd(&prof_exact(), 1u);
#endif
    }
    return c.ex;
}

__device__ __forceinline__ bool exact_better(double va, const Cand& a, double vb, const Cand& b) {
    if (sbits(va) != sbits(vb)) return sbits(va) > sbits(vb);
    if (a.row != b.row) return a.row < b.row;
    return a.col < b.col;
}

// Is a strictly better than b (larger score, then smaller (row, col))?
__device__ __forceinline__ bool better(Cand& a, Cand& b, int pivot, const double* diag) {
    if (a.key == KEY_NONE) return false;
    if (b.key == KEY_NONE) return true;
    // the same unordered pair seen from its two rows: equal scores
    if (a.row == b.col && a.col == b.row) return a.row < b.row;
    if (a.row == b.row && a.col == b.col) return false;
    if (pivot == PJAC_PIVOT_GREEDY) {
        if (a.key != b.key) return a.key > b.key;
    } else {
        int km = max(a.key, b.key);
        if (km >= KEY_SUB) {
            long long d = (long long)a.key - (long long)b.key;
            if (d > KEY_GAP_TIE) return true;
            if (d < -KEY_GAP_TIE) return false;
        }
    }
    double va = cand_value(a, pivot, diag), vb = cand_value(b, pivot, diag);
    return exact_better(va, a, vb, b);
}

__device__ __forceinline__ int block_max_int(int v, Sh& sh) {
    int w = __reduce_max_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0) sh.wkey[threadIdx.x >> 5] = w;
    __syncthreads();
    int r = sh.wkey[0];
#pragma unroll
    for (int k = 1; k < NT / 32; ++k) r = max(r, sh.wkey[k]);
    __syncthreads();
    return r;
}

// ---- row cache: a list of up to two entries and a key bound F ----------
// Key bound for the entries below an exactly known one (every entry with an
// FP64 score <= b's has a key <= the result): the key itself for the greedy
// rule (monotone), b's key plus the key error margin for the gap rule (keys
// below KEY_SUB are bounded by KEY_SUB + margin), KEY_NONE when there is no
// such entry.
__device__ __forceinline__ int bound_from_exact(const Cand& b, int pivot) {
    if (b.key == KEY_NONE) return KEY_NONE;
    if (pivot == PJAC_PIVOT_GREEDY) return b.key;
    if (b.key == KEY_ZERO) return KEY_ZERO;
    return max(b.key, KEY_SUB) + KEY_GAP_TIE;
}

// Insert entry e into the list (cur, sec) whose outside entries have keys
// <= F; an entry that leaves the list raises F to its key.  e is always
// compared with the head exactly, so a head that was the row's maximum stays
// it; below the head, an entry whose key is <= F may stay outside.
__device__ __forceinline__ void list_insert(Cand& e, Cand& cur, Cand& sec, int& F, int pivot,
                                            const double* diag) {
    if (e.key == KEY_NONE) return;
    if (cur.key == KEY_NONE) {
        if (F != KEY_NONE && e.key <= F) return;
        cur = e;
        return;
    }
    if (better(e, cur, pivot, diag)) {
        if (sec.key != KEY_NONE) F = (F == KEY_NONE) ? sec.key : max(F, sec.key);
        sec = cur;
        cur = e;
        return;
    }
    if (F != KEY_NONE && e.key <= F) return;     // stays outside, under the bound
    if (sec.key == KEY_NONE) { sec = e; return; }
    if (better(e, sec, pivot, diag)) {
        F = (F == KEY_NONE) ? sec.key : max(F, sec.key);
        sec = e;
        return;
    }
    F = (F == KEY_NONE) ? e.key : max(F, e.key);
}

// Two largest keys (with multiplicity) of a set, as a pair k1 >= k2.
__device__ __forceinline__ void key_push(int k, int& k1, int& k2) {
    if (k > k1) { k2 = k1; k1 = k; }
    else if (k > k2) k2 = k;
}
// Warp-wide two largest keys from per-lane pairs (every lane gets them).
__device__ __forceinline__ void warp_top2_keys(int& k1, int& k2) {
    const int m1 = __reduce_max_sync(0xffffffffu, k1);
    const unsigned at = __ballot_sync(0xffffffffu, k1 == m1);
    const int m2 = __reduce_max_sync(0xffffffffu, k1 == m1 ? k2 : k1);
    k1 = m1;
    k2 = (__popc(at) > 1) ? m1 : m2;
}
// Key bound F of a row whose head is h, given the two largest keys of all
// its entries: the largest key of the entries other than h.
__device__ __forceinline__ int bound_without_head(const Cand& h, int k1, int k2) {
    return (h.key == k1) ? k2 : k1;
}

// Is the list head cur certainly the row's exact maximum, given only that
// the entries outside the list have keys <= F?
__device__ __forceinline__ bool head_certified(const Cand& cur, int F, int pivot) {
    if (cur.key == KEY_NONE) return false;
    if (F == KEY_NONE) return true;
    if (pivot == PJAC_PIVOT_GREEDY) return cur.key > F;
    if (cur.key == KEY_ZERO) return F <= KEY_ZERO;   // the row's maximum is 0
    if (cur.key < KEY_SUB) return false;              // keys do not decide there
    return (long long)cur.key > (long long)F + KEY_GAP_TIE;
}

__device__ __forceinline__ Cand shfl_cand(const Cand& c, int src) {
    Cand o;
    o.key = __shfl_sync(0xffffffffu, c.key, src);
    o.row = __shfl_sync(0xffffffffu, c.row, src);
    o.col = __shfl_sync(0xffffffffu, c.col, src);
    o.pad = 0;
    o.x = __shfl_sync(0xffffffffu, c.x, src);
    o.ex = __shfl_sync(0xffffffffu, c.ex, src);
    return o;
}

// Block-wide exact argmax of one candidate per thread.  Phase 1 takes the
// maximum key; phase 2 (only when several threads are within the tie band)
// evaluates the contenders exactly.  Uniform call (all threads).
__device__ Cand block_select(Cand mine, int pivot, const double* diag, Sh& sh) {
    int kmax = block_max_int(mine.key, sh);
    if (kmax == KEY_NONE) return no_cand();
    bool exact_all = (pivot != PJAC_PIVOT_GREEDY) && kmax < KEY_SUB;
    int tie = (pivot == PJAC_PIVOT_GREEDY) ? 0 : KEY_GAP_TIE;
    bool cont = mine.key != KEY_NONE && (exact_all || (long long)mine.key >= (long long)kmax - tie);
    int nc = __syncthreads_count(cont);
    if (nc == 1) {
        if (cont) sh.out = mine;
        __syncthreads();
        Cand r = sh.out;
        __syncthreads();
        return r;
    }
    double v = -2.0;
    if (cont) v = cand_value(mine, pivot, diag);
    int lane = threadIdx.x & 31;
    // warp argmax on (v desc, row asc, col asc)
    double bv = v;
    int br = mine.row, bc = mine.col, bl = lane;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        double ov = __shfl_xor_sync(0xffffffffu, bv, off);
        int orr = __shfl_xor_sync(0xffffffffu, br, off);
        int oc = __shfl_xor_sync(0xffffffffu, bc, off);
        int ol = __shfl_xor_sync(0xffffffffu, bl, off);
        const long long ob = sbits(ov), bb = sbits(bv);
        bool take = (ob > bb) || (ob == bb && (orr < br || (orr == br && (oc < bc || (oc == bc && ol < bl)))));
        if (take) { bv = ov; br = orr; bc = oc; bl = ol; }
    }
    if (lane == bl) {
        Cand w = mine;
        if (sbits(bv) < 0) w.key = KEY_NONE;   // no contender (the -2 sentinel)
        sh.wc[threadIdx.x >> 5] = w;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Cand best = no_cand();
        double vb = -2.0;
        for (int w = 0; w < NT / 32; ++w) {
            Cand c = sh.wc[w];
            if (c.key == KEY_NONE) continue;
            double vc = cand_value(c, pivot, diag);
            if (best.key == KEY_NONE || exact_better(vc, c, vb, best)) { best = c; vb = vc; }
        }
        sh.out = best;
    }
    __syncthreads();
    Cand r = sh.out;
    __syncthreads();
    return r;
}

// Exact argmax of one candidate per lane over a warp (every lane gets the
// winner), without block barriers.  Keys first; lanes whose key is within
// the tie band of the maximum are contenders, and only several contenders
// need their exact scores (computed in parallel; wb, when given, is the
// cache entry the lane's candidate came from and keeps its exact score).
// Contenders that are all one pair seen from its two rows have equal
// scores and the row with row < col wins, as in better().
__device__ Cand warp_select(Cand c, int pivot, const double* diag, Cand* wb) {
    const int lane = threadIdx.x & 31;
    const int m = __reduce_max_sync(0xffffffffu, c.key);
    if (m == KEY_NONE) return no_cand();
    const bool gap = pivot != PJAC_PIVOT_GREEDY;
    const bool exact_all = gap && m < KEY_SUB;
    const int tie = gap ? KEY_GAP_TIE : 0;
    const bool cont = c.key != KEY_NONE && (exact_all || (long long)c.key >= (long long)m - tie);
    const unsigned b = __ballot_sync(0xffffffffu, cont);
    int src;
    if (__popc(b) == 1) {
        src = __ffs(b) - 1;
    } else {
        const int pid = cont ? ((min(c.row, c.col) << 15) | max(c.row, c.col)) : INT_MAX;
        const int pmin = __reduce_min_sync(0xffffffffu, pid);
        const int pmax = __reduce_max_sync(0xffffffffu, cont ? pid : -1);
        if (pmin == pmax) {
            // one pair, possibly seen from both rows: the row < col view
            const unsigned lo = __ballot_sync(0xffffffffu, cont && c.row < c.col);
            src = __ffs(lo ? lo : b) - 1;
        } else {
            double v = -2.0;
            if (cont) {
                v = cand_value(c, pivot, diag);
                if (wb && wb->row == c.row && wb->col == c.col) wb->ex = c.ex;
            }
            double bv = v;
            int br = cont ? c.row : INT_MAX, bc = cont ? c.col : INT_MAX, bl = lane;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double ov = __shfl_xor_sync(0xffffffffu, bv, off);
                const int orr = __shfl_xor_sync(0xffffffffu, br, off);
                const int oc = __shfl_xor_sync(0xffffffffu, bc, off);
                const int ol = __shfl_xor_sync(0xffffffffu, bl, off);
                const long long ob = sbits(ov), bb = sbits(bv);
                const bool take =
                    (ob > bb) || (ob == bb && (orr < br || (orr == br && (oc < bc || (oc == bc && ol < bl)))));
                if (take) { bv = ov; br = orr; bc = oc; bl = ol; }
            }
            src = bl;
        }
    }
    Cand r;
    r.key = __shfl_sync(0xffffffffu, c.key, src);
    r.row = __shfl_sync(0xffffffffu, c.row, src);
    r.col = __shfl_sync(0xffffffffu, c.col, src);
    r.pad = __shfl_sync(0xffffffffu, c.pad, src);
    r.x = __shfl_sync(0xffffffffu, c.x, src);
    r.ex = __shfl_sync(0xffffffffu, c.ex, src);
    return r;
}

// The CTA's three exact argmaxes (best own row, its part of row i, of row j)
// and the two largest keys of its parts of rows i and j, with one block
// barrier: every warp selects its own winners, then warp 0 selects among
// the warps' winners.  The results are valid in warp 0 only (the warp that
// evaluates and publishes them).  cache/k0/k1: the row cache, so that exact
// scores computed in warp 0 stay with the cached entries.
__device__ void cta_select3(Cand& c0, Cand& c1, Cand& c2, int pivot, const double* diag, Sh& sh,
                            int (&kA)[2], int (&kB)[2], Cand* wb0, Cand* cache, int k0, int k1) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const Cand w0 = warp_select(c0, pivot, diag, wb0);
    const Cand w1 = warp_select(c1, pivot, diag, nullptr);
    const Cand w2 = warp_select(c2, pivot, diag, nullptr);
    warp_top2_keys(kA[0], kA[1]);
    warp_top2_keys(kB[0], kB[1]);
    if (lane == 0) {
        sh.ww[warp][0] = w0;
        sh.ww[warp][1] = w1;
        sh.ww[warp][2] = w2;
        sh.wkk[warp][0] = kA[0]; sh.wkk[warp][1] = kA[1]; sh.wkk[warp][2] = kB[0]; sh.wkk[warp][3] = kB[1];
    }
    __syncthreads();
    if (warp >= 4) return;
    // warps 0-2 select one of the three candidates each, warp 3 merges the
    // keys; warp 0 collects after a barrier of these four warps
    if (warp < 3) {
        Cand c = (lane < NT / 32) ? sh.ww[lane][warp] : no_cand();
        Cand* wb = nullptr;
        if (warp == 0 && c.key != KEY_NONE && c.row >= k0 && c.row < k1) wb = &cache[c.row - k0];
        const Cand r = warp_select(c, pivot, diag, wb);
        if (warp == 0) c0 = r;
        else if (lane == 0) sh.sel3[warp] = r;
    } else if (lane == 0) {
        int a1 = KEY_NONE, a2 = KEY_NONE, b1 = KEY_NONE, b2 = KEY_NONE;
#pragma unroll
        for (int w = 0; w < NT / 32; ++w) {
            key_push(sh.wkk[w][0], a1, a2);
            key_push(sh.wkk[w][1], a1, a2);
            key_push(sh.wkk[w][2], b1, b2);
            key_push(sh.wkk[w][3], b1, b2);
        }
        sh.kk3[0] = a1; sh.kk3[1] = a2; sh.kk3[2] = b1; sh.kk3[3] = b2;
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");
    if (warp != 0) return;
    c1 = sh.sel3[1];
    c2 = sh.sel3[2];
    kA[0] = sh.kk3[0]; kA[1] = sh.kk3[1]; kB[0] = sh.kk3[2]; kB[1] = sh.kk3[3];
}

__device__ __forceinline__ double block_sum(double v, Sh& sh) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0) sh.wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
#pragma unroll
    for (int k = 0; k < NT / 32; ++k) r += sh.wsum[k];
    __syncthreads();
    return r;
}

__device__ __forceinline__ double block_maxabs(double v, Sh& sh) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    if ((threadIdx.x & 31) == 0) sh.wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
#pragma unroll
    for (int k = 0; k < NT / 32; ++k) r = fmax(r, sh.wsum[k]);
    __syncthreads();
    return r;
}

// Key of a positive value on the gap-key scale (floor(2^20 log2 v) within
// the same error band).
__device__ __forceinline__ int value_key(double v) {
    if (v <= 0.0) return KEY_ZERO;
    return gap_key(v, 0.0);
}

template <bool CLUSTER>
__device__ __forceinline__ void cta_exchange_sync() {
    if (CLUSTER) {
        asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
        asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
    } else {
        __syncthreads();
    }
}

template <bool CLUSTER>
__device__ __forceinline__ const Slot* peer_slot(Sh& sh, int par, int r) {
    if (CLUSTER) {
        cg::cluster_group cl = cg::this_cluster();
        return cl.map_shared_rank(&sh.slots[par], r);
    }
    return &sh.slots[par];
}

// Rescan row k (block-wide): its best entry over l != k, in sec its second
// entry, and in F the key bound of its remaining entries (from its third).
__device__ Cand rescan_row(const JacArgs& a, int k, const double* diag, Sh& sh, Cand& sec, int& F,
                           bool store_keys = false) {
    const double* row = a.A + (long long)k * a.lda;
    int* krow = (store_keys && a.K) ? a.K + (long long)k * a.ldk : nullptr;
    double dk = diag[k];
#ifdef PJAC_PROFILE
    const long long t_r0 = clock64();
#endif
    Cand t1 = no_cand(), t2 = no_cand(), t3 = no_cand();
    for (int l0 = threadIdx.x; l0 < a.n; l0 += 4 * NT) {
        double xs[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int l = l0 + u * NT;
            xs[u] = (l < a.n) ? ldcg(row + l) : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            int l = l0 + u * NT;
            if (l >= a.n || l == k) continue;
            Cand c;
            c.row = k; c.col = l; c.pad = 0; c.x = xs[u]; c.ex = -1.0;
            c.key = entry_key(a.pivot, xs[u], a.pivot == PJAC_PIVOT_GREEDY ? 0.0 : __dadd_rn(dk, -diag[l]));
            if (krow) __stcg(krow + l, c.key);
            // most entries fail against the third at once
            if (better(c, t3, a.pivot, diag)) {
                if (better(c, t2, a.pivot, diag)) {
                    t3 = t2;
                    if (better(c, t1, a.pivot, diag)) { t2 = t1; t1 = c; }
                    else t2 = c;
                } else {
                    t3 = c;
                }
            }
        }
    }
#ifdef PJAC_PROFILE
    const long long t_s0 = clock64();
#endif
    Cand b = block_select(t1, a.pivot, diag, sh);
#ifdef PJAC_PROFILE
    const long long t_s1 = clock64();
#endif
    const bool w1 = t1.key != KEY_NONE && t1.col == b.col;
    Cand offer = w1 ? t2 : t1;
    sec = block_select(offer, a.pivot, diag, sh);
    // the thread's best entry that is neither b nor sec
    Cand o3 = t1;
    if (o3.key != KEY_NONE && (o3.col == b.col || o3.col == sec.col)) o3 = t2;
    if (o3.key != KEY_NONE && (o3.col == b.col || o3.col == sec.col)) o3 = t3;
    Cand third = block_select(o3, a.pivot, diag, sh);
    F = bound_from_exact(third, a.pivot);
#ifdef PJAC_PROFILE
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        PROF_ADD(20, t_s0 - t_r0);
        PROF_ADD(21, t_s1 - t_s0);
        PROF_ADD(22, clock64() - t_s1);
        PROF_ADD(23, 1);
    }
#endif
    return b;
}

// off(A)^2 * 2^-2e over the owned rows, e = ilogb(||A1||_F) (as the oracle).
// Row rescan from the stored keys (column k of K holds the keys of row k):
// each thread keeps the four largest keys of its columns, each warp the four
// largest of its threads' lists, and warp 0 merges the warps' lists: the
// head b is the exact maximum among the entries within the tie band of the
// largest key, sec the exact best of the listed entries other than b, and F
// the largest listed key other than b's and sec's (an entry left out of a
// list has a key no larger than that list's smallest).  One block barrier
// besides the final one.  Returns false, with nothing written, when some
// warp's list is full of contenders for the maximum: then only the full
// rescan is exact.
__device__ bool rescan_row_keys(const JacArgs& a, int k, const double* diag, Sh& sh, Cand& b, Cand& sec,
                                int& F) {
    const int* kr = a.K + (long long)k * a.ldk;
    const double* row = a.A + (long long)k * a.lda;
    int lk[4] = {KEY_NONE, KEY_NONE, KEY_NONE, KEY_NONE}, lc[4] = {-1, -1, -1, -1};
    constexpr int CH = 16;
    for (int l0 = threadIdx.x; l0 < a.n; l0 += CH * NT) {
        int ks[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const int l = l0 + u * NT;
            ks[u] = (l < a.n && l != k) ? __ldcg(kr + l) : KEY_NONE;
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            int kk = ks[u], cc = l0 + u * NT;
            if (kk <= lk[3]) continue;
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (kk > lk[q]) {
                    const int tk = lk[q], tc = lc[q];
                    lk[q] = kk; lc[q] = cc;
                    kk = tk; cc = tc;
                }
        }
    }
    // each warp's four largest keys: four rounds of the maximum over the
    // lanes' list heads, popped at the first lane that holds it
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int wk = KEY_NONE, wc = -1;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int m = __reduce_max_sync(0xffffffffu, lk[0]);
        const int src = __ffs(__ballot_sync(0xffffffffu, lk[0] == m)) - 1;
        const int col = __shfl_sync(0xffffffffu, lc[0], src);
        if (lane == q) { wk = m; wc = col; }
        if (lane == src) {
            lk[0] = lk[1]; lc[0] = lc[1];
            lk[1] = lk[2]; lc[1] = lc[2];
            lk[2] = lk[3]; lc[2] = lc[3];
            lk[3] = KEY_NONE; lc[3] = -1;
        }
    }
    if (lane < 4) {
        sh.rk[warp * 4 + lane] = wk;
        sh.rc[warp * 4 + lane] = wc;
    }
    __syncthreads();
    // warp 0 merges the 32 listed entries (lane l: entry l mod 4 of warp l / 4)
    if (warp == 0) {
        const int ek = sh.rk[lane], ec = sh.rc[lane];
        const int kmax = __reduce_max_sync(0xffffffffu, ek);
        int ok = 1;
        Cand bb = no_cand(), ss = no_cand();
        int ff = KEY_NONE;
        if (kmax != KEY_NONE) {
            const bool gap = a.pivot != PJAC_PIVOT_GREEDY;
            const bool exact_all = gap && kmax < KEY_SUB;
            const int tie = gap ? KEY_GAP_TIE : 0;
            // a warp whose fourth entry contends for the maximum may have left
            // contenders out: then only the full rescan is exact
            const bool ovf = (lane & 3) == 3 && ek != KEY_NONE &&
                             (exact_all || (long long)ek >= (long long)kmax - tie);
            if (__any_sync(0xffffffffu, ovf)) {
                ok = 0;
            } else {
                Cand c = no_cand();
                if (ek != KEY_NONE) {
                    c.key = ek; c.row = k; c.col = ec; c.x = ldcg(row + ec);
                }
                bb = warp_select(c, a.pivot, diag, nullptr);
                const Cand c2 = (c.key != KEY_NONE && c.col != bb.col) ? c : no_cand();
                ss = warp_select(c2, a.pivot, diag, nullptr);
                const int rk = (ek != KEY_NONE && ec != bb.col && ec != ss.col) ? ek : KEY_NONE;
                ff = __reduce_max_sync(0xffffffffu, rk);
            }
        }
        if (lane == 0) {
            sh.rs_ok = ok;
            sh.rs_b = bb;
            sh.rs_s = ss;
            sh.rs_f = ff;
        }
    }
    __syncthreads();
    if (!sh.rs_ok) return false;
    b = sh.rs_b;
    sec = sh.rs_s;
    F = sh.rs_f;
    return true;
}

// This CTA's part of sum_{k<l} a_kl^2 (the strict upper triangle; the
// matrix is stored in full and symmetric): rows k = rank (mod P), eight rows
// at a time with eight independent partial sums, so that the loads of a
// block overlap and no FMA waits on the previous one.  SCALED multiplies
// every entry by `scale` (a power of two) first, for norms near the ends of
// the exponent range; otherwise the squares cannot overflow or lose
// anything that matters and one FMA per entry is enough.
template <bool SCALED>
__device__ double upper_offsum_t(const JacArgs& a, int rank, int P, double scale, Sh& sh) {
    double acc[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    const int n = a.n;
    for (int kb = rank; kb < n; kb += 8 * P) {
        for (int l = ((kb + 1) / NT) * NT + (int)threadIdx.x; l < n; l += NT) {
            double x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int k = kb + u * P;
                x[u] = (k < n && l > k) ? ldcg(a.A + (long long)k * a.lda + l) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const double y = SCALED ? __dmul_rn(x[u], scale) : x[u];
                acc[u] = __fma_rn(y, y, acc[u]);
            }
        }
    }
    double t = __dadd_rn(__dadd_rn(__dadd_rn(acc[0], acc[1]), __dadd_rn(acc[2], acc[3])),
                         __dadd_rn(__dadd_rn(acc[4], acc[5]), __dadd_rn(acc[6], acc[7])));
    return block_sum(t, sh);
}

__device__ double upper_offsum(const JacArgs& a, int rank, int P, Sh& sh) {
    return sh.scaled_sum ? upper_offsum_t<true>(a, rank, P, sh.scale, sh)
                         : upper_offsum_t<false>(a, rank, P, sh.scale, sh);
}

// off(A) = sqrt(2 g) from the cluster's sum g of the upper-triangle parts
__device__ __forceinline__ double off_from_sum(double g, const Sh& sh) {
    if (!(sh.normf > 0.0)) return 0.0;
    const double r = sqrt(2.0 * g);
    return sh.scaled_sum ? __dmul_rn(r, 1.0 / sh.scale) : r;
}

// Solve one problem.  rank/P: this CTA's rank in the cluster and the
// cluster size.  Shared arrays: diag[n]; per owned row: cache[m] (the list
// head, the row's exact best entry), cache2[m] (the list's second entry or
// none), cachef[m] (the key bound F of the entries outside the list);
// resc[m].
template <bool CLUSTER, int MR>
__device__ void jacobi_problem(const JacArgs& a, int rank, int P, Sh& sh, double* diag,
                               Cand* cache, Cand* cache2, int* cachef, int* resc) {
    const int n = a.n;
    const int tid = threadIdx.x;
    const int mchunk = (n + P - 1) / P;
    const int k0 = min(n, rank * mchunk);
    const int k1 = min(n, k0 + mchunk);
    const int pivot = a.pivot;
    const unsigned long long start = now_ns();
#ifdef PJAC_PROFILE
    long long pt = clock64();
    unsigned int pex = 0;
    if (tid == 0) prof_exact() = 0;
    __syncthreads();
#define LAP(k) do { if (rank == 0 && tid == 0) { long long nw = clock64(); PROF_ADD(k, nw - pt); pt = nw; \
        unsigned int ce = prof_exact(); PROF_ADD(12 + (k), ce - pex); pex = ce; } } while (0)
// time since the last LAP, without starting a new phase
#define SLAP(k) do { if (rank == 0 && tid == 0) PROF_ADD(24 + (k), clock64() - pt); } while (0)
#else
#define LAP(k) ((void)0)
#define SLAP(k) ((void)0)
#endif

    for (int k = tid; k < n; k += NT) diag[k] = ldcg(a.A + (long long)k * a.lda + k);

    // ||A1||_F with the oracle's scaling: max |a|, then sum of (a 2^-e)^2.
    double mx = 0.0;
    for (int k = k0; k < k1; ++k)
        for (int l = tid; l < n; l += NT) mx = fmax(mx, fabs(ldcg(a.A + (long long)k * a.lda + l)));
    mx = block_maxabs(mx, sh);
    int par = 0;
    if (tid == 0) sh.slots[par].sum = mx;
    cta_exchange_sync<CLUSTER>();
    if (tid == 0) {
        double g = 0.0;
        for (int r = 0; r < P; ++r) g = fmax(g, peer_slot<CLUSTER>(sh, par, r)->sum);
        sh.scale = (g > 0.0) ? ldexp(1.0, -ilogb(g)) : 1.0;
        sh.normf = g;   // temporary: max |a|
    }
    par ^= 1;
    __syncthreads();
    {
        double acc = 0.0;
        double scl = sh.scale;
        for (int k = k0; k < k1; ++k)
            for (int l = tid; l < n; l += NT) {
                double x = __dmul_rn(ldcg(a.A + (long long)k * a.lda + l), scl);
                acc = __fma_rn(x, x, acc);
            }
        acc = block_sum(acc, sh);
        if (tid == 0) sh.slots[par].sum = acc;
    }
    cta_exchange_sync<CLUSTER>();
    if (tid == 0) {
        double g = 0.0;
        for (int r = 0; r < P; ++r) g += peer_slot<CLUSTER>(sh, par, r)->sum;
        double maxa = sh.normf;
        double nf = (maxa > 0.0) ? ldexp(sqrt(g), ilogb(maxa)) : 0.0;
        sh.normf = nf;
        sh.thr = a.tol * nf;
        sh.eps_li = a.tol * nf / (2.0 * (double)n * (double)(n - 1));
        sh.scale = (nf > 0.0) ? ldexp(1.0, -ilogb(nf)) : 1.0;
        sh.scaled_sum = !(nf >= 0x1p-300 && nf <= 0x1p300);
        sh.key_eps = value_key(sh.eps_li);
    }
    par ^= 1;
    __syncthreads();

    long long rot = 0, sweeps = 0;
    int status = PJAC_ENOCONV;
    double last_score = 0.0;
    const long long ce = a.check_every > 0 ? a.check_every : n;

    // ---- convergence test (collective over the cluster) ----
    auto offdiag_check = [&](bool& stop_now) {
        double part = upper_offsum(a, rank, P, sh);
        if (tid == 0) {
            sh.slots[par].sum = part;
            sh.slots[par].flags = (rank == 0 && a.budget_ns > 0 && (long long)(now_ns() - start) > a.budget_ns) ? 1 : 0;
        }
        cta_exchange_sync<CLUSTER>();
        if (tid == 0) {
            double g = 0.0;
            for (int r = 0; r < P; ++r) g += peer_slot<CLUSTER>(sh, par, r)->sum;
            const double off = off_from_sum(g, sh);
            int dec = 0;
            if (peer_slot<CLUSTER>(sh, par, 0)->flags & 1) dec = 2;
            else if (a.stop == PJAC_STOP_OFFDIAG && off <= sh.thr) dec = 1;
            sh.decision = dec;
        }
        par ^= 1;
        __syncthreads();
        stop_now = sh.decision != 0;
        if (sh.decision == 1) status = PJAC_OK;
        if (sh.decision == 2) status = PJAC_ETIMEOUT;
    };

    // ---- rotate rows/cols i,j for the owned indices, and V ----
    // Loads of the entries a rotation (i,j) changes, issued before the
    // rotation parameters are known (they depend only on i, j).
    double px[MR], py[MR], pvx[MR], pvy[MR];
    auto preload = [&](int i, int j) {
        const double* Ai = a.A + (long long)i * a.lda;
        const double* Aj = a.A + (long long)j * a.lda;
#pragma unroll
        for (int r = 0; r < MR; ++r) {
            int k = k0 + tid + r * NT;
            px[r] = py[r] = pvx[r] = pvy[r] = 0.0;
            if (k < k1) {
                px[r] = ldcg(Ai + k);
                py[r] = ldcg(Aj + k);
                if (a.V) {
                    pvx[r] = a.V[(long long)i * a.ldv + k];
                    pvy[r] = a.V[(long long)j * a.ldv + k];
                }
            }
        }
    };

    // pI (pJ): this thread's best entry of the new row i (row j) over its
    // owned columns; kI (kJ): the two largest keys among them.
    auto rotate_owned = [&](int i, int j, const double c, const double s, const double dii_new,
                            const double djj_new, bool score, bool withV, Cand& pI, Cand& pJ, int (&kI)[2],
                            int (&kJ)[2]) {
        double* Ai = a.A + (long long)i * a.lda;
        double* Aj = a.A + (long long)j * a.lda;
        const int cmin = min(i, j), cmax = max(i, j);
        const double di = diag[i], dj = diag[j];   // already updated
#pragma unroll
        for (int r = 0; r < MR; ++r) {
            int k = k0 + tid + r * NT;
            if (k >= k1) break;
            if (withV && a.V) {
                double* Vi = a.V + (long long)i * a.ldv;
                double* Vj = a.V + (long long)j * a.ldv;
                double vx = pvx[r], vy = pvy[r];
                Vi[k] = __fma_rn(c, vx, __dmul_rn(s, vy));
                Vj[k] = __fma_rn(c, vy, -__dmul_rn(s, vx));
            }
            if (k == i) {
                stcg(Ai + i, dii_new);
                stcg(Aj + i, 0.0);
                stcg(Ai + j, 0.0);
                if (score && a.K) {
                    const int kz = (pivot == PJAC_PIVOT_GREEDY) ? 0 : KEY_ZERO;
                    __stcg(a.K + (long long)j * a.ldk + i, kz);
                    __stcg(a.K + (long long)i * a.ldk + j, kz);
                }
                if (score) {
                    Cand z; z.key = (pivot == PJAC_PIVOT_GREEDY) ? 0 : KEY_ZERO; z.row = j; z.col = i;
                    z.pad = 0; z.x = 0.0; z.ex = -1.0;
                    if (better(z, pJ, pivot, diag)) pJ = z;
                    key_push(z.key, kJ[0], kJ[1]);
                }
                continue;
            }
            if (k == j) {
                stcg(Aj + j, djj_new);
                stcg(Ai + j, 0.0);
                stcg(Aj + i, 0.0);
                if (score) {
                    Cand z; z.key = (pivot == PJAC_PIVOT_GREEDY) ? 0 : KEY_ZERO; z.row = i; z.col = j;
                    z.pad = 0; z.x = 0.0; z.ex = -1.0;
                    if (better(z, pI, pivot, diag)) pI = z;
                    key_push(z.key, kI[0], kI[1]);
                }
                continue;
            }
            double x = px[r], y = py[r];
            double xn = __fma_rn(c, x, __dmul_rn(s, y));
            double yn = __fma_rn(c, y, -__dmul_rn(s, x));
            double* Ak = a.A + (long long)k * a.lda;
            stcg(Ai + k, xn);
            stcg(Aj + k, yn);
            stcg(Ak + i, xn);
            stcg(Ak + j, yn);
            if (!score) continue;
            if (r == 0) SLAP(5);
            double dk = diag[k];
            int kx, ky;
            if (pivot == PJAC_PIVOT_GREEDY) {
                kx = greedy_key(xn);
                ky = greedy_key(yn);
            } else {
                kx = gap_key(xn, __dadd_rn(dk, -di));
                ky = gap_key(yn, __dadd_rn(dk, -dj));
            }
            if (r == 0) SLAP(6);
            if (a.K) {
                __stcg(a.K + (long long)i * a.ldk + k, kx);
                __stcg(a.K + (long long)k * a.ldk + i, kx);
                __stcg(a.K + (long long)j * a.ldk + k, ky);
                __stcg(a.K + (long long)k * a.ldk + j, ky);
            }
            Cand ci; ci.key = kx; ci.row = i; ci.col = k; ci.pad = 0; ci.x = xn; ci.ex = -1.0;
            Cand cj; cj.key = ky; cj.row = j; cj.col = k; cj.pad = 0; cj.x = yn; cj.ex = -1.0;
            if (better(ci, pI, pivot, diag)) pI = ci;
            if (better(cj, pJ, pivot, diag)) pJ = cj;
            key_push(kx, kI[0], kI[1]);
            key_push(ky, kJ[0], kJ[1]);
            // own row k: only its entries (k,i), (k,j) changed
            Cand e1, e2;
            e1.row = k; e1.pad = 0; e1.ex = -1.0;
            e2 = e1;
            if (cmin == i) { e1.col = i; e1.key = kx; e1.x = xn; e2.col = j; e2.key = ky; e2.x = yn; }
            else           { e1.col = j; e1.key = ky; e1.x = yn; e2.col = i; e2.key = kx; e2.x = xn; }
            (void)cmax;
            Cand cur = cache[k - k0];
            Cand sec = cache2[k - k0];
            int F = cachef[k - k0];
            if (sec.key != KEY_NONE && (sec.col == i || sec.col == j)) sec = no_cand();
            bool lost = false;
            if (cur.key != KEY_NONE && (cur.col == i || cur.col == j)) {
                cur = sec;
                sec = no_cand();
                lost = true;
            }
            list_insert(e1, cur, sec, F, pivot, diag);
            list_insert(e2, cur, sec, F, pivot, diag);
            if (cur.key == KEY_NONE || (lost && !head_certified(cur, F, pivot))) {
                int slot = atomicAdd(&sh.nresc, 1);
                resc[slot] = k;
            } else {
                cache[k - k0] = cur;
                cache2[k - k0] = sec;
                cachef[k - k0] = F;
            }
            if (r == 0) SLAP(7);
        }
    };

    if (pivot == PJAC_PIVOT_RANDOM) {
        // Sec. 4.2's comparator: the pair of every step is drawn, not
        // selected; every CTA draws the same pair and computes the same
        // rotation from the entries the last cluster barrier made visible
        bool stop_now = false;
        for (;;) {
            if (rot % ce == 0) {
                offdiag_check(stop_now);
                if (stop_now) break;
            }
            if (rot >= a.max_rot) { status = PJAC_ENOCONV; break; }
            int i, j;
            random_pair(a.seed, rot, n, i, j);
            const double q = ldcg(a.A + (long long)i * a.lda + j);
            if (tid == 0) {
                Rot rp = rot_params(diag[i], diag[j], q);
                sh.c = rp.c; sh.s = rp.s;
                sh.dii = __fma_rn(rp.t, q, diag[i]);
                sh.djj = __fma_rn(-rp.t, q, diag[j]);
            }
            __syncthreads();
            const double c = sh.c, s = sh.s, dii = sh.dii, djj = sh.djj;
            __syncthreads();
            if (tid == 0) { diag[i] = dii; diag[j] = djj; }
            __syncthreads();
            Cand d1 = no_cand(), d2 = no_cand();
            int dk1[2] = {KEY_NONE, KEY_NONE}, dk2[2] = {KEY_NONE, KEY_NONE};
            preload(i, j);
            rotate_owned(i, j, c, s, dii, djj, false, true, d1, d2, dk1, dk2);
            rot++;
            cta_exchange_sync<CLUSTER>();
        }
        last_score = 0.0;
    } else if (pivot == PJAC_PIVOT_CYCLIC) {
        bool stop_now = false;
        for (;;) {
            offdiag_check(stop_now);
            if (stop_now) break;
            sweeps++;
            bool any = false;
            bool budget = false;
            for (int i = 0; i < n - 1 && !budget; ++i) {
                for (int j = i + 1; j < n; ++j) {
                    double q = ldcg(a.A + (long long)i * a.lda + j);
                    if (q == 0.0) continue;
                    if (rot >= a.max_rot) { budget = true; status = PJAC_ENOCONV; break; }
                    if (tid == 0) {
                        Rot rp = rot_params(diag[i], diag[j], q);
                        sh.c = rp.c; sh.s = rp.s;
                        sh.dii = __fma_rn(rp.t, q, diag[i]);
                        sh.djj = __fma_rn(-rp.t, q, diag[j]);
                    }
                    __syncthreads();
                    double c = sh.c, s = sh.s, dii = sh.dii, djj = sh.djj;
                    __syncthreads();
                    if (tid == 0) { diag[i] = dii; diag[j] = djj; }
                    __syncthreads();
                    Cand d1 = no_cand(), d2 = no_cand();
                    int dk1[2] = {KEY_NONE, KEY_NONE}, dk2[2] = {KEY_NONE, KEY_NONE};
                    preload(i, j);
                    rotate_owned(i, j, c, s, dii, djj, false, true, d1, d2, dk1, dk2);
                    rot++;
                    any = true;
                    cta_exchange_sync<CLUSTER>();
                }
            }
            if (budget) break;
            if (!any) { status = PJAC_OK; break; }
        }
        last_score = 0.0;
    } else {
        // initial scan (Sec. 3.2: O(n^2) scores once)
        for (int k = k0; k < k1; ++k) {
            Cand s2;
            int F;
            Cand b = rescan_row(a, k, diag, sh, s2, F, true);
            if (tid == 0) { cache[k - k0] = b; cache2[k - k0] = s2; cachef[k - k0] = F; }
        }
        if (CLUSTER && a.K) cta_exchange_sync<CLUSTER>();   // every row's keys are stored
        __syncthreads();
        // The pending pivot, the same in every thread after publish_select:
        // pdec (0 rotate, 1 converged, 2 time budget, 3 rotation budget),
        // indices and rotation.
        int pdec = 1, ppi = 0, ppj = 0;
        double pend_c = 1.0, pend_s = 0.0;
        // Publish this CTA's three candidates (best own row, its part of row
        // i, its part of row j) with their exact scores and tangents --
        // evaluated by three lanes at once, from one shared denominator --
        // push them into every rank's inbox, and select after the cluster
        // barrier.  The cosines and sines are not on the path to the
        // decision: after the barrier, while warp 0 decides, warps 5 and 6
        // finish them for every published candidate.  Every CTA ends with
        // the same winner in sh.sel and its rotation in pend_c, pend_s and
        // sh.t; the owners of rows i and j take those rows' new bests.
        // i, j < 0: no rows i, j (first selection).
        // Between the cluster barrier's arrive and its wait every thread
        // applies the rotation just made to its entries of V's columns i
        // and j (loaded at the top of the step): the V update is off the
        // path from one selection to the next.
        auto publish_select = [&](Cand loc, Cand pI, Cand pJ, const int (&kI)[2], const int (&kJ)[2], int i,
                                  int j, bool vupd, double vc, double vs) {
            if (tid < 3) {
                Cand c = (tid == 0) ? loc : (tid == 1 ? pI : pJ);
                double rd = 1.0, rq = 0.0, rt = 0.0;   // rot_cs: c = 1, s = 0
                if (c.key != KEY_NONE) {
                    int ci = min(c.row, c.col), cj = max(c.row, c.col);
                    EvalHead ev = eval_pair_head(diag[ci], diag[cj], c.x);
                    if (pivot != PJAC_PIVOT_GREEDY) c.ex = ev.l;
                    rd = ev.den;
                    rq = ev.q4;
                    rt = ev.t;
                }
                sh.stage.cand[tid] = c;
                sh.stage.prm[tid][0] = rd;
                sh.stage.prm[tid][1] = rq;
                sh.stage.prm[tid][2] = rt;
                if (tid == 0) {
                    sh.stage.sum = 0.0; sh.stage.flags = sh.tflag; sh.stage.pad = 0;
                    sh.stage.ki[0] = kI[0]; sh.stage.ki[1] = kI[1];
                    sh.stage.kj[0] = kJ[0]; sh.stage.kj[1] = kJ[1];
                }
            }
            SLAP(0);
            __syncwarp();
            if (tid < P) {
                if (CLUSTER) {
                    cg::cluster_group cl = cg::this_cluster();
                    *cl.map_shared_rank(&sh.inbox[par][rank], tid) = sh.stage;
                } else {
                    sh.inbox[par][0] = sh.stage;
                }
            }
            SLAP(1);
#ifdef PJAC_PROFILE
            const long long t_arr = clock64();
            if (tid == 0 && i >= 0 && rank < 16) atomicAdd(&g_rank[rank], (unsigned long long)(t_arr - sh.t_top));
#endif
            if (CLUSTER) asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
            if (vupd && a.V) {
                double* Vi = a.V + (long long)i * a.ldv;
                double* Vj = a.V + (long long)j * a.ldv;
#pragma unroll
                for (int r = 0; r < MR; ++r) {
                    const int k = k0 + tid + r * NT;
                    if (k < k1) {
                        const double vx = pvx[r], vy = pvy[r];
                        Vi[k] = __fma_rn(vc, vx, __dmul_rn(vs, vy));
                        Vj[k] = __fma_rn(vc, vy, -__dmul_rn(vs, vx));
                    }
                }
            }
            if (CLUSTER) asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
            else __syncthreads();
            LAP(5);
#ifdef PJAC_PROFILE
            const long long t_wait = clock64();
            if (tid == 0 && i >= 0 && rank < 16) atomicAdd(&g_rank[16 + rank], (unsigned long long)(t_wait - t_arr));
#define WLAP(k) do { if (rank == 0 && lane == 0) PROF_ADD(32 + (k), clock64() - t_wait); } while (0)
#else
#define WLAP(k) ((void)0)
#endif
            const int warp = tid >> 5, lane = tid & 31;
            if (warp == 0) {
                // the winner over all 3P published candidates, and the
                // decision on it, broadcast through shared memory
                Cand g = no_cand();
                for (int e = lane; e < 3 * P; e += 32) {
                    const Slot& sl = sh.inbox[par][e / 3];
                    const int q3 = e - 3 * (e / 3);
                    Cand c = sl.cand[q3];
                    c.pad = e;
                    if (better(c, g, pivot, diag)) g = c;
                }
                WLAP(4);
                g = warp_select(g, pivot, diag, nullptr);
                WLAP(5);
                if (lane == 0) {
                    double v = -1.0;
                    int dec = 0;
                    if (g.key == KEY_NONE) dec = 1;   // n < 2
                    else if (pivot == PJAC_PIVOT_GREEDY) {
                        v = fabs(g.x);
                        if (sbits(v) == 0) dec = 1;
                    } else {
                        v = cand_value(g, pivot, diag);   // exact score published with the candidate
                        if (sbits(v) == 0) dec = 1;
                        if (!dec && a.stop == PJAC_STOP_LIBOUND && sbits(v) <= sbits(sh.eps_li)) dec = 1;
                    }
                    if (!dec && rot >= a.max_rot) dec = 3;
                    if (sh.inbox[par][0].flags & 1) dec = 2;   // time budget spent
                    sh.decision = dec;
                    sh.sel = g;
                    if (sbits(v) >= 0) sh.q = v;
                    if (!dec) {
                        const int i2 = min(g.row, g.col), j2 = max(g.row, g.col);
                        const double* pr = sh.inbox[par][g.pad / 3].prm[g.pad % 3];
                        sh.pi = i2;
                        sh.pj = j2;
                        sh.win = g.pad;
                        sh.t = pr[2];
                        // the pending rotation's diagonal, undone if the
                        // convergence test stops before the rotation
                        sh.old_di = diag[i2];
                        sh.old_dj = diag[j2];
                        diag[i2] = __fma_rn(pr[2], g.x, sh.old_di);
                        diag[j2] = __fma_rn(-pr[2], g.x, sh.old_dj);
                    }
                    sh.nresc = 0;
                }
                WLAP(0);
            } else if (i >= 0 && (warp == 1 || warp == 2)) {
                // new heads of rows i and j and their bounds F; the owning
                // CTA writes them into its cache
                Cand c = no_cand();
                int ka = KEY_NONE, kb = KEY_NONE;   // two largest keys of the row
                if (lane < P) {
                    const Slot& sl = sh.inbox[par][lane];
                    c = sl.cand[warp];
                    c.pad = lane * 3 + warp;
                    ka = (warp == 1) ? sl.ki[0] : sl.kj[0];
                    kb = (warp == 1) ? sl.ki[1] : sl.kj[1];
                }
                c = warp_select(c, pivot, diag, nullptr);
                warp_top2_keys(ka, kb);
                const int row = (warp == 1) ? i : j;
                if (lane == 0 && row >= k0 && row < k1) {
                    cache[row - k0] = c;
                    cache2[row - k0] = no_cand();
                    cachef[row - k0] = bound_without_head(c, ka, kb);
                }
                if (warp == 1) WLAP(1);
            } else if (warp >= 5) {
                // cosine and sine of every published candidate's rotation
                // (warps 5 and 6: not on warp 0's scheduler, whose FP64
                // pipe the decision needs)
                const int e = (warp - 5) * 32 + lane;
                if (e < 3 * P) {
                    const double* pr = sh.inbox[par][e / 3].prm[e % 3];
                    rot_cs(pr[0], pr[1], pr[2], sh.cs[e][0], sh.cs[e][1]);
                }
                if (warp == 5) WLAP(2);
            }
            par ^= 1;
            __syncthreads();
            if (warp == 0) WLAP(3);
#undef WLAP
            pdec = sh.decision;
            ppi = sh.pi;
            ppj = sh.pj;
            if (pdec == 0) {
                pend_c = sh.cs[sh.win][0];
                pend_s = sh.cs[sh.win][1];
            }
        };

        // first selection
        {
            Cand loc = no_cand();
#pragma unroll
            for (int r = 0; r < MR; ++r) {
                int k = k0 + tid + r * NT;
                if (k >= k1) break;
                Cand c = cache[k - k0];
                if (better(c, loc, pivot, diag)) loc = c;
            }
            if (tid == 0) sh.tflag = 0;
            loc = block_select(loc, pivot, diag, sh);
            const int kn[2] = {KEY_NONE, KEY_NONE};
            publish_select(loc, no_cand(), no_cand(), kn, kn, -1, -1, false, 1.0, 0.0);
        }
        bool stop_now = false;
        long long until_check = 0;   // rotations to the next convergence test (rot mod ce == 0)
        for (;;) {
            LAP(7);
#ifdef PJAC_PROFILE
            sh.t_top = clock64();
#endif
            if (pdec == 2) { status = PJAC_ETIMEOUT; break; }
            if (pdec == 0) preload(ppi, ppj);   // the loads do not depend on the test below
            if (until_check == 0) {
                until_check = ce;
                offdiag_check(stop_now);
                if (stop_now) {
                    if (tid == 0 && pdec == 0) {   // the pending rotation is not applied
                        diag[ppi] = sh.old_di;
                        diag[ppj] = sh.old_dj;
                    }
                    break;
                }
            }
            LAP(0);
            SLAP(3);
            if (pdec == 1) { status = PJAC_OK; break; }
            if (pdec == 3) { status = PJAC_ENOCONV; break; }
            LAP(1);
            const int i = ppi, j = ppj;
            const double c = pend_c, s = pend_s, dii = diag[i], djj = diag[j];
            Cand pI = no_cand(), pJ = no_cand();
            int kI[2] = {KEY_NONE, KEY_NONE}, kJ[2] = {KEY_NONE, KEY_NONE};
            rotate_owned(i, j, c, s, dii, djj, true, false, pI, pJ, kI, kJ);
            SLAP(4);
            rot++;
            --until_check;
            __syncthreads();
            LAP(2);
            // rescans of owned rows whose best was in column i or j
            const int nr = sh.nresc;
            if (tid == 0) PROF_ADD(9, nr);
#ifdef PJAC_PROFILE
            const long long t_rs = clock64();
#endif
            for (int r = 0; r < nr; ++r) {
                int k = resc[r];
                Cand s2, b;
                int F;
                if (!(a.K && rescan_row_keys(a, k, diag, sh, b, s2, F))) b = rescan_row(a, k, diag, sh, s2, F);
                if (tid == 0) { cache[k - k0] = b; cache2[k - k0] = s2; cachef[k - k0] = F; }
            }
#ifdef PJAC_PROFILE
            if (rank == 0 && tid == 0 && nr > 0) { PROF_ADD(38, nr); PROF_ADD(39, clock64() - t_rs); }
#endif
            __syncthreads();
            LAP(3);
            if (tid == 0)
                sh.tflag = (rank == 0 && a.budget_ns > 0 && (long long)(now_ns() - start) > a.budget_ns) ? 1 : 0;
            Cand loc = no_cand();
#pragma unroll
            for (int r = 0; r < MR; ++r) {
                int k = k0 + tid + r * NT;
                if (k >= k1) break;
                if (k == i || k == j) continue;
                Cand& cc = cache[k - k0];   // exact scores computed here stay in the cache
                if (better(cc, loc, pivot, diag)) loc = cc;
            }
            Cand* wb = (loc.key != KEY_NONE) ? &cache[loc.row - k0] : nullptr;
            SLAP(2);
            cta_select3(loc, pI, pJ, pivot, diag, sh, kI, kJ, wb, cache, k0, k1);
            LAP(4);
            publish_select(loc, pI, pJ, kI, kJ, i, j, true, c, s);
            LAP(6);
        }
#undef LAP
#undef SLAP
        if (rank == 0 && tid == 0) PROF_ADD(10, rot);
        if (tid == 0) last_score = sh.sel.key == KEY_NONE ? 0.0 :
                          (pivot == PJAC_PIVOT_GREEDY ? fabs(sh.sel.x) : cand_value(sh.sel, pivot, diag));
    }

    // final off(A) and outputs
    double part = upper_offsum(a, rank, P, sh);
    if (tid == 0) sh.slots[par].sum = part;
    cta_exchange_sync<CLUSTER>();
    if (tid == 0) {
        double g = 0.0;
        for (int r = 0; r < P; ++r) g += peer_slot<CLUSTER>(sh, par, r)->sum;
        sh.q = off_from_sum(g, sh);
    }
    // keep peers' shared memory alive until everyone has read it
    cta_exchange_sync<CLUSTER>();
    for (int k = k0 + tid; k < k1; k += NT) a.Wd[k] = diag[k];
    if (rank == 0 && tid == 0 && a.info) {
        DevInfo inf;
        inf.rotations = rot;
        inf.sweeps = sweeps;
        inf.off = sh.q;
        inf.normf = sh.normf;
        inf.max_score = last_score;
        inf.status = status;
        inf.n = n;
        inf.steps = rot;
        *a.info = inf;
    }
}

size_t jacobi_smem_bytes(int n, int P) {
    int m = (n + P - 1) / P;
    return (size_t)n * sizeof(double) + 2 * (size_t)m * sizeof(Cand) + 2 * (size_t)m * sizeof(int) + 16;
}

template <bool CLUSTER>
__global__ void __launch_bounds__(NT, 1) jacobi_single_kernel(JacArgs a) {
    __shared__ Sh sh;
    extern __shared__ __align__(16) unsigned char dyn[];
    int P = 1, rank = 0;
    if (CLUSTER) {
        cg::cluster_group cl = cg::this_cluster();
        P = (int)cl.num_blocks();
        rank = (int)cl.block_rank();
    }
    int m = (a.n + P - 1) / P;
    double* diag = reinterpret_cast<double*>(dyn);
    Cand* cache = reinterpret_cast<Cand*>(diag + a.n);
    Cand* cache2 = cache + m;
    int* cachef = reinterpret_cast<int*>(cache2 + m);
    int* resc = cachef + m;
    jacobi_problem<CLUSTER, MAXR>(a, rank, P, sh, diag, cache, cache2, cachef, resc);
}

// Batched form: each CTA takes problems from a queue (largest first).  MR
// owned indices per thread: 1 when every order is <= NT (fewer registers,
// two CTAs per SM), else MAXR.
template <int MR>
__global__ void __launch_bounds__(NT, MR == 1 ? 2 : 1) jacobi_batched_kernel(const BatchDesc* desc, int nb,
                                                           const int* order, int* counter,
                                                           int pivot, int stop, double tol,
                                                           long long max_rot_per_n2,
                                                           long long budget_ns, unsigned long long seed) {
    __shared__ Sh sh;
    __shared__ int next;
    extern __shared__ __align__(16) unsigned char dyn[];
    for (;;) {
        if (threadIdx.x == 0) next = atomicAdd(counter, 1);
        __syncthreads();
        int t = next;
        __syncthreads();
        if (t >= nb) break;
        BatchDesc d = desc[order[t]];
        JacArgs a;
        a.A = d.A; a.lda = d.n; a.V = d.V; a.ldv = d.n; a.Wd = d.Wd; a.n = d.n;
        a.pivot = pivot; a.stop = stop; a.tol = tol;
        a.max_rot = max_rot_per_n2 * (long long)d.n * (long long)d.n;
        a.check_every = d.n; a.budget_ns = budget_ns; a.info = d.info; a.seed = seed;
        double* diag = reinterpret_cast<double*>(dyn);
        Cand* cache = reinterpret_cast<Cand*>(diag + d.n);
        Cand* cache2 = cache + d.n;
        int* cachef = reinterpret_cast<int*>(cache2 + d.n);
        int* resc = cachef + d.n;
        jacobi_problem<false, MR>(a, 0, 1, sh, diag, cache, cache2, cachef, resc);
        __syncthreads();
    }
}

int jacobi_auto_cluster(int n) {
    if (n <= 384) return 1;
    if (n <= 1024) return 4;
    if (n <= 2048) return 8;
    return 16;
}

cudaError_t launch_jacobi(const JacArgs& a, int P, cudaStream_t st) {
    if (P < 1) P = 1;
    int m = (a.n + P - 1) / P;
    if (m > NT * MAXR) return cudaErrorInvalidValue;
    size_t smem = jacobi_smem_bytes(a.n, P);
    if (P == 1) {
        cudaError_t e = cudaFuncSetAttribute(jacobi_single_kernel<false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        jacobi_single_kernel<false><<<1, NT, smem, st>>>(a);
        return cudaGetLastError();
    }
    cudaError_t e = cudaFuncSetAttribute(jacobi_single_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (P > 8) {
        e = cudaFuncSetAttribute(jacobi_single_kernel<true>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = P;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3(P);
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, jacobi_single_kernel<true>, a);
}

template <int MR>
static cudaError_t launch_batched_mr(const BatchDesc* d_desc, int nb, const int* d_order, int* d_counter,
                                     int pivot, int stop, double tol, long long max_rot_per_n2,
                                     long long budget_ns, size_t smem, int ctas, unsigned long long seed,
                                     cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(jacobi_batched_kernel<MR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    // no more CTAs than can be resident at once (the queue feeds them all)
    int dev = 0, sms = 148, per_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jacobi_batched_kernel<MR>, NT, smem);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    if (ctas > sms * per_sm) ctas = sms * per_sm;
    e = cudaMemsetAsync(d_counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    jacobi_batched_kernel<MR><<<ctas, NT, smem, st>>>(d_desc, nb, d_order, d_counter, pivot, stop, tol,
                                                      max_rot_per_n2, budget_ns, seed);
    return cudaGetLastError();
}

cudaError_t launch_jacobi_batched(const BatchDesc* d_desc, int nb, const int* d_order,
                                  int* d_counter, int pivot, int stop, double tol,
                                  long long max_rot_per_n2, long long budget_ns, int max_n,
                                  int ctas, unsigned long long seed, cudaStream_t st) {
    if (max_n > NT * MAXR) return cudaErrorInvalidValue;
    size_t smem = jacobi_smem_bytes(max_n, 1);
    if (max_n <= NT)
        return launch_batched_mr<1>(d_desc, nb, d_order, d_counter, pivot, stop, tol, max_rot_per_n2,
                                    budget_ns, smem, ctas, seed, st);
    return launch_batched_mr<MAXR>(d_desc, nb, d_order, d_counter, pivot, stop, tol, max_rot_per_n2,
                                   budget_ns, smem, ctas, seed, st);
}

// ---------------------------------------------------------------------------
// Readout: W ascending (ties by index), V's columns in the same order.
// ---------------------------------------------------------------------------
__global__ void rank_kernel(const double* Wd, int n, int* rank) {
    __shared__ unsigned long long tile[256];
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long mine = (k < n) ? order_key(Wd[k]) : 0ULL;
    int r = 0;
    for (int base = 0; base < n; base += 256) {
        int l = base + threadIdx.x;
        tile[threadIdx.x] = (l < n) ? order_key(Wd[l]) : ~0ULL;
        __syncthreads();
        int lim = min(256, n - base);
        for (int u = 0; u < lim; ++u) {
            unsigned long long o = tile[u];
            int l2 = base + u;
            r += (o < mine) || (o == mine && l2 < k);
        }
        __syncthreads();
    }
    if (k < n) rank[k] = r;
}

__global__ void gather_kernel(const double* Wd, const double* Vws, long long ldvws, int n,
                              const int* rank, double* W, double* V, long long ldv) {
    int col = blockIdx.y;
    int r = rank[col];
    if (blockIdx.x == 0 && threadIdx.x == 0) W[r] = Wd[col];
    if (V == nullptr) return;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x)
        V[(long long)r * ldv + row] = Vws[(long long)col * ldvws + row];
}

cudaError_t launch_readout(const double* Wd, const double* Vws, long long ldvws, int n,
                           double* W, double* V, long long ldv, int* rank_ws, cudaStream_t st) {
    rank_kernel<<<(n + 255) / 256, 256, 0, st>>>(Wd, n, rank_ws);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 g((n + 255) / 256, n);
    gather_kernel<<<g, 256, 0, st>>>(Wd, Vws, ldvws, n, rank_ws, W, V, ldv);
    return cudaGetLastError();
}

// Batched readout: one CTA per problem, sort by ranks in shared memory.
__global__ void readout_batched_kernel(const BatchDesc* desc, int nb) {
    extern __shared__ __align__(16) unsigned char dyn[];
    int p = blockIdx.x;
    if (p >= nb) return;
    BatchDesc d = desc[p];
    int n = d.n;
    unsigned long long* keys = reinterpret_cast<unsigned long long*>(dyn);
    int* rank = reinterpret_cast<int*>(keys + n);
    for (int k = threadIdx.x; k < n; k += blockDim.x) keys[k] = order_key(d.Wd[k]);
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        unsigned long long mine = keys[k];
        int r = 0;
        for (int l = 0; l < n; ++l) r += (keys[l] < mine) || (keys[l] == mine && l < k);
        rank[k] = r;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < n; k += blockDim.x) d.Wout[rank[k]] = d.Wd[k];
    if (d.Vout) {
        for (long long e = threadIdx.x; e < (long long)n * n; e += blockDim.x) {
            int col = (int)(e / n), row = (int)(e % n);
            d.Vout[(long long)rank[col] * n + row] = d.V[(long long)col * n + row];
        }
    }
}

cudaError_t launch_readout_batched(const BatchDesc* d_desc, int nb, int max_n, cudaStream_t st) {
    size_t smem = (size_t)max_n * (sizeof(unsigned long long) + sizeof(int));
    readout_batched_kernel<<<nb, 256, smem, st>>>(d_desc, nb);
    return cudaGetLastError();
}

__global__ void info_batched_kernel(const BatchDesc* desc, int nb, pjac_info* infos) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nb) return;
    DevInfo d = *desc[p].info;
    pjac_info o;
    o.rotations = d.rotations;
    double pairs = 0.5 * (double)d.n * (double)(d.n - 1);
    o.sweeps = (d.sweeps > 0) ? (double)d.sweeps : (pairs > 0 ? (double)d.rotations / pairs : 0.0);
    o.off_rel = d.normf > 0 ? d.off / d.normf : 0.0;
    o.max_score = d.max_score;
    o.status = d.status;
    o.n = d.n;
    o.ms_precond = 0.f;
    o.ms_transform = 0.f;
    o.ms_jacobi = 0.f;
    o.steps = d.steps;
    infos[p] = o;
}

__global__ void info_single_kernel(const DevInfo* src, pjac_info* dst) {
    DevInfo d = *src;
    pjac_info o;
    o.rotations = d.rotations;
    double pairs = 0.5 * (double)d.n * (double)(d.n - 1);
    o.sweeps = (d.sweeps > 0) ? (double)d.sweeps : (pairs > 0 ? (double)d.rotations / pairs : 0.0);
    o.off_rel = d.normf > 0 ? d.off / d.normf : 0.0;
    o.max_score = d.max_score;
    o.status = d.status;
    o.n = d.n;
    o.ms_precond = 0.f;
    o.ms_transform = 0.f;
    o.ms_jacobi = 0.f;
    o.steps = d.steps;
    *dst = o;
}

#ifdef PJAC_PROFILE
extern "C" int pjac_prof_read(unsigned long long* out, int reset) {
    cudaMemcpyFromSymbol(out, g_prof, sizeof(unsigned long long) * 40);
    if (reset) {
        unsigned long long z[40] = {0};
        cudaMemcpyToSymbol(g_prof, z, sizeof(z));
    }
    return 0;
}
extern "C" int pjac_prof_rank_read(unsigned long long* out, int reset) {
    cudaMemcpyFromSymbol(out, g_rank, sizeof(unsigned long long) * 32);
    if (reset) {
        unsigned long long z[32] = {0};
        cudaMemcpyToSymbol(g_rank, z, sizeof(z));
    }
    return 0;
}
#endif

cudaError_t launch_info_single(const DevInfo* src, pjac_info* dst, cudaStream_t st) {
    info_single_kernel<<<1, 1, 0, st>>>(src, dst);
    return cudaGetLastError();
}

cudaError_t launch_info_batched(const BatchDesc* d_desc, int nb, pjac_info* infos, cudaStream_t st) {
    info_batched_kernel<<<(nb + 127) / 128, 128, 0, st>>>(d_desc, nb, infos);
    return cudaGetLastError();
}

// Loads this file's kernels on the current device: asking for a kernel's
// attributes loads it, where a first launch would otherwise do so later.
cudaError_t preload_jacobi_kernels() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, jacobi_single_kernel<true>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, jacobi_single_kernel<false>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, jacobi_batched_kernel<1>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, jacobi_batched_kernel<MAXR>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, rank_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, gather_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, readout_batched_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, info_batched_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, info_single_kernel);
    return e;
}

}  // namespace pjac
