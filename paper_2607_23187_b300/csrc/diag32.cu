// Low-precision spectral decomposition of the preconditioner (Shao &
// Nakatsukasa, Sec. 2.1: A = V_l Lambda_l V_l^T + O(||A|| u_l), u_l = single
// precision as in Sec. 4).  The paper does not say which low-precision
// eigensolver to use; here it is a blocked parallel-order two-sided Jacobi
// method in FP32.
//
// The order-npad matrix (npad = n rounded up to 128; the padding rows and
// columns are zero, so every rotation that touches them is the identity and
// they never mix with the real indices) is cut into nb = npad/32 blocks of
// 32 indices.  A sweep is the nb-1 rounds of the round-robin tournament over
// the blocks.  In one round the nb/2 block pairs are disjoint; the two
// blocks of pair P form its 64-index super-block, and
//   phase 1  each pair's 64 x 64 diagonal super-block S_PP is diagonalised
//            in shared memory by inner parallel-order sweeps (63 rounds of
//            32 disjoint 2x2 rotations each); the product G_P of those
//            rotations is kept as E_P = G_P - I;
//   phase 2  every off-diagonal super-block becomes G_P^T S_PQ G_Q and the
//            accumulated basis becomes X G_P on the columns of P: dense
//            64 x 64 x 64 products in FP32.
// So a sweep streams the matrix through HBM nb-1 times instead of npad-1
// times for the scalar parallel order, and the streamed work is dense.
//
// Storage: the off-diagonal part in FP32 (kept exactly symmetric), the
// diagonal in FP64 (so rotations inside clusters narrower than FP32
// resolution still see their true differences), both scaled by a power of
// two that brings the largest entry into [1/2, 1) (the basis does not
// depend on the scale).  Two uses:
//   diag_fp32    the decomposition of fl32(A): the basis X starts at I and
//                is Q0 at the end;
//   refine_fp32  the same iteration on a nearly diagonal B = X^T fl32(A) X
//                formed with FP64 products; the basis is carried as
//                D = X - I (X <- X G  is  D <- D G + E), which keeps the
//                small D's relative precision.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>
#include "internal.h"

namespace cg = cooperative_groups;

namespace pjac {

namespace {

constexpr int BJ_NT = 256;   // threads per CTA
constexpr int BJ_LD = 68;    // row stride of the 64 x 64 GEMM operands in shared memory (float4 rows)
constexpr int BJ_ZLD = 65;   // odd row stride where a tile is read along columns
constexpr int BJ_TILE = 64 * BJ_LD;
constexpr size_t BJ_SMEM = 6 * BJ_TILE * sizeof(float);   // phase 2: six operand tiles (104,448 B)
// entries below this (after scaling the largest to [1/2, 1)) are not rotated
// away: far below the FP32 resolution of the matrix (and of the stopping
// tests), and their squares would leave the normal range
constexpr float BJ_TINY = 8.673617379884035e-19f;   // 2^-60

__host__ __device__ inline long long bj_npad(int n) { return ((long long)(n + 127) / 128) * 128; }

// workspace (floats): O[npad^2] | X[npad^2] | dg[npad] doubles |
// G[2][npairs][64*64] (G = I + E row-major, by round parity) |
// Gc[2][npairs][64*64] (the same G column-major) | Ed[2][npairs][64] (the
// diagonal of E) | acc[8] doubles | slots
struct BjWs {
    float* O;
    float* X;
    double* dg;
    float* G;
    float* Gc;
    float* Ed;
    double* acc;   // [0..3] convergence sums (two slots), [4] max |entry| (bit pattern)
    int* slots;
};

__host__ __device__ inline BjWs bj_ws(float* ws, int n) {
    const long long npad = bj_npad(n), nn = npad * npad, npairs = npad / 64;
    BjWs w;
    w.O = ws;
    w.X = ws + nn;
    w.dg = reinterpret_cast<double*>(ws + 2 * nn);
    w.G = ws + 2 * nn + 2 * npad;
    w.Gc = w.G + 2 * npairs * 4096;
    w.Ed = w.Gc + 2 * npairs * 4096;
    w.acc = reinterpret_cast<double*>(w.Ed + 2 * npairs * 64);
    w.slots = reinterpret_cast<int*>(w.acc + 8);
    return w;
}

// Round-robin tournament (circle method) on N players, N even: in round r
// pair 0 is (N-1, r) and pair k >= 1 is ((r+k) mod (N-1), (r-k) mod (N-1)).
__host__ __device__ __forceinline__ void circle_pair(int r, int k, int N, int& p, int& q) {
    if (k == 0) {
        p = N - 1;
        q = r;
    } else {
        p = (r + k) % (N - 1);
        q = (r - k + (N - 1)) % (N - 1);
    }
}

// global index of super-block index t of the pair (bi, bj)
__device__ __forceinline__ int sup_idx(int t, int bi, int bj) { return t < 32 ? bi * 32 + t : bj * 32 + t - 32; }

}  // namespace

// Z = G_a^T X G_b (G = [[c,-s],[s,c]]) for one 2x2 block, written as
// Z[u][v] = (t(0,0) + t(1,1)) + (t(0,1) + t(1,0)) with
// t(r,w) = (G_a[r][u] * G_b[w][v]) * X[r][w].  The block (b,a), computed
// from X^T with the roles of a and b exchanged, forms the same products and
// sums them in the same pairs, so it is exactly the transpose: a matrix
// stays exactly symmetric through every rotation.
__device__ __forceinline__ void rot2x2_sym(float ca, float sa, float cb, float sb, float x00, float x01,
                                           float x10, float x11, float& z00, float& z01, float& z10,
                                           float& z11) {
    const float ga[2][2] = {{ca, -sa}, {sa, ca}};
    const float gb[2][2] = {{cb, -sb}, {sb, cb}};
    const float x[2][2] = {{x00, x01}, {x10, x11}};
    float z[2][2];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            float t00 = __fmul_rn(__fmul_rn(ga[0][u], gb[0][v]), x[0][0]);
            float t11 = __fmul_rn(__fmul_rn(ga[1][u], gb[1][v]), x[1][1]);
            float t01 = __fmul_rn(__fmul_rn(ga[0][u], gb[1][v]), x[0][1]);
            float t10 = __fmul_rn(__fmul_rn(ga[1][u], gb[0][v]), x[1][0]);
            z[u][v] = __fadd_rn(__fadd_rn(t00, t11), __fadd_rn(t01, t10));
        }
    z00 = z[0][0]; z01 = z[0][1]; z10 = z[1][0]; z11 = z[1][1];
}

namespace {

// ---------------------------------------------------------------------------
// phase 1: one pair's diagonal super-block, inner sweeps in shared memory
// ---------------------------------------------------------------------------
// The diagonal is carried as an unevaluated sum hi + lo of two floats
// (about 48 significant bits): the differences d_p - d_q that steer the
// rotations stay accurate inside clusters far narrower than FP32 resolution,
// and every step runs on the FP32 pipes.
struct InnerSm {
    float S[64 * BJ_ZLD];   // off-diagonal part, full symmetric storage (row u, col v)
    float E[64 * BJ_ZLD];   // E = G - I
    float dh[64], dl[64];   // diagonal, hi + lo
    float4 prm[2][32];      // (c, s, c - 1, -) of the round's 32 rotations, by round parity
    int pq[2][32];          // p | q << 8
};
static_assert(sizeof(InnerSm) <= BJ_SMEM, "phase-1 shared memory");

// (h, l) += (ph, pl) for normalised float-float numbers (Knuth's TwoSum,
// then Dekker's FastTwoSum to renormalise)
__device__ __forceinline__ void ff_add(float& h, float& l, float ph, float pl) {
    const float s = h + ph;
    const float bb = s - h;
    float e = (h - (s - bb)) + (ph - bb);
    e = e + (l + pl);
    const float nh = s + e;
    l = e - (nh - s);
    h = nh;
}

// Warp 0: the rotations of inner round `ir` (pair table row ir) into buffer
// `buf`; the 2x2 diagonal blocks are finished here (t b moves into the
// diagonal, the pair's off-diagonal entry becomes zero).
__device__ __forceinline__ void inner_rotations(InnerSm& s, const unsigned short* __restrict__ ptab, int ir,
                                                int buf) {
    const int k = threadIdx.x;
    const int pqv = ptab[ir * 32 + k];
    const int p = pqv & 255, q = pqv >> 8;
    const float b = s.S[p * BJ_ZLD + q];
    float c = 1.0f, sn = 0.0f, cm1 = 0.0f;
    if (fabsf(b) >= BJ_TINY) {
        // d_p - d_q: the hi parts subtract exactly when they are close
        const float d = (s.dh[p] - s.dh[q]) + (s.dl[p] - s.dl[q]);
        // |d| < 2 and 2^-60 <= |b| < 1: no overflow, and 4 b^2 is normal
        const float den = fabsf(d) + sqrtf(fmaf(d, d, 4.0f * (b * b)));
        float t = __fdividef(2.0f * fabsf(b), den);
        if (d != 0.0f && ((d < 0.0f) != (b < 0.0f))) t = -t;
        c = rsqrtf(fmaf(t, t, 1.0f));
        sn = t * c;
        cm1 = __fdividef(-(t * t) * (c * c), 1.0f + c);   // c - 1 without cancellation
        const float ph = t * b, pl = fmaf(t, b, -ph);      // t b exactly
        ff_add(s.dh[p], s.dl[p], ph, pl);
        ff_add(s.dh[q], s.dl[q], -ph, -pl);
        s.S[p * BJ_ZLD + q] = 0.0f;
        s.S[q * BJ_ZLD + p] = 0.0f;
    }
    s.prm[buf][k] = make_float4(c, sn, cm1, 0.0f);
    s.pq[buf][k] = pqv;
}

__device__ void bj_inner(int k, int round, int nblk, long long npad, float* __restrict__ O,
                         double* __restrict__ dg, float* __restrict__ Gg, float* __restrict__ Gcg,
                         float* __restrict__ Edg, int inner_sweeps, float* sm,
                         const unsigned short* __restrict__ ptab) {
    InnerSm& s = *reinterpret_cast<InnerSm*>(sm);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int bi, bj;
    circle_pair(round, k, nblk, bi, bj);
    for (int e = tid; e < 4096; e += BJ_NT) {
        const int u = e & 63, v = e >> 6;
        s.S[u * BJ_ZLD + v] = __ldcg(O + sup_idx(u, bi, bj) + sup_idx(v, bi, bj) * npad);
        s.E[u * BJ_ZLD + v] = 0.0f;
    }
    if (tid < 64) {
        const double d = __ldcg(dg + sup_idx(tid, bi, bj));
        const float h = (float)d;
        s.dh[tid] = h;
        s.dl[tid] = (float)(d - (double)h);
    }
    __syncthreads();
    if (warp == 0) inner_rotations(s, ptab, 0, 0);
    __syncthreads();
    const int total = 63 * inner_sweeps;
    for (int g = 0; g < total; ++g) {
        const int buf = g & 1;
        // off-diagonal 2x2 blocks: warp-uniform row pair u, lane = column
        // pair v.  The blocks are disjoint, so all loads go first.
        {
            const int pqv = s.pq[buf][lane];
            const int pv = pqv & 255, qv = pqv >> 8;
            const float4 rv = s.prm[buf][lane];
            int pu[4], qu[4];
            float4 ru[4];
            float x[4][4];
#pragma unroll
            for (int it = 0; it < 4; ++it) {
                const int pqu = s.pq[buf][warp + 8 * it];
                pu[it] = pqu & 255;
                qu[it] = pqu >> 8;
                ru[it] = s.prm[buf][warp + 8 * it];
                x[it][0] = s.S[pu[it] * BJ_ZLD + pv];
                x[it][1] = s.S[pu[it] * BJ_ZLD + qv];
                x[it][2] = s.S[qu[it] * BJ_ZLD + pv];
                x[it][3] = s.S[qu[it] * BJ_ZLD + qv];
            }
#pragma unroll
            for (int it = 0; it < 4; ++it) {
                if (warp + 8 * it == lane) continue;   // the pair's own block: done with its rotation
                float z00, z01, z10, z11;
                rot2x2_sym(ru[it].x, ru[it].y, rv.x, rv.y, x[it][0], x[it][1], x[it][2], x[it][3], z00, z01, z10,
                           z11);
                s.S[pu[it] * BJ_ZLD + pv] = z00;
                s.S[pu[it] * BJ_ZLD + qv] = z01;
                s.S[qu[it] * BJ_ZLD + pv] = z10;
                s.S[qu[it] * BJ_ZLD + qv] = z11;
            }
        }
        __syncthreads();
        if (warp == 0) {
            if (g + 1 < total) inner_rotations(s, ptab, (g + 1) % 63, buf ^ 1);
        } else {
            // E <- E J + (J - I): rows lane and lane + 32 of the pairs
            // warp-1, warp+6, ... (at most 5); loads first
            float e0[5][2], e1[5][2];
            int pp[5], qq[5];
            float4 rr[5];
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                const int kk = warp - 1 + 7 * j;
                if (kk < 32) {
                    const int pqv = s.pq[buf][kk];
                    pp[j] = pqv & 255;
                    qq[j] = pqv >> 8;
                    rr[j] = s.prm[buf][kk];
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        e0[j][h] = s.E[(lane + 32 * h) * BJ_ZLD + pp[j]];
                        e1[j][h] = s.E[(lane + 32 * h) * BJ_ZLD + qq[j]];
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < 5; ++j) {
                if (warp - 1 + 7 * j >= 32) continue;
                const float4 r = rr[j];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int i = lane + 32 * h;
                    float v0 = e0[j][h] * r.x + e1[j][h] * r.y;
                    float v1 = -e0[j][h] * r.y + e1[j][h] * r.x;
                    if (i == pp[j]) { v0 += r.z; v1 -= r.y; }
                    if (i == qq[j]) { v0 += r.y; v1 += r.z; }
                    s.E[i * BJ_ZLD + pp[j]] = v0;
                    s.E[i * BJ_ZLD + qq[j]] = v1;
                }
            }
        }
        __syncthreads();
    }
    for (int e = tid; e < 4096; e += BJ_NT) {
        const int u = e & 63, v = e >> 6;
        __stcg(O + sup_idx(u, bi, bj) + sup_idx(v, bi, bj) * npad, s.S[u * BJ_ZLD + v]);
        const int r = e >> 6, cc = e & 63;   // G row-major, contiguous in cc
        const float ev = s.E[r * BJ_ZLD + cc];
        __stcg(Gg + (long long)k * 4096 + r * 64 + cc, r == cc ? 1.0f + ev : ev);
        const float et = s.E[cc * BJ_ZLD + r];   // column-major: element (cc, r) at [r][cc]
        __stcg(Gcg + (long long)k * 4096 + r * 64 + cc, r == cc ? 1.0f + et : et);
    }
    if (tid < 64) {
        dg[sup_idx(tid, bi, bj)] = (double)s.dh[tid] + (double)s.dl[tid];
        __stcg(Edg + (long long)k * 64 + tid, s.E[tid * BJ_ZLD + tid]);
    }
    __syncthreads();
}

// ---------------------------------------------------------------------------
// phase 2: dense 64 x 64 x 64 products in FP32
// ---------------------------------------------------------------------------
// Shared-memory tiles (64 x BJ_LD floats each): operand tiles L[2] and
// R[2] double-buffered so that the next unit's copies run under the
// current unit's products, G_P and T for the off-diagonal units.
constexpr int BJ_L0 = 0, BJ_R0 = 2, BJ_GP = 4, BJ_T = 5;

__device__ __forceinline__ void cp16(float* smem, const float* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// acc[a][b] = sum_k L[k][4ty+a] R[k][4tx+b]; L and R k-major with row
// stride BJ_LD.  A warp reads two distinct L rows (broadcast) and one
// 256-byte R row per k.
__device__ __forceinline__ void mm64(const float* __restrict__ L, const float* __restrict__ R, float acc[4][4]) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0f;
#pragma unroll 8
    for (int k = 0; k < 64; ++k) {
        const float4 x = *reinterpret_cast<const float4*>(L + k * BJ_LD + 4 * ty);
        const float4 y = *reinterpret_cast<const float4*>(R + k * BJ_LD + 4 * tx);
        const float xa[4] = {x.x, x.y, x.z, x.w};
        const float yb[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(xa[a], yb[b], acc[a][b]);
    }
}

// copies (in flight until the next wait) of G (row-major 64 x 64 in global)
// to dst[k*BJ_LD + j]
__device__ __forceinline__ void issue_g(const float* __restrict__ G, float* dst) {
    for (int f = threadIdx.x; f < 1024; f += BJ_NT) {
        const int k = f >> 4, j4 = (f & 15) * 4;
        cp16(dst + k * BJ_LD + j4, G + k * 64 + j4);
    }
}

// copies of the 64 x 64 tile M[row(u) + col(v)*npad] to dst[v*BJ_LD + u];
// rows are two runs of 32 (r0, r1) or one run of 64 (r1 = r0 + 32)
__device__ __forceinline__ void issue_tile(const float* __restrict__ M, long long npad, int r0, int r1, int c0,
                                           int c1, float* dst) {
    for (int f = threadIdx.x; f < 1024; f += BJ_NT) {
        const int v = f >> 4, u4 = (f & 15) * 4;
        const int gr = u4 < 32 ? r0 + u4 : r1 + u4 - 32;
        const int gc = v < 32 ? c0 + v : c1 + v - 32;
        cp16(dst + v * BJ_LD + u4, M + gr + (long long)gc * npad);
    }
}

__device__ __forceinline__ void store_acc4(float acc[4][4], float* dst) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int a = 0; a < 4; ++a)
        *reinterpret_cast<float4*>(dst + (4 * ty + a) * BJ_LD + 4 * tx) =
            make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
}

// [lo, hi): part `part` of `parts` equal contiguous shares of `count` units
__device__ __forceinline__ void unit_range(long long count, int part, int parts, long long& lo, long long& hi) {
    lo = count * part / parts;
    hi = count * (part + 1) / parts;
}

// pair indices of off-diagonal unit u (kp < kq, kp-major order)
__device__ __forceinline__ void off_unit(long long u, int npairs, int& kp, int& kq) {
    kp = 0;
    long long rem = u;
    while (rem >= npairs - 1 - kp) {
        rem -= npairs - 1 - kp;
        ++kp;
    }
    kq = kp + 1 + (int)rem;
}

// Off-diagonal units [lo, hi) of round `round`: S_PQ <- G_P^T S_PQ G_Q,
// written to S_PQ and, transposed, to S_QP.  Consecutive units share kp, so
// G_P is copied once per change of kp; the next unit's S_PQ and G_Q are
// copied during the current unit's products.
__device__ void run_off_units(long long lo, long long hi, int npairs, int round, int nblk, long long npad,
                              float* __restrict__ O, const float* __restrict__ Gg, float* sm) {
    if (lo >= hi) return;
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    float* Gp = sm + BJ_GP * BJ_TILE;
    float* Tb = sm + BJ_T * BJ_TILE;
    int kp, kq;
    off_unit(lo, npairs, kp, kq);
    {
        int pi, pj, qi, qj;
        circle_pair(round, kp, nblk, pi, pj);
        circle_pair(round, kq, nblk, qi, qj);
        issue_tile(O, npad, pi * 32, pj * 32, qi * 32, qj * 32, sm + BJ_L0 * BJ_TILE);
        issue_g(Gg + (long long)kq * 4096, sm + BJ_R0 * BJ_TILE);
        issue_g(Gg + (long long)kp * 4096, Gp);
        cp_commit();
    }
    int b = 0;
    for (long long u = lo; u < hi; ++u, b ^= 1) {
        int kp1 = kp, kq1 = kq;
        const bool more = u + 1 < hi;
        if (more) {
            off_unit(u + 1, npairs, kp1, kq1);
            int pi, pj, qi, qj;
            circle_pair(round, kp1, nblk, pi, pj);
            circle_pair(round, kq1, nblk, qi, qj);
            issue_tile(O, npad, pi * 32, pj * 32, qi * 32, qj * 32, sm + (BJ_L0 + (b ^ 1)) * BJ_TILE);
            issue_g(Gg + (long long)kq1 * 4096, sm + (BJ_R0 + (b ^ 1)) * BJ_TILE);
            cp_commit();
            cp_wait_prev();
        } else {
            cp_wait_all();
        }
        __syncthreads();
        float acc[4][4];
        mm64(sm + (BJ_L0 + b) * BJ_TILE, sm + (BJ_R0 + b) * BJ_TILE, acc);   // T = S_PQ G_Q
        store_acc4(acc, Tb);
        __syncthreads();
        mm64(Gp, Tb, acc);                                                    // Z = G_P^T T
        int pi, pj, qi, qj;
        circle_pair(round, kp, nblk, pi, pj);
        circle_pair(round, kq, nblk, qi, qj);
        // Z[i][j], i = 4ty + a (P side), j = 4tx + b (Q side): four
        // consecutive rows of a column, and four consecutive columns of a
        // row of the transpose, are 16-byte stores
        const int rP = sup_idx(4 * ty, pi, pj), rQ = sup_idx(4 * tx, qi, qj);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            *reinterpret_cast<float4*>(O + rP + (long long)(rQ + c) * npad) =
                make_float4(acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
            *reinterpret_cast<float4*>(O + rQ + (long long)(rP + c) * npad) =
                make_float4(acc[c][0], acc[c][1], acc[c][2], acc[c][3]);
        }
        if (more && kp1 != kp) {
            __syncthreads();   // everyone is done with G_P
            issue_g(Gg + (long long)kp1 * 4096, Gp);
            cp_commit();
            cp_wait_all();
        }
        kp = kp1;
        kq = kq1;
    }
    __syncthreads();
}

// Basis units on the FP32 pipes (the refinement pass, whose products must
// keep FP32 accuracy relative to the correction D): round `round` (G of
// that round in Gg, E's diagonal in
// Edg): unit v is the 64 rows [64 (v % nrt), +64) of the columns of pair
// v / nrt, X <- X G, plus E = G - I on the pair's own rows when the basis is
// carried as D = X - I.  Units are taken one at a time from the queue
// counter *xq (zero at the start of the step), one unit ahead so that its
// copies run under the current unit's product; CTAs that finish their inner
// solve early take more.
__device__ void run_basis_queue_simt(int* xq, long long nX, long long nrt, int round, int nblk, long long npad,
                                float* __restrict__ X, const float* __restrict__ Gg, const float* __restrict__ Edg,
                                int delta, float* sm, long long* s_next) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    if (threadIdx.x == 0) *s_next = atomicAdd(xq, 1);
    __syncthreads();
    long long v = *s_next;
    __syncthreads();
    auto issue = [&](long long unit, int buf) {
        const int k = (int)(unit / nrt), r0 = (int)(unit % nrt) * 64;
        int bi, bj;
        circle_pair(round, k, nblk, bi, bj);
        issue_tile(X, npad, r0, r0 + 32, bi * 32, bj * 32, sm + (BJ_L0 + buf) * BJ_TILE);
        issue_g(Gg + (long long)k * 4096, sm + (BJ_R0 + buf) * BJ_TILE);
        cp_commit();
    };
    if (v < nX) issue(v, 0);
    int b = 0;
    while (v < nX) {
        if (threadIdx.x == 0) *s_next = atomicAdd(xq, 1);
        __syncthreads();
        const long long vn = *s_next;
        if (vn < nX) {
            issue(vn, b ^ 1);
            cp_wait_prev();
        } else {
            cp_wait_all();
        }
        __syncthreads();
        const float* Rb = sm + (BJ_R0 + b) * BJ_TILE;
        float acc[4][4];
        mm64(sm + (BJ_L0 + b) * BJ_TILE, Rb, acc);
        const int k = (int)(v / nrt), r0 = (int)(v % nrt) * 64;
        int bi, bj;
        circle_pair(round, k, nblk, bi, bj);
        const int g0 = r0 + 4 * ty;   // this thread's four rows
        if (delta) {
            const int blk = g0 >> 5;
            if (blk == bi || blk == bj) {
                const int t0 = blk == bi ? g0 - bi * 32 : 32 + g0 - bj * 32;
#pragma unroll
                for (int a = 0; a < 4; ++a)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const int t = t0 + a, j = 4 * tx + c;
                        acc[a][c] += t == j ? __ldcg(Edg + (long long)k * 64 + t) : Rb[t * BJ_LD + j];
                    }
            }
        }
        const int cQ = sup_idx(4 * tx, bi, bj);
#pragma unroll
        for (int c = 0; c < 4; ++c)
            *reinterpret_cast<float4*>(X + g0 + (long long)(cQ + c) * npad) =
                make_float4(acc[0][c], acc[1][c], acc[2][c], acc[3][c]);
        __syncthreads();   // L[b], R[b] and s_next free again
        v = vn;
        b ^= 1;
    }
}

// ---------------------------------------------------------------------------
// basis units on the tensor cores: X <- X G for 128 rows of the pair's 64
// columns, one tcgen05.mma chain of kind::tf32 (M = 128, N = 64, K = 8 per
// instruction) into a TMEM accumulator.  FP32 accuracy from TF32 operands by
// the three-term split x = hi + lo (hi: x with its low 13 mantissa bits
// cleared, lo = x - hi exactly): X G ~ Xhi Ghi + Xhi Glo + Xlo Ghi, whose
// dropped term and the truncation of lo are below 2^-20 of |X||G| per
// product.  Operands are staged through registers into the K-major
// 128-byte-swizzled shared-memory layout the matrix descriptors describe.
// ---------------------------------------------------------------------------
constexpr int TC_A_BYTES = 128 * 128;   // 128 rows x 32 K (FP32) = one swizzle column
constexpr int TC_B_BYTES = 64 * 128;    // 64 rows x 32 K
// layout inside the (1024-byte aligned) unit buffer: A hi [2 K-halves], A lo, B hi, B lo
constexpr int TC_OFF_AHI = 0, TC_OFF_ALO = 2 * TC_A_BYTES, TC_OFF_BHI = 4 * TC_A_BYTES,
              TC_OFF_BLO = 4 * TC_A_BYTES + 2 * TC_B_BYTES;
constexpr int TC_BYTES = 4 * TC_A_BYTES + 4 * TC_B_BYTES;   // 96 KB
constexpr int TC_TMEM_COLS = 64;
static_assert(TC_BYTES + 1023 <= (int)BJ_SMEM, "tensor-core operands in the dynamic shared memory");
// instruction descriptor: D FP32, A and B TF32, both K-major, N = 64, M = 128
constexpr uint32_t TC_IDESC = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(64 >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
// byte offset of element (row r, k) (k < 32) in a K-major tile of 128-byte
// rows with the 128-byte swizzle (16-byte chunk c of row r at c ^ (r mod 8))
__device__ __forceinline__ uint32_t sw128_off(int r, int k) {
    return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((((k >> 2) ^ (r & 7)) << 4) | ((k & 3) << 2)));
}
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);   // start address
    d |= (uint64_t)1 << 16;                     // leading-dimension offset (unused with this swizzle)
    d |= (uint64_t)(1024 >> 4) << 32;           // stride between 8-row groups
    d |= (uint64_t)1 << 46;                     // descriptor version
    d |= (uint64_t)2 << 61;                     // 128-byte swizzle
    return d;
}
__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
    hi = __uint_as_float(__float_as_uint(x) & 0xffffe000u);
    lo = x - hi;   // exact: x and hi share sign and exponent
}
__device__ __forceinline__ void tc_mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
        "l"(a), "l"(b), "r"(TC_IDESC), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tc_commit_to(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
          "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// bounded wait on the MMA completion barrier; false (and *err set) when the
// bound runs out
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, int* err) {
    const uint32_t a = smem_u32(bar);
    for (long long it = 0; it < (1LL << 24); ++it) {
        uint32_t ok;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
            : "=r"(ok)
            : "r"(a), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    atomicExch(err, 1);
    return false;
}

// Basis units of round `round` (G of that round in Gg row-major and Gcg
// column-major, E's diagonal in Edg): unit v is the 128 rows
// [128 (v % nrb), +128) of the columns of pair v / nrb, X <- X G, plus
// E = G - I on the pair's own rows when the basis is carried as D = X - I.
// Units are taken one at a time from the queue counter *xq (zero at the
// start of the step); CTAs that finish their inner solve early take more.
// tc: the CTA's TMEM accumulator, bar/phase: its MMA completion barrier.
__device__ __forceinline__ void tc_tile_coords(int e, int& r4, int& c) {
    const int ln = e & 31, grp = e >> 5;
    r4 = (grp & 15) * 8 + (ln & 1) * 4;
    c = (grp >> 4) * 16 + (ln >> 1);
}

// four of the thread's eight 16-byte loads of a 128 x 64 basis tile (half h)
__device__ __forceinline__ void tc_load_half(const float* __restrict__ X, long long npad, int r0, int bi, int bj,
                                             int h, float4 (&xv)[4]) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int r4, c;
        tc_tile_coords(threadIdx.x + 256 * (4 * h + u), r4, c);
        xv[u] = __ldcg(reinterpret_cast<const float4*>(X + r0 + r4 + (long long)sup_idx(c, bi, bj) * npad));
    }
}

// split and swizzled stores of the loads of tc_load_half
__device__ __forceinline__ void tc_store_half(unsigned char* tcs, int h, const float4 (&xv)[4]) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        int r4, c;
        tc_tile_coords(threadIdx.x + 256 * (4 * h + u), r4, c);
        const float xs[4] = {xv[u].x, xv[u].y, xv[u].z, xv[u].w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float hi, lo;
            split_tf32(xs[i], hi, lo);
            const uint32_t off = (uint32_t)((c >> 5) * TC_A_BYTES) + sw128_off(r4 + i, c & 31);
            *reinterpret_cast<float*>(tcs + TC_OFF_AHI + off) = hi;
            *reinterpret_cast<float*>(tcs + TC_OFF_ALO + off) = lo;
        }
    }
}

__device__ void run_basis_queue(int* xq, long long nX, long long nrb, int round, int nblk, long long npad,
                                float* __restrict__ X, const float* __restrict__ Gg,
                                const float* __restrict__ Gcg, const float* __restrict__ Edg, int delta,
                                unsigned char* tcs, uint32_t tmem, uint64_t* bar, uint32_t& phase, int* err,
                                long long* s_next) {
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // a software pipeline over the CTA's units: the queue index of the next
    // unit is fetched, and the first half of its tile loaded, while the
    // current unit's products run
    if (tid == 0) *s_next = atomicAdd(xq, 1);
    __syncthreads();
    long long v = *s_next;
    __syncthreads();
    float4 xa[4];
    if (v < nX) {
        int bi, bj;
        circle_pair(round, (int)(v / nrb), nblk, bi, bj);
        tc_load_half(X, npad, (int)(v % nrb) * 128, bi, bj, 0, xa);
    }
    while (v < nX) {
        if (tid == 0) *s_next = atomicAdd(xq, 1);
        const int k = (int)(v / nrb), r0 = (int)(v % nrb) * 128;
        int bi, bj;
        circle_pair(round, k, nblk, bi, bj);
        // A = X[r0 .. r0+128, pair k's columns]: a warp covers 8 rows (two
        // lanes per column) x 16 columns, so each swizzled store hits 32
        // distinct banks
        tc_store_half(tcs, 0, xa);
        tc_load_half(X, npad, r0, bi, bj, 1, xa);
        // B = G as N x K (row n = column j of G, K = t)
        const float* gc = Gcg + (long long)k * 4096;
        tc_store_half(tcs, 1, xa);
        for (int h8 = 0; h8 < 16; h8 += 8) {
            float gv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int grp = (tid + 256 * (h8 + u)) >> 5;
                const int nrow = (grp & 7) * 8 + (lane & 7), t = (grp >> 3) * 4 + (lane >> 3);
                gv[u] = __ldcg(gc + nrow * 64 + t);
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int grp = (tid + 256 * (h8 + u)) >> 5;
                const int nrow = (grp & 7) * 8 + (lane & 7), t = (grp >> 3) * 4 + (lane >> 3);
                float h, l;
                split_tf32(gv[u], h, l);
                const uint32_t off = (uint32_t)((t >> 5) * TC_B_BYTES) + sw128_off(nrow, t & 31);
                *reinterpret_cast<float*>(tcs + TC_OFF_BHI + off) = h;
                *reinterpret_cast<float*>(tcs + TC_OFF_BLO + off) = l;
            }
        }
        // the operands, written by the generic proxy, are read by the tensor cores
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        const long long vn = *s_next;
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t base = smem_u32(tcs);
            uint32_t acc = 0;
#pragma unroll
            for (int kh = 0; kh < 2; ++kh)
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t ahi = sw128_desc(base + TC_OFF_AHI + kh * TC_A_BYTES) + 2 * kk;
                    const uint64_t alo = sw128_desc(base + TC_OFF_ALO + kh * TC_A_BYTES) + 2 * kk;
                    const uint64_t bhi = sw128_desc(base + TC_OFF_BHI + kh * TC_B_BYTES) + 2 * kk;
                    const uint64_t blo = sw128_desc(base + TC_OFF_BLO + kh * TC_B_BYTES) + 2 * kk;
                    tc_mma_tf32(tmem, alo, bhi, acc);
                    acc = 1;
                    tc_mma_tf32(tmem, ahi, blo, 1);
                    tc_mma_tf32(tmem, ahi, bhi, 1);
                }
            tc_commit_to(bar);
        }
        // the next unit's first loads run under the products
        if (vn < nX) {
            int ni, nj;
            circle_pair(round, (int)(vn / nrb), nblk, ni, nj);
            tc_load_half(X, npad, (int)(vn % nrb) * 128, ni, nj, 0, xa);
        }
        // every thread waits; the outcome is made uniform (tcgen05.ld is a
        // whole-warp instruction)
        const bool done = __syncthreads_and(tc_wait(bar, phase, err) ? 1 : 0) != 0;
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        if (done) {
            // warp w reads TMEM lanes 32 (w mod 4) .. (rows) and columns 32 (w / 4) ..
            const int q = warp & 3, ch = warp >> 2;
            const int r = q * 32 + lane, g = r0 + r;
            int t0 = -1;
            if (delta) {
                const int blk = g >> 5;
                if (blk == bi) t0 = g - bi * 32;
                else if (blk == bj) t0 = 32 + g - bj * 32;
            }
            for (int half = 0; half < 2; ++half) {
                uint32_t vv[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(ch * 32 + half * 16), vv);
#pragma unroll
                for (int c = 0; c < 16; ++c) {
                    const int j = ch * 32 + half * 16 + c;
                    float z = __uint_as_float(vv[c]);
                    if (t0 >= 0)
                        z += (t0 == j) ? __ldcg(Edg + (long long)k * 64 + t0)
                                       : __ldcg(Gg + (long long)k * 4096 + t0 * 64 + j);
                    X[g + (long long)sup_idx(j, bi, bj) * npad] = z;
                }
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();   // shared operands and the accumulator free again; s_next read by all
        v = vn;
    }
}

// The whole iteration in one cooperative launch.  Per round r:
//   step 1  inner solves of round r (one CTA per pair) and the basis update
//           of round r - 1 (it only needs E of that round, kept in the other
//           parity buffer), taken from a queue by every CTA once its inner
//           solve, if any, is done;
//   step 2  the off-diagonal super-blocks of round r on every CTA;
// grid-wide barriers between the steps.  The basis update of the last round
// runs once the iteration stops.  The convergence test after each sweep is
// taken by every CTA from the same global sums.
//   delta = 0: S = fl32(A) (its diagonal too), basis X = I;  out = X
//   delta = 1: S = B with the FP64 diagonal, D = 0;           out = D
// acc[4] must be zero at launch (the scale's maximum is reduced into it).
template <bool TC>
__global__ void __launch_bounds__(BJ_NT, 2) bjac32_coop_kernel(const double* __restrict__ A, long long lda, int n,
                                                               float* ws, float* __restrict__ out, int max_sweeps,
                                                               int inner_sweeps, int delta, double stop_tol,
                                                               int slot) {
    cg::grid_group grid = cg::this_grid();
    extern __shared__ __align__(16) float sm[];
    __shared__ unsigned short ptab[63 * 32];
    __shared__ double s_off[BJ_NT / 32], s_all[BJ_NT / 32];
    __shared__ long long s_chunk;
    __shared__ __align__(8) uint64_t tc_bar;   // completion of the basis unit's MMA chain
    __shared__ uint32_t tc_slot;                // TMEM address of the accumulator
    const long long npad = bj_npad(n), nn = npad * npad;
    const BjWs w = bj_ws(ws, n);
    int* xq = w.slots + 2;   // basis-unit queue of the current step 1
    int* tc_err = w.slots + 3;   // set when a wait for the tensor cores runs out
    // the tensor cores' operand buffer: 1024-byte aligned for the swizzle
    unsigned char* tcs = reinterpret_cast<unsigned char*>(
        (reinterpret_cast<uintptr_t>(sm) + 1023) & ~(uintptr_t)1023);
    if (TC) {
        if (threadIdx.x == 0) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&tc_bar)) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        if (threadIdx.x < 32) {
            asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                             smem_u32(&tc_slot)),
                         "r"(TC_TMEM_COLS)
                         : "memory");
            asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
        }
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    }
    __syncthreads();
    if (TC) asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = TC ? tc_slot : 0u;
    uint32_t tc_phase = 0;
    const int nblk = (int)(npad / 32), npairs = nblk / 2;
    const long long gstride = (long long)gridDim.x * blockDim.x;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (int t = threadIdx.x; t < 63 * 32; t += BJ_NT) {
        int p, q;
        circle_pair(t >> 5, t & 31, 64, p, q);
        ptab[t] = (unsigned short)(p | (q << 8));
    }
    // scale 2^-e with max |A| * 2^-e in [1/2, 1)
    {
        double mx = 0.0;
        for (long long e = gtid; e < (long long)n * n; e += gstride) {
            const int r = (int)(e % n), c = (int)(e / n);
            mx = fmax(mx, fabs(A[r + (long long)c * lda]));
        }
        for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
        if ((threadIdx.x & 31) == 0) s_off[threadIdx.x >> 5] = mx;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int k = 1; k < BJ_NT / 32; ++k) mx = fmax(mx, s_off[k]);
            atomicMax(reinterpret_cast<unsigned long long*>(w.acc + 4), (unsigned long long)__double_as_longlong(mx));
        }
    }
    grid.sync();
    int ex = 0;
    {
        const double mx = __ldcg(w.acc + 4);
        if (mx > 0.0) frexp(mx, &ex);
        ex = max(ex, -1000);   // keep 2^-ex finite for matrices of subnormal numbers
    }
    const double scale = ldexp(1.0, -ex);
    for (long long e = gtid; e < nn; e += gstride) {
        const int r = (int)(e % npad), c = (int)(e / npad);
        w.O[e] = (r != c && r < n && c < n) ? (float)(A[r + (long long)c * lda] * scale) : 0.0f;
        w.X[e] = (!delta && r == c) ? 1.0f : 0.0f;
    }
    for (long long p = gtid; p < npad; p += gstride) {
        double d = 0.0;
        if (p < n) {
            d = A[p + p * lda] * scale;
            if (!delta) d = (double)(float)d;
        }
        w.dg[p] = d;
    }
    if (gtid < 4) w.acc[gtid] = 0.0;
    if (gtid == 0) {
        *xq = 0;
        *tc_err = 0;
    }
    grid.sync();
    const long long nA = (long long)npairs * (npairs - 1) / 2;
    const long long nrb = npad / 128, nrt = npad / 64;
    const long long nX = nrb * npairs;    // tensor-core basis units (128 rows)
    const long long nXs = nrt * npairs;   // FP32-pipe basis units (64 rows)
    long long ax_lo, ax_hi;
    unit_range(nA, blockIdx.x, gridDim.x, ax_lo, ax_hi);
    const long long gbuf = (long long)npairs * 4096, ebuf = (long long)npairs * 64;
    long long gr = 0;          // rounds done (all sweeps): parity of the G buffers
    int pend_round = -1;       // round whose basis update is pending
    double prev = -1.0;
    int done = max_sweeps;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        for (int r = 0; r < nblk - 1; ++r, ++gr) {
            float* Gr = w.G + (gr & 1) * gbuf;
            float* Gcr = w.Gc + (gr & 1) * gbuf;
            float* Er = w.Ed + (gr & 1) * ebuf;
            for (int k = blockIdx.x; k < npairs; k += gridDim.x)
                bj_inner(k, r, nblk, npad, w.O, w.dg, Gr, Gcr, Er, inner_sweeps, sm, ptab);
            if (pend_round >= 0) {
                if (!TC || delta)
                    run_basis_queue_simt(xq, nXs, nrt, pend_round, nblk, npad, w.X, w.G + ((gr - 1) & 1) * gbuf,
                                         w.Ed + ((gr - 1) & 1) * ebuf, delta, sm, &s_chunk);
                else
                    run_basis_queue(xq, nX, nrb, pend_round, nblk, npad, w.X, w.G + ((gr - 1) & 1) * gbuf,
                                    w.Gc + ((gr - 1) & 1) * gbuf, w.Ed + ((gr - 1) & 1) * ebuf, delta, tcs, tmem,
                                    &tc_bar, tc_phase, tc_err, &s_chunk);
            }
            grid.sync();
            if (gtid == 0) *xq = 0;   // nobody takes from the queue until the next step 1
            run_off_units(ax_lo, ax_hi, npairs, r, nblk, npad, w.O, Gr, sm);
            pend_round = r;
            grid.sync();
        }
        // off(S)^2 and ||S||_F^2
        double off = 0.0, all = 0.0;
        for (long long e = gtid; e < nn; e += gstride) {
            const double v = (double)__ldcg(w.O + e);
            off += v * v;
        }
        for (long long p = gtid; p < npad; p += gstride) {
            const double d = __ldcg(w.dg + p);
            all += d * d;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            all += __shfl_xor_sync(0xffffffffu, all, o);
        }
        if ((threadIdx.x & 31) == 0) {
            s_off[threadIdx.x >> 5] = off;
            s_all[threadIdx.x >> 5] = all;
        }
        __syncthreads();
        double* acc = w.acc + 2 * (sweep & 1);
        if (threadIdx.x == 0) {
            double o2 = 0, a2 = 0;
            for (int k = 0; k < BJ_NT / 32; ++k) {
                o2 += s_off[k];
                a2 += s_all[k];
            }
            atomicAdd(acc, o2);
            atomicAdd(acc + 1, a2 + o2);
        }
        grid.sync();
        const double o2 = __ldcg(acc), a2 = __ldcg(acc + 1);
        // converged, or no longer improving.  The first sweeps from a poor
        // start shrink off(S) only by a small factor (linear phase while
        // off(S) is above the cluster gaps), so the stagnation test waits.
        const bool stop = (a2 == 0.0 || o2 <= stop_tol * a2) || (sweep >= 4 && prev >= 0.0 && o2 > 0.9 * prev);
        prev = o2;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            double* other = w.acc + 2 * ((sweep + 1) & 1);
            other[0] = 0.0;
            other[1] = 0.0;
        }
        if (stop) {
            done = sweep + 1;
            break;
        }
        grid.sync();   // the other slot is zero before anyone adds to it
    }
    // the last round's basis update
    if (pend_round >= 0) {
        if (!TC || delta)
            run_basis_queue_simt(xq, nXs, nrt, pend_round, nblk, npad, w.X, w.G + ((gr - 1) & 1) * gbuf,
                                 w.Ed + ((gr - 1) & 1) * ebuf, delta, sm, &s_chunk);
        else
            run_basis_queue(xq, nX, nrb, pend_round, nblk, npad, w.X, w.G + ((gr - 1) & 1) * gbuf,
                            w.Gc + ((gr - 1) & 1) * gbuf, w.Ed + ((gr - 1) & 1) * ebuf, delta, tcs, tmem, &tc_bar,
                            tc_phase, tc_err, &s_chunk);
    }
    grid.sync();
    if (blockIdx.x == 0 && threadIdx.x == 0) w.slots[slot] = done;
    // indices never move, so the basis is in the original column order;
    // the padding columns are unit vectors of padding rows and are dropped
    const long long tot = (long long)n * n;
    for (long long e = gtid; e < tot; e += gstride) {
        const int r = (int)(e % n), c = (int)(e / n);
        out[e] = __ldcg(w.X + r + (long long)c * npad);
    }
    if (TC) {
        asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
        __syncthreads();
        if (threadIdx.x < 32) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS)
                         : "memory");
        }
    }
}

int bj_inner_sweeps() { return 1; }

cudaError_t bj_launch(const double* A, long long lda, int n, float* out, float* ws, int max_sweeps, int delta,
                      double stop_tol, int slot, int max_grid, cudaStream_t st) {
    // the tensor cores take the first pass's basis updates while the two
    // FP32 matrices fit in L2 (npad <= 2048: 32 MB); at larger orders the
    // units' staging through registers waits on DRAM and the FP32-pipe
    // units with their asynchronous copies are faster (measured at 4096)
    const bool tc = delta == 0 && bj_npad(n) <= 2048;
    const void* kern = tc ? (const void*)bjac32_coop_kernel<true> : (const void*)bjac32_coop_kernel<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BJ_SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, BJ_NT, BJ_SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const BjWs w = bj_ws(ws, n);
    e = cudaMemsetAsync(w.acc, 0, 8 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const long long npad = bj_npad(n);
    const long long npairs = npad / 64;
    const long long units = std::max(npairs * (npairs - 1) / 2, npairs + (npad / 128) * npairs);
    int grid = (int)std::min<long long>((long long)sms * std::min(per_sm, 2), units);
    if (max_grid > 0 && grid > max_grid) grid = max_grid;   // share the GPU (all CTAs must be co-resident)
    int inner = bj_inner_sweeps();
    void* args[] = {(void*)&A,      (void*)&lda,   (void*)&n,        (void*)&ws,   (void*)&out,
                    (void*)&max_sweeps, (void*)&inner, (void*)&delta, (void*)&stop_tol, (void*)&slot};
    return cudaLaunchCooperativeKernel(kern, dim3(grid), dim3(BJ_NT), args, BJ_SMEM,
                                       st);
}

}  // namespace

size_t diag_fp32_ws_floats(int n) {
    const long long npad = bj_npad(n), npairs = npad / 64;
    return (size_t)(2 * npad * npad + 2 * npad + 2 * npairs * (2 * 4096 + 64) + 16 + 16);   // ... acc[8] | slots[3]
}

// Q0 <- eigenvectors of fl32(A) (n x n, ld n).  ws: diag_fp32_ws_floats(n)
// floats, 16-byte aligned.  One cooperative launch; nothing waits on the host.
cudaError_t diag_fp32(const double* A, long long lda, int n, float* Q0, float* ws, int* iws, int max_sweeps,
                      int max_grid, cudaStream_t st) {
    (void)iws;
    return bj_launch(A, lda, n, Q0, ws, max_sweeps, 0, 1e-15, 0, max_grid, st);
}

// D with X (I + D) an eigenbasis of fl32(A) to FP32 accuracy, from
// B = X^T fl32(A) X (n x n, ld n, nearly diagonal).
cudaError_t refine_fp32(const double* B, int n, float* Dout, float* ws, int max_sweeps, int max_grid,
                        cudaStream_t st) {
    return bj_launch(B, n, n, Dout, ws, max_sweeps, 1, 1e-20, 1, max_grid, st);
}

// Loads this file's kernels on the current device: asking for a kernel's
// attributes loads it, where a first launch would otherwise do so later.
cudaError_t preload_diag32_kernels() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, bjac32_coop_kernel<true>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, bjac32_coop_kernel<false>);
    return e;
}

// Sweeps made by the last diag_fp32 / refine_fp32 launches on workspace ws
// (host copy; synchronises the device).
cudaError_t fp32_sweeps_done(float* ws, int n, int* diag, int* refine) {
    int v[2] = {0, 0};
    cudaError_t e = cudaMemcpy(v, bj_ws(ws, n).slots, sizeof(v), cudaMemcpyDeviceToHost);
    if (diag) *diag = v[0];
    if (refine) *refine = v[1];
    return e;
}

}  // namespace pjac
