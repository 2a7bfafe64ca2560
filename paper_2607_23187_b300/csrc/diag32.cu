// Low-precision spectral decomposition of the preconditioner (Shao &
// Nakatsukasa, Sec. 2.1: A = V_l Lambda_l V_l^T + O(||A|| u_l), u_l = single
// precision as in Sec. 4).  The paper does not say which low-precision
// eigensolver to use; here it is a blocked parallel-order two-sided Jacobi
// method in FP32.
//
// The order-npad matrix (npad = n rounded up to 64; the padding rows and
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
// Storage: the off-diagonal part in FP32 (kept exactly symmetric: each
// off-diagonal super-block is computed once and written with its
// transpose), the diagonal in FP64 (so rotations inside clusters narrower
// than FP32 resolution still see their true differences).  Two uses:
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
constexpr size_t BJ_SMEM = 4 * BJ_TILE * sizeof(float);   // phase 2: four operand tiles

__host__ __device__ inline long long bj_npad(int n) { return ((long long)(n + 63) / 64) * 64; }

// workspace (floats): O[npad^2] | X[npad^2] | dg[npad] doubles | E[npairs][64*64] | acc[4] doubles | slots
struct BjWs {
    float* O;
    float* X;
    double* dg;
    float* E;
    double* acc;
    int* slots;
};

__host__ __device__ inline BjWs bj_ws(float* ws, int n) {
    const long long npad = bj_npad(n), nn = npad * npad, npairs = npad / 64;
    BjWs w;
    w.O = ws;
    w.X = ws + nn;
    w.dg = reinterpret_cast<double*>(ws + 2 * nn);
    w.E = ws + 2 * nn + 2 * npad;
    w.acc = reinterpret_cast<double*>(w.E + npairs * 4096);
    w.slots = reinterpret_cast<int*>(w.acc + 4);
    return w;
}

// Round-robin tournament (circle method) on N players, N even: in round r
// pair 0 is (N-1, r) and pair k >= 1 is ((r+k) mod (N-1), (r-k) mod (N-1)).
__device__ __forceinline__ void circle_pair(int r, int k, int N, int& p, int& q) {
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
// t(r,w) = (G_a[r][u] * G_b[w][v]) * X[r][w].  The block (b,a) is the
// transpose formed from the same products summed in the same pairs, so a
// matrix stays exactly symmetric through every rotation.
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
__device__ void bj_inner(int k, int round, int nblk, long long npad, float* __restrict__ O,
                         double* __restrict__ dg, float* __restrict__ Eg, int inner_sweeps, float* sm,
                         const unsigned short* __restrict__ tri) {
    float* Ss = sm;                      // off-diagonal part, 64 x 65 (row u, col v)
    float* Es = Ss + 64 * BJ_ZLD;        // E = G - I, 64 x 65
    double* dS = reinterpret_cast<double*>(Es + 64 * BJ_ZLD);   // FP64 diagonal
    float* pc = reinterpret_cast<float*>(dS + 64);              // c[32] s[32] (c-1)[32]
    int* pix = reinterpret_cast<int*>(pc + 96);                 // p[32] q[32]
    const int tid = threadIdx.x;
    int bi, bj;
    circle_pair(round, k, nblk, bi, bj);
    for (int e = tid; e < 4096; e += BJ_NT) {
        const int u = e & 63, v = e >> 6;
        Ss[u * BJ_ZLD + v] = O[sup_idx(u, bi, bj) + sup_idx(v, bi, bj) * npad];
        Es[u * BJ_ZLD + v] = 0.0f;
    }
    if (tid < 64) dS[tid] = dg[sup_idx(tid, bi, bj)];
    __syncthreads();
    for (int isw = 0; isw < inner_sweeps; ++isw) {
        for (int ir = 0; ir < 63; ++ir) {
            if (tid < 32) {
                int p, q;
                circle_pair(ir, tid, 64, p, q);
                const float b = Ss[p * BJ_ZLD + q];
                float c = 1.0f, s = 0.0f, cm1 = 0.0f;
                if (b != 0.0f) {
                    const double dd = dS[p] - dS[q];
                    const float d = (float)dd;
                    // hypotf neither overflows nor underflows: den >= 2|b| > 0
                    const float den = fabsf(d) + hypotf(d, 2.0f * b);
                    float t = 2.0f * fabsf(b) / den;
                    if (dd != 0.0 && ((dd < 0.0) != (b < 0.0f))) t = -t;
                    c = rsqrtf(1.0f + t * t);
                    s = t * c;
                    cm1 = -(t * t) * (c * c) / (1.0f + c);   // c - 1 without cancellation
                    const double tb = (double)t * (double)b;
                    dS[p] += tb;
                    dS[q] -= tb;
                    Ss[p * BJ_ZLD + q] = 0.0f;
                    Ss[q * BJ_ZLD + p] = 0.0f;
                }
                pc[tid] = c;
                pc[32 + tid] = s;
                pc[64 + tid] = cm1;
                pix[tid] = p;
                pix[32 + tid] = q;
            }
            __syncthreads();
            // off-diagonal 2x2 blocks (pair u rows, pair v columns), u < v,
            // written with their transposes
            for (int w = tid; w < 496; w += BJ_NT) {
                const int uv = tri[w];
                const int u = uv & 255, v = uv >> 8;
                const int pu = pix[u], qu = pix[32 + u], pv = pix[v], qv = pix[32 + v];
                float z00, z01, z10, z11;
                rot2x2_sym(pc[u], pc[32 + u], pc[v], pc[32 + v], Ss[pu * BJ_ZLD + pv], Ss[pu * BJ_ZLD + qv],
                           Ss[qu * BJ_ZLD + pv], Ss[qu * BJ_ZLD + qv], z00, z01, z10, z11);
                Ss[pu * BJ_ZLD + pv] = z00;
                Ss[pu * BJ_ZLD + qv] = z01;
                Ss[qu * BJ_ZLD + pv] = z10;
                Ss[qu * BJ_ZLD + qv] = z11;
                Ss[pv * BJ_ZLD + pu] = z00;
                Ss[qv * BJ_ZLD + pu] = z01;
                Ss[pv * BJ_ZLD + qu] = z10;
                Ss[qv * BJ_ZLD + qu] = z11;
            }
            // E <- E J + (J - I) on columns p, q of every row
            for (int w = tid; w < 2048; w += BJ_NT) {
                const int i = w & 63, kk = w >> 6;
                const int p = pix[kk], q = pix[32 + kk];
                const float c = pc[kk], s = pc[32 + kk], cm1 = pc[64 + kk];
                const float e0 = Es[i * BJ_ZLD + p], e1 = Es[i * BJ_ZLD + q];
                float v0 = e0 * c + e1 * s;
                float v1 = -e0 * s + e1 * c;
                if (i == p) { v0 += cm1; v1 -= s; }
                if (i == q) { v0 += s; v1 += cm1; }
                Es[i * BJ_ZLD + p] = v0;
                Es[i * BJ_ZLD + q] = v1;
            }
            __syncthreads();
        }
    }
    for (int e = tid; e < 4096; e += BJ_NT) {
        const int u = e & 63, v = e >> 6;
        O[sup_idx(u, bi, bj) + sup_idx(v, bi, bj) * npad] = Ss[u * BJ_ZLD + v];
        const int r = e >> 6, cc = e & 63;   // E row-major, contiguous in cc
        Eg[(long long)k * 4096 + r * 64 + cc] = Es[r * BJ_ZLD + cc];
    }
    if (tid < 64) dg[sup_idx(tid, bi, bj)] = dS[tid];
    __syncthreads();
}

// ---------------------------------------------------------------------------
// phase 2: dense 64 x 64 x 64 products in FP32
// ---------------------------------------------------------------------------
// acc[a][b] += sum_k L[k][4ty+a] R[k][4tx+b]; L and R k-major with row
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

// dst[k*BJ_LD + j] = E[k][j] + (k == j): G = I + E, row-major
__device__ __forceinline__ void load_g(const float* __restrict__ E, float* dst) {
    for (int f = threadIdx.x; f < 1024; f += BJ_NT) {
        const int k = f >> 4, j4 = (f & 15) * 4;
        float4 v = *reinterpret_cast<const float4*>(E + k * 64 + j4);
        if (k >= j4 && k < j4 + 4) {
            if (k == j4) v.x += 1.0f;
            else if (k == j4 + 1) v.y += 1.0f;
            else if (k == j4 + 2) v.z += 1.0f;
            else v.w += 1.0f;
        }
        *reinterpret_cast<float4*>(dst + k * BJ_LD + j4) = v;
    }
}

// dst[v*BJ_LD + u] = M[row(u) + col(v)*npad]: a 64 x 64 tile, column-major;
// rows are two runs of 32 (r0, r1) or one run of 64 (r1 = r0 + 32)
__device__ __forceinline__ void load_tile(const float* __restrict__ M, long long npad, int r0, int r1, int c0,
                                          int c1, float* dst) {
    for (int f = threadIdx.x; f < 1024; f += BJ_NT) {
        const int v = f >> 4, u4 = (f & 15) * 4;
        const int gr = u4 < 32 ? r0 + u4 : r1 + u4 - 32;
        const int gc = v < 32 ? c0 + v : c1 + v - 32;
        *reinterpret_cast<float4*>(dst + v * BJ_LD + u4) =
            *reinterpret_cast<const float4*>(M + gr + (long long)gc * npad);
    }
}

__device__ __forceinline__ void store_acc(float acc[4][4], float* dst, int ld) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) dst[(4 * ty + a) * ld + 4 * tx + b] = acc[a][b];
}

__device__ __forceinline__ void store_acc4(float acc[4][4], float* dst) {
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
    for (int a = 0; a < 4; ++a)
        *reinterpret_cast<float4*>(dst + (4 * ty + a) * BJ_LD + 4 * tx) =
            make_float4(acc[a][0], acc[a][1], acc[a][2], acc[a][3]);
}

// off-diagonal super-block (kp, kq), kp < kq: S_PQ <- G_P^T S_PQ G_Q, and
// its transpose into S_QP
__device__ void bj_apply_off(int kp, int kq, int round, int nblk, long long npad, float* __restrict__ O,
                             const float* __restrict__ Eg, float* sm) {
    float* Lb = sm;                  // S_PQ (k-major), later Z (stride 65)
    float* Rb = sm + BJ_TILE;        // G_Q
    float* Tb = sm + 2 * BJ_TILE;    // T = S_PQ G_Q, row-major
    float* Gb = sm + 3 * BJ_TILE;    // G_P
    int pi, pj, qi, qj;
    circle_pair(round, kp, nblk, pi, pj);
    circle_pair(round, kq, nblk, qi, qj);
    load_tile(O, npad, pi * 32, pj * 32, qi * 32, qj * 32, Lb);
    load_g(Eg + (long long)kq * 4096, Rb);
    load_g(Eg + (long long)kp * 4096, Gb);
    __syncthreads();
    float acc[4][4];
    mm64(Lb, Rb, acc);               // T[i][j] = sum_k S[i][k] G_Q[k][j]
    store_acc4(acc, Tb);
    __syncthreads();
    mm64(Gb, Tb, acc);               // Z[i][j] = sum_k G_P[k][i] T[k][j]
    store_acc(acc, Lb, BJ_ZLD);
    __syncthreads();
    for (int e = threadIdx.x; e < 4096; e += BJ_NT) {
        const int i = e & 63, j = e >> 6;
        O[sup_idx(i, pi, pj) + sup_idx(j, qi, qj) * npad] = Lb[i * BJ_ZLD + j];
        const int i2 = e >> 6, j2 = e & 63;
        O[sup_idx(j2, qi, qj) + sup_idx(i2, pi, pj) * npad] = Lb[i2 * BJ_ZLD + j2];
    }
    __syncthreads();
}

// basis rows [64 rt, 64 rt + 64) on the columns of pair k: X <- X G_k, plus
// E_k on the pair's own rows when the basis is carried as D = X - I
__device__ void bj_apply_basis(int rt, int k, int round, int nblk, long long npad, float* __restrict__ X,
                               const float* __restrict__ Eg, int delta, float* sm) {
    float* Lb = sm;
    float* Rb = sm + BJ_TILE;
    float* Zb = sm + 2 * BJ_TILE;    // stride 65
    int bi, bj;
    circle_pair(round, k, nblk, bi, bj);
    const int r0 = rt * 64;
    load_tile(X, npad, r0, r0 + 32, bi * 32, bj * 32, Lb);
    const float* Ek = Eg + (long long)k * 4096;
    load_g(Ek, Rb);
    __syncthreads();
    float acc[4][4];
    mm64(Lb, Rb, acc);
    store_acc(acc, Zb, BJ_ZLD);
    __syncthreads();
    for (int e = threadIdx.x; e < 4096; e += BJ_NT) {
        const int i = e & 63, j = e >> 6;
        const int g = r0 + i;
        float z = Zb[i * BJ_ZLD + j];
        if (delta) {
            const int blk = g >> 5;
            if (blk == bi) z += Ek[(g - bi * 32) * 64 + j];
            else if (blk == bj) z += Ek[(32 + g - bj * 32) * 64 + j];
        }
        X[g + (long long)sup_idx(j, bi, bj) * npad] = z;
    }
    __syncthreads();
}

// The whole iteration in one cooperative launch; the phases and rounds are
// separated by grid-wide barriers and the convergence test after each sweep
// is taken by every CTA from the same global sums.
//   delta = 0: S = fl32(A) (its diagonal too), basis X = I;  out = X
//   delta = 1: S = B with the FP64 diagonal, D = 0;           out = D
__global__ void __launch_bounds__(BJ_NT) bjac32_coop_kernel(const double* __restrict__ A, long long lda, int n,
                                                            float* ws, float* __restrict__ out, int max_sweeps,
                                                            int inner_sweeps, int delta, double stop_tol,
                                                            int slot) {
    cg::grid_group grid = cg::this_grid();
    extern __shared__ __align__(16) float sm[];
    __shared__ unsigned short tri[496];
    __shared__ double s_off[BJ_NT / 32], s_all[BJ_NT / 32];
    const long long npad = bj_npad(n), nn = npad * npad;
    const BjWs w = bj_ws(ws, n);
    const int nblk = (int)(npad / 32), npairs = nblk / 2;
    const long long gstride = (long long)gridDim.x * blockDim.x;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (int t = threadIdx.x; t < 496; t += BJ_NT) {
        int u = 0, rem = t;
        while (rem >= 31 - u) { rem -= 31 - u; ++u; }
        tri[t] = (unsigned short)(u | ((u + 1 + rem) << 8));
    }
    for (long long e = gtid; e < nn; e += gstride) {
        const int r = (int)(e % npad), c = (int)(e / npad);
        w.O[e] = (r != c && r < n && c < n) ? (float)A[r + (long long)c * lda] : 0.0f;
        w.X[e] = (!delta && r == c) ? 1.0f : 0.0f;
    }
    for (long long p = gtid; p < npad; p += gstride) {
        double d = 0.0;
        if (p < n) {
            d = A[p + p * lda];
            if (!delta) d = (double)(float)d;
        }
        w.dg[p] = d;
    }
    if (gtid < 4) w.acc[gtid] = 0.0;
    grid.sync();
    const int nA = npairs * (npairs - 1) / 2;
    const int nunits = nA + (int)(npad / 64) * npairs;
    double prev = -1.0;
    int done = max_sweeps;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        for (int r = 0; r < nblk - 1; ++r) {
            for (int k = blockIdx.x; k < npairs; k += gridDim.x)
                bj_inner(k, r, nblk, npad, w.O, w.dg, w.E, inner_sweeps, sm, tri);
            grid.sync();
            for (int u = blockIdx.x; u < nunits; u += gridDim.x) {
                if (u < nA) {
                    int kp = 0, rem = u;
                    while (rem >= npairs - 1 - kp) { rem -= npairs - 1 - kp; ++kp; }
                    bj_apply_off(kp, kp + 1 + rem, r, nblk, npad, w.O, w.E, sm);
                } else {
                    const int v = u - nA;
                    bj_apply_basis(v / npairs, v % npairs, r, nblk, npad, w.X, w.E, delta, sm);
                }
            }
            grid.sync();
        }
        // off(S)^2 and ||S||_F^2
        double off = 0.0, all = 0.0;
        for (long long e = gtid; e < nn; e += gstride) {
            const double v = (double)w.O[e];
            off += v * v;
        }
        for (long long p = gtid; p < npad; p += gstride) all += w.dg[p] * w.dg[p];
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
    if (blockIdx.x == 0 && threadIdx.x == 0) w.slots[slot] = done;
    // indices never move, so the basis is in the original column order;
    // the padding columns are unit vectors of padding rows and are dropped
    const long long tot = (long long)n * n;
    for (long long e = gtid; e < tot; e += gstride) {
        const int r = (int)(e % n), c = (int)(e / n);
        out[e] = w.X[r + (long long)c * npad];
    }
}

int bj_inner_sweeps() { return 1; }

cudaError_t bj_launch(const double* A, long long lda, int n, float* out, float* ws, int max_sweeps, int delta,
                      double stop_tol, int slot, int max_grid, cudaStream_t st) {
    cudaError_t e =
        cudaFuncSetAttribute(bjac32_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BJ_SMEM);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bjac32_coop_kernel, BJ_NT, BJ_SMEM);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    const long long npad = bj_npad(n);
    const long long npairs = npad / 64;
    const long long units = npairs * (npairs - 1) / 2 + (npad / 64) * npairs;
    int grid = (int)std::min<long long>((long long)sms * std::min(per_sm, 3), std::max<long long>(units, 1));
    if (max_grid > 0 && grid > max_grid) grid = max_grid;   // share the GPU (all CTAs must be co-resident)
    int inner = bj_inner_sweeps();
    void* args[] = {(void*)&A,      (void*)&lda,   (void*)&n,        (void*)&ws,   (void*)&out,
                    (void*)&max_sweeps, (void*)&inner, (void*)&delta, (void*)&stop_tol, (void*)&slot};
    return cudaLaunchCooperativeKernel((const void*)bjac32_coop_kernel, dim3(grid), dim3(BJ_NT), args, BJ_SMEM,
                                       st);
}

}  // namespace

size_t diag_fp32_ws_floats(int n) {
    const long long npad = bj_npad(n), npairs = npad / 64;
    return (size_t)(2 * npad * npad + 2 * npad + npairs * 4096 + 8 + 16);
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
    return cudaFuncGetAttributes(&fa, bjac32_coop_kernel);
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
