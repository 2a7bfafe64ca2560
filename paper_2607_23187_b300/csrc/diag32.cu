// Low-precision spectral decomposition of the preconditioner (Shao &
// Nakatsukasa, Sec. 2.1: A = V_l Lambda_l V_l^T + O(||A|| u_l), u_l = single
// precision as in Sec. 4).  The paper does not say which low-precision
// eigensolver to use; here it is a parallel-order two-sided Jacobi method in
// FP32 on fl32(A): each round rotates n/2 disjoint pairs at once, n-1 rounds
// (the round-robin tournament) make a sweep.
//
// Layout: the matrix is kept in "position order" so that the pairs of every
// round are the adjacent positions (2k, 2k+1).  Between rounds the tournament
// moves players by one seat, which is a permutation sigma with
// sigma(p) in {p-2, p+2} (and two fixed points); each round reads the
// previous buffer through sigma and writes the rotated result to the other
// buffer, so every access stays within a few elements of a straight stream.
// The column order of Q0 is irrelevant to the preconditioner.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>
#include "internal.h"

namespace cg = cooperative_groups;

namespace pjac {

// Sweeps made by the last diag32 (which = 0) and refine32 (which = 1) launch
// on a workspace: two ints at its end, outside every area the kernels use.
__host__ __device__ inline int* sweep_slot(float* ws, int n) {
    const long long npad = ((n + 31) / 32) * 32;
    return reinterpret_cast<int*>(ws + (4 * npad * npad + 6 * npad + 64) - 4);
}

// new position -> old position (m = npad/2 pairs)
__device__ __forceinline__ int tour_sigma(int p, int m) {
    if (p == 0) return 0;
    if (p == 2) return 1;
    if ((p & 1) == 0) return p - 2;
    if (p == 2 * m - 1) return 2 * m - 2;
    return p + 2;
}

__device__ __forceinline__ void rot32(float app, float aqq, float apq, float& c, float& s) {
    if (apq == 0.0f) { c = 1.0f; s = 0.0f; return; }
    // hypotf neither overflows nor underflows, so den >= 2|apq| > 0 even
    // when d == 0 and apq^2 is below the FP32 range (converged clusters)
    float d = app - aqq;
    float den = fabsf(d) + hypotf(d, 2.0f * apq);
    float t = 2.0f * fabsf(apq) / den;
    if (d != 0.0f && ((d < 0.0f) != (apq < 0.0f))) t = -t;
    c = rsqrtf(1.0f + t * t);
    s = t * c;
}

// Z = G_a^T X G_b (G = [[c,-s],[s,c]]) for one 2x2 block, written as
// Z[u][v] = (t(0,0) + t(1,1)) + (t(0,1) + t(1,0)) with
// t(r,w) = (G_a[r][u] * G_b[w][v]) * X[r][w].  The block (b,a) computes the
// transpose from the same products summed in the same pairs, so the FP32
// matrix stays exactly symmetric through every round.
__device__ __forceinline__ void rot2x2_sym(float ca, float sa, float cb, float sb, float x00, float x01,
                                           float x10, float x11, float& z00, float& z01, float& z10,
                                           float& z11) {
    // G[r][u]: G[0][0]=c, G[0][1]=-s, G[1][0]=s, G[1][1]=c
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

// One tile of one round.  Tiles [0, T*T) rotate the 32x32 tiles of A; tiles
// [T*T, 2*T*T) rotate the tiles of Q.  (T = npad/32.)  256 threads.
__device__ __forceinline__ void round_tile(int b, const float* __restrict__ A0, float* __restrict__ A1,
                                           const float* __restrict__ Q0, float* __restrict__ Q1, int npad,
                                           float (*cs_r)[2], float (*cs_c)[2]) {
    const int T = npad / 32;
    const int m = npad / 2;
    bool isA = b < T * T;
    if (!isA) b -= T * T;
    const int tr = b % T, tc = b / T;     // tile row (positions tr*32..), tile col
    const int tid = threadIdx.x;
    // each thread: one 2x2 block (row pair a, col pair bb) of the tile.  Its
    // entries do not depend on the rotations, so they are loaded first and
    // their latency overlaps the rotations' computation below.
    const int a = tid & 15, bb = tid >> 4;
    const int rp = tr * 32 + 2 * a, cp = tc * 32 + 2 * bb;
    const int c0 = tour_sigma(cp, m), c1 = tour_sigma(cp + 1, m);
    float x00, x10, x01, x11;
    if (isA) {
        const int r0 = tour_sigma(rp, m), r1 = tour_sigma(rp + 1, m);
        x00 = A0[r0 + (long long)c0 * npad];
        x10 = A0[r1 + (long long)c0 * npad];
        x01 = A0[r0 + (long long)c1 * npad];
        x11 = A0[r1 + (long long)c1 * npad];
    } else {
        // Q rows are plain (no permutation); columns follow the positions.
        // This thread's rows: tr*32 + a and tr*32 + a + 16.
        const int r = tr * 32 + a;
        x00 = Q0[r + (long long)c0 * npad];
        x01 = Q0[r + (long long)c1 * npad];
        x10 = Q0[r + 16 + (long long)c0 * npad];
        x11 = Q0[r + 16 + (long long)c1 * npad];
    }
    // rotation of the 16 pairs of this tile's columns (and rows, for A)
    if (tid < 32) {
        int which = tid >> 4, k = tid & 15;
        int pairpos = (which == 0 ? tc : tr) * 32 + 2 * k;   // positions (pairpos, pairpos+1)
        int sp = tour_sigma(pairpos, m), sq = tour_sigma(pairpos + 1, m);
        float app = A0[sp + (long long)sp * npad];
        float aqq = A0[sq + (long long)sq * npad];
        float apq = A0[sp + (long long)sq * npad];
        float c, s;
        rot32(app, aqq, apq, c, s);   // padding rows/cols are zero: identity
        if (which == 0) { cs_c[k][0] = c; cs_c[k][1] = s; }
        else { cs_r[k][0] = c; cs_r[k][1] = s; }
    }
    __syncthreads();
    const float cb = cs_c[bb][0], sb = cs_c[bb][1];
    if (isA) {
        const float ca = cs_r[a][0], sa = cs_r[a][1];
        float z00, z01, z10, z11;
        rot2x2_sym(ca, sa, cb, sb, x00, x01, x10, x11, z00, z01, z10, z11);
        if (rp == cp && sa != 0.0f) { z01 = 0.0f; z10 = 0.0f; }
        A1[rp + (long long)cp * npad] = z00;
        A1[rp + 1 + (long long)cp * npad] = z10;
        A1[rp + (long long)(cp + 1) * npad] = z01;
        A1[rp + 1 + (long long)(cp + 1) * npad] = z11;
    } else {
        const int r = tr * 32 + a;
        Q1[r + (long long)cp * npad] = x00 * cb + x01 * sb;
        Q1[r + (long long)(cp + 1) * npad] = -x00 * sb + x01 * cb;
        Q1[r + 16 + (long long)cp * npad] = x10 * cb + x11 * sb;
        Q1[r + 16 + (long long)(cp + 1) * npad] = -x10 * sb + x11 * cb;
    }
    __syncthreads();
}

// The whole diagonalisation in one cooperative launch: rounds separated by
// grid-wide barriers, the convergence test after every sweep decided by
// every CTA from the same global sums.  acc: 4 doubles, zero on entry.
__global__ void __launch_bounds__(256) diag32_coop_kernel(const double* __restrict__ A, long long lda, int n,
                                                          int npad, float* Ab0, float* Ab1, float* Qb0,
                                                          float* Qb1, float* Qout, double* acc,
                                                          int max_sweeps) {
    cg::grid_group grid = cg::this_grid();
    __shared__ float cs_r[16][2], cs_c[16][2];
    __shared__ double s_off[8], s_all[8];
    const long long nn = (long long)npad * npad;
    const long long gstride = (long long)gridDim.x * blockDim.x;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += gstride) {
        int r = (int)(e % npad), c = (int)(e / npad);
        Ab0[e] = (r < n && c < n) ? (float)A[r + (long long)c * lda] : 0.0f;
        Qb0[e] = (r == c) ? 1.0f : 0.0f;
    }
    grid.sync();
    float* Ab[2] = {Ab0, Ab1};
    float* Qb[2] = {Qb0, Qb1};
    const int T = npad / 32;
    const int ntiles = 2 * T * T;
    int cur = 0;
    double prev = -1.0;
    int done = max_sweeps;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        for (int r = 0; r < npad - 1; ++r) {
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x)
                round_tile(t, Ab[cur], Ab[cur ^ 1], Qb[cur], Qb[cur ^ 1], npad, cs_r, cs_c);
            cur ^= 1;
            grid.sync();
        }
        // off(A)^2 and ||A||^2 of the FP32 matrix, in slot (sweep & 1)
        double off = 0.0, all = 0.0;
        const float* Ac = Ab[cur];
        for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn; e += gstride) {
            int rr = (int)(e % npad), cc = (int)(e / npad);
            double v = (double)Ac[e];
            all += v * v;
            if (rr != cc) off += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            all += __shfl_xor_sync(0xffffffffu, all, o);
        }
        if ((threadIdx.x & 31) == 0) { s_off[threadIdx.x >> 5] = off; s_all[threadIdx.x >> 5] = all; }
        __syncthreads();
        double* slot = acc + 2 * (sweep & 1);
        if (threadIdx.x == 0) {
            double o2 = 0, a2 = 0;
            for (int w = 0; w < 8; ++w) { o2 += s_off[w]; a2 += s_all[w]; }
            atomicAdd(slot, o2);
            atomicAdd(slot + 1, a2);
        }
        grid.sync();
        double o2 = __ldcg(slot), a2 = __ldcg(slot + 1);
        bool stop = (a2 == 0.0 || o2 <= 1e-15 * a2) || (sweep >= 4 && prev >= 0.0 && o2 > 0.9 * prev);
        prev = o2;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            double* other = acc + 2 * ((sweep + 1) & 1);
            other[0] = 0.0;
            other[1] = 0.0;
        }
        if (stop) { done = sweep + 1; break; }
        grid.sync();   // the other slot is zero before anyone adds to it
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) sweep_slot(Ab0, n)[0] = done;
    // Q0 (n x n, ld n).  After whole sweeps (npad-1 rounds each) every
    // player is back at its own position, so the first n positions are the
    // real indices; padding indices are zero rows/columns that only ever
    // take identity rotations, so their columns of Q are unit vectors of
    // padding rows and are dropped.
    const float* Qc = Qb[cur];
    const long long tot = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot; e += gstride) {
        int r = (int)(e % n), c = (int)(e / n);
        Qout[e] = Qc[r + (long long)c * npad];
    }
}

// ---------------------------------------------------------------------------
// Refinement of the FP32 eigenbasis.  FP32 Jacobi on fl32(A) accumulates
// rounding over its many rotation layers and ends about sqrt(layers) * u_32
// from an eigenbasis of fl32(A).  Given X = fl64(Q0) and
// B = X^T fl64(fl32(A)) X (formed with FP64 products; nearly diagonal), a few
// more parallel-order Jacobi sweeps on B finish the decomposition of
// fl32(A): the off-diagonal part of B is kept in FP32 (its entries are
// small, so their rounding is small), the diagonal in FP64, and the
// accumulated rotation as E + D with E the permutation of the tournament
// seats and D small in FP32.  Output D (n x n): X (I + D) is an eigenbasis
// of fl32(A) to FP32 accuracy, the decomposition Sec. 2.1 asks for.
// ---------------------------------------------------------------------------
struct RefPair { float c, s, cm1, t, b; int pp, pq; };

__device__ __forceinline__ void refine_tile(int bt, const float* __restrict__ O0, float* __restrict__ O1,
                                            const float* __restrict__ D0, float* __restrict__ D1,
                                            const double* __restrict__ dg0, double* __restrict__ dg1,
                                            const int* __restrict__ pl0, int* __restrict__ pl1, int npad,
                                            RefPair* pr_r, RefPair* pr_c) {
    const int T = npad / 32;
    const int m = npad / 2;
    bool isO = bt < T * T;
    if (!isO) bt -= T * T;
    const int tr = bt % T, tc = bt / T;
    const int tid = threadIdx.x;
    // this thread's 2x2 block (row pair a, col pair bb), loaded before the
    // rotations are known (its entries do not depend on them)
    const int a = tid & 15, bb = tid >> 4;
    const int rp = tr * 32 + 2 * a, cp = tc * 32 + 2 * bb;
    const int c0 = tour_sigma(cp, m), c1 = tour_sigma(cp + 1, m);
    const int r0 = tour_sigma(rp, m), r1 = tour_sigma(rp + 1, m);
    float x00 = 0.0f, x10 = 0.0f, x01 = 0.0f, x11 = 0.0f;
    if (isO) {
        if (rp != cp) {
            x00 = O0[r0 + (long long)c0 * npad];
            x10 = O0[r1 + (long long)c0 * npad];
            x01 = O0[r0 + (long long)c1 * npad];
            x11 = O0[r1 + (long long)c1 * npad];
        }
    } else {
        const int r = tr * 32 + a;   // rows r and r + 16
        x00 = D0[r + (long long)c0 * npad];
        x01 = D0[r + (long long)c1 * npad];
        x10 = D0[r + 16 + (long long)c0 * npad];
        x11 = D0[r + 16 + (long long)c1 * npad];
    }
    if (tid < 32) {
        int which = tid >> 4, k = tid & 15;
        int pairpos = (which == 0 ? tc : tr) * 32 + 2 * k;
        int sp = tour_sigma(pairpos, m), sq = tour_sigma(pairpos + 1, m);
        float b = O0[sp + (long long)sq * npad];
        RefPair r;
        r.b = b;
        r.pp = pl0[sp];
        r.pq = pl0[sq];
        if (b == 0.0f) {
            r.c = 1.0f; r.s = 0.0f; r.cm1 = 0.0f; r.t = 0.0f;
        } else {
            double dd = dg0[sp] - dg0[sq];
            float d = (float)dd;
            float den = fabsf(d) + hypotf(d, 2.0f * b);
            float t = 2.0f * fabsf(b) / den;
            if (dd != 0.0 && ((dd < 0.0) != (b < 0.0f))) t = -t;
            float c = rsqrtf(1.0f + t * t);
            r.t = t;
            r.c = c;
            r.s = t * c;
            r.cm1 = -(t * t) * (c * c) / (1.0f + c);    // c - 1 without cancellation
        }
        if (which == 0) pr_c[k] = r;
        else pr_r[k] = r;
    }
    __syncthreads();
    const RefPair pc = pr_c[bb];
    if (isO) {
        const RefPair pa = pr_r[a];
        float z00, z01, z10, z11;
        if (rp == cp) {
            // diagonal block: its rotation moves b into the FP64 diagonal
            z00 = z01 = z10 = z11 = 0.0f;
            if (a == bb) {
                double tb = (double)pa.t * (double)pa.b;
                dg1[rp] = dg0[r0] + tb;
                dg1[rp + 1] = dg0[r1] - tb;
                pl1[rp] = pl0[r0];
                pl1[rp + 1] = pl0[r1];
            }
        } else {
            rot2x2_sym(pa.c, pa.s, pc.c, pc.s, x00, x01, x10, x11, z00, z01, z10, z11);
        }
        O1[rp + (long long)cp * npad] = z00;
        O1[rp + 1 + (long long)cp * npad] = z10;
        O1[rp + (long long)(cp + 1) * npad] = z01;
        O1[rp + 1 + (long long)(cp + 1) * npad] = z11;
    } else {
        for (int h = 0; h < 2; ++h) {
            const int r = tr * 32 + a + 16 * h;
            const float q0 = h ? x10 : x00, q1 = h ? x11 : x01;
            float v0 = q0 * pc.c + q1 * pc.s;
            float v1 = -q0 * pc.s + q1 * pc.c;
            if (r == pc.pp) { v0 += pc.cm1; v1 -= pc.s; }
            if (r == pc.pq) { v0 += pc.s; v1 += pc.cm1; }
            D1[r + (long long)cp * npad] = v0;
            D1[r + (long long)(cp + 1) * npad] = v1;
        }
    }
    __syncthreads();
}

// ws layout (floats): O[2][npad^2], D[2][npad^2], then dg[2][npad] doubles,
// pl[2][npad] ints, acc[4] doubles.
__global__ void __launch_bounds__(256) refine32_coop_kernel(const double* __restrict__ B, int n, int npad,
                                                            float* ws, float* Dout, int max_sweeps) {
    cg::grid_group grid = cg::this_grid();
    __shared__ RefPair pr_r[16], pr_c[16];
    __shared__ double s_off[8], s_all[8];
    const long long nn = (long long)npad * npad;
    float* Ob[2] = {ws, ws + nn};
    float* Db[2] = {ws + 2 * nn, ws + 3 * nn};
    double* dgb0 = reinterpret_cast<double*>(ws + 4 * nn);
    double* dgb[2] = {dgb0, dgb0 + npad};
    int* plb0 = reinterpret_cast<int*>(dgb0 + 2 * npad);
    int* plb[2] = {plb0, plb0 + npad};
    double* acc = reinterpret_cast<double*>(plb0 + 2 * npad + 2);   // 8-byte aligned (npad even)
    const long long gstride = (long long)gridDim.x * blockDim.x;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long e = gtid; e < nn; e += gstride) {
        int r = (int)(e % npad), c = (int)(e / npad);
        Ob[0][e] = (r != c && r < n && c < n) ? (float)B[r + (long long)c * n] : 0.0f;
        Db[0][e] = 0.0f;
    }
    for (long long e = gtid; e < npad; e += gstride) {
        int p = (int)e;
        dgb[0][p] = (p < n) ? B[p + (long long)p * n] : 0.0;
        plb[0][p] = p;
    }
    if (gtid < 4) acc[gtid] = 0.0;
    grid.sync();
    const int T = npad / 32;
    const int ntiles = 2 * T * T;
    int cur = 0;
    double prev = -1.0;
    int done = max_sweeps;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        for (int r = 0; r < npad - 1; ++r) {
            for (int t = blockIdx.x; t < ntiles; t += gridDim.x)
                refine_tile(t, Ob[cur], Ob[cur ^ 1], Db[cur], Db[cur ^ 1], dgb[cur], dgb[cur ^ 1], plb[cur],
                            plb[cur ^ 1], npad, pr_r, pr_c);
            cur ^= 1;
            grid.sync();
        }
        double off = 0.0, all = 0.0;
        for (long long e = gtid; e < nn; e += gstride) {
            double v = (double)Ob[cur][e];
            off += v * v;
        }
        for (long long e = gtid; e < npad; e += gstride) {
            double v = dgb[cur][e];
            all += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            all += __shfl_xor_sync(0xffffffffu, all, o);
        }
        if ((threadIdx.x & 31) == 0) { s_off[threadIdx.x >> 5] = off; s_all[threadIdx.x >> 5] = all; }
        __syncthreads();
        double* slot = acc + 2 * (sweep & 1);
        if (threadIdx.x == 0) {
            double o2 = 0, a2 = 0;
            for (int w = 0; w < 8; ++w) { o2 += s_off[w]; a2 += s_all[w]; }
            atomicAdd(slot, o2);
            atomicAdd(slot + 1, a2);
        }
        grid.sync();
        double o2 = __ldcg(slot), a2 = __ldcg(slot + 1);
        // converged well past FP32 accuracy, or no longer improving.  The
        // first sweeps of a poor start only shrink off(B) by a factor 2-3
        // (linear phase until off(B) is below the cluster gaps), so the
        // stagnation test waits for the quadratic phase.
        bool stop = (a2 == 0.0 || o2 <= 1e-20 * a2) || (sweep >= 4 && prev >= 0.0 && o2 > 0.9 * prev);
        prev = o2;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            double* other = acc + 2 * ((sweep + 1) & 1);
            other[0] = 0.0;
            other[1] = 0.0;
        }
        if (stop) { done = sweep + 1; break; }
        grid.sync();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) sweep_slot(ws, n)[1] = done;
    // whole sweeps bring every player back to its own seat: D is in the
    // original column order
    const float* Dc = Db[cur];
    const long long tot = (long long)n * n;
    for (long long e = gtid; e < tot; e += gstride) {
        int r = (int)(e % n), c = (int)(e / n);
        Dout[e] = Dc[r + (long long)c * npad];
    }
}

cudaError_t refine_fp32(const double* B, int n, float* Dout, float* ws, int max_sweeps, int max_grid,
                        cudaStream_t st) {
    int npad = ((n + 31) / 32) * 32;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, refine32_coop_kernel, 256, 0);
    if (e != cudaSuccess) return e;
    int T = npad / 32;
    int grid = std::min(sms * std::max(1, std::min(per_sm, 4)), 2 * T * T);
    if (max_grid > 0 && grid > max_grid) grid = max_grid;   // share the GPU (all CTAs must be co-resident)
    void* args[] = {(void*)&B, (void*)&n, (void*)&npad, (void*)&ws, (void*)&Dout, (void*)&max_sweeps};
    return cudaLaunchCooperativeKernel((const void*)refine32_coop_kernel, dim3(grid), dim3(256), args, 0, st);
}

size_t diag_fp32_ws_floats(int n) {
    long long npad = ((n + 31) / 32) * 32;
    // refine32 also needs 2 npad doubles + 2 npad ints + 4 doubles
    return (size_t)(4 * npad * npad + 6 * npad + 64);
}

// Q0 <- eigenvectors of fl32(A) (approximately).  ws: diag_fp32_ws_floats(n)
// floats.  One cooperative launch; nothing waits on the host.
cudaError_t diag_fp32(const double* A, long long lda, int n, float* Q0, float* ws, int* iws,
                      int max_sweeps, int max_grid, cudaStream_t st) {
    (void)iws;
    int npad = ((n + 31) / 32) * 32;
    long long nn = (long long)npad * npad;
    float* Ab0 = ws;
    float* Ab1 = ws + nn;
    float* Qb0 = ws + 2 * nn;
    float* Qb1 = ws + 3 * nn;
    double* acc = reinterpret_cast<double*>(ws + 4 * nn);   // 8-byte aligned: nn is even
    cudaError_t e = cudaMemsetAsync(acc, 0, 4 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, diag32_coop_kernel, 256, 0);
    if (e != cudaSuccess) return e;
    int T = npad / 32;
    int grid = std::min(sms * std::max(1, std::min(per_sm, 4)), 2 * T * T);
    if (max_grid > 0 && grid > max_grid) grid = max_grid;   // share the GPU (all CTAs must be co-resident)
    void* args[] = {(void*)&A, (void*)&lda, (void*)&n, (void*)&npad, (void*)&Ab0, (void*)&Ab1, (void*)&Qb0,
                    (void*)&Qb1, (void*)&Q0, (void*)&acc, (void*)&max_sweeps};
    return cudaLaunchCooperativeKernel((const void*)diag32_coop_kernel, dim3(grid), dim3(256), args, 0, st);
}

// Loads this file's kernels on the current device: asking for a kernel's
// attributes loads it, where a first launch would otherwise do so later.
cudaError_t preload_diag32_kernels() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, diag32_coop_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, refine32_coop_kernel);
    return e;
}

}  // namespace pjac

namespace pjac {
// Sweeps made by the last diag32 / refine32 launches on workspace ws (host
// copy; synchronises the device).
cudaError_t fp32_sweeps_done(float* ws, int n, int* diag, int* refine) {
    int v[2] = {0, 0};
    cudaError_t e = cudaMemcpy(v, sweep_slot(ws, n), sizeof(v), cudaMemcpyDeviceToHost);
    if (diag) *diag = v[0];
    if (refine) *refine = v[1];
    return e;
}
}  // namespace pjac
