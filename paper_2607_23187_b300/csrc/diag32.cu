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
    // each thread: one 2x2 block (row pair a, col pair bb) of the tile
    const int a = tid & 15, bb = tid >> 4;
    const int rp = tr * 32 + 2 * a, cp = tc * 32 + 2 * bb;
    const float cb = cs_c[bb][0], sb = cs_c[bb][1];
    if (isA) {
        const float ca = cs_r[a][0], sa = cs_r[a][1];
        int r0 = tour_sigma(rp, m), r1 = tour_sigma(rp + 1, m);
        int c0 = tour_sigma(cp, m), c1 = tour_sigma(cp + 1, m);
        float x00 = A0[r0 + (long long)c0 * npad], x10 = A0[r1 + (long long)c0 * npad];
        float x01 = A0[r0 + (long long)c1 * npad], x11 = A0[r1 + (long long)c1 * npad];
        float z00, z01, z10, z11;
        rot2x2_sym(ca, sa, cb, sb, x00, x01, x10, x11, z00, z01, z10, z11);
        if (rp == cp && sa != 0.0f) { z01 = 0.0f; z10 = 0.0f; }
        A1[rp + (long long)cp * npad] = z00;
        A1[rp + 1 + (long long)cp * npad] = z10;
        A1[rp + (long long)(cp + 1) * npad] = z01;
        A1[rp + 1 + (long long)(cp + 1) * npad] = z11;
    } else {
        // Q rows are plain (no permutation); columns follow the positions
        int c0 = tour_sigma(cp, m), c1 = tour_sigma(cp + 1, m);
        for (int r = tr * 32 + a; r < tr * 32 + 32; r += 16) {
            float q0 = Q0[r + (long long)c0 * npad], q1 = Q0[r + (long long)c1 * npad];
            Q1[r + (long long)cp * npad] = q0 * cb + q1 * sb;
            Q1[r + (long long)(cp + 1) * npad] = -q0 * sb + q1 * cb;
        }
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
        if (stop) break;
        grid.sync();   // the other slot is zero before anyone adds to it
    }
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

size_t diag_fp32_ws_floats(int n) {
    long long npad = ((n + 31) / 32) * 32;
    return (size_t)(4 * npad * npad + 64);
}

// Q0 <- eigenvectors of fl32(A) (approximately).  ws: diag_fp32_ws_floats(n)
// floats.  One cooperative launch; nothing waits on the host.
cudaError_t diag_fp32(const double* A, long long lda, int n, float* Q0, float* ws, int* iws,
                      int max_sweeps, cudaStream_t st) {
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
    void* args[] = {(void*)&A, (void*)&lda, (void*)&n, (void*)&npad, (void*)&Ab0, (void*)&Ab1, (void*)&Qb0,
                    (void*)&Qb1, (void*)&Q0, (void*)&acc, (void*)&max_sweeps};
    return cudaLaunchCooperativeKernel((const void*)diag32_coop_kernel, dim3(grid), dim3(256), args, 0, st);
}

}  // namespace pjac
