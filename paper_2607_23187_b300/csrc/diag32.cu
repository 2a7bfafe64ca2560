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
#include <cuda_runtime.h>
#include <cstdint>
#include "internal.h"

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
    float d = app - aqq;
    float den = fabsf(d) + sqrtf(d * d + 4.0f * apq * apq);
    float t = 2.0f * fabsf(apq) / den;
    if (d != 0.0f && ((d < 0.0f) != (apq < 0.0f))) t = -t;
    c = rsqrtf(1.0f + t * t);
    s = t * c;
}

// One round.  Blocks [0, T*T) rotate the 32x32 tiles of A; blocks
// [T*T, 2*T*T) rotate the tiles of Q.  (T = npad/32.)
__global__ void __launch_bounds__(256) round_kernel(const float* __restrict__ A0, float* __restrict__ A1,
                                                    const float* __restrict__ Q0, float* __restrict__ Q1,
                                                    int npad, int n, const int* __restrict__ done) {
    __shared__ float cs_r[16][2], cs_c[16][2];
    if (*done) return;
    const int T = npad / 32;
    const int m = npad / 2;
    int b = blockIdx.x;
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
        // Y = G_a^T X G_b with G = [[c,-s],[s,c]]
        float y00 = ca * x00 + sa * x10, y10 = -sa * x00 + ca * x10;
        float y01 = ca * x01 + sa * x11, y11 = -sa * x01 + ca * x11;
        float z00 = y00 * cb + y01 * sb, z01 = -y00 * sb + y01 * cb;
        float z10 = y10 * cb + y11 * sb, z11 = -y10 * sb + y11 * cb;
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
}

__global__ void init32_kernel(const double* A, long long lda, int n, int npad, float* A32, float* Q32) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)npad * npad;
    for (; e < tot; e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e % npad), c = (int)(e / npad);
        A32[e] = (r < n && c < n) ? (float)A[r + (long long)c * lda] : 0.0f;
        Q32[e] = (r == c) ? 1.0f : 0.0f;
    }
}

// Convergence test after a sweep (device side, no host round trip).
// st: [0] done flag, [1] index of the buffer holding the result, [2] sweeps;
// acc: off^2, ||A||^2 of this sweep, then the previous sweep's off^2.
__global__ void conv32_kernel(double* acc, int* st, int cur) {
    if (st[0]) return;
    double o2 = acc[0], a2 = acc[1], prev = acc[2];
    int sweep = st[2];
    st[1] = cur;
    st[2] = sweep + 1;
    bool stop = (a2 == 0.0 || o2 <= 1e-13 * a2) || (sweep >= 3 && prev >= 0.0 && o2 > 0.25 * prev);
    acc[2] = o2;
    acc[0] = 0.0;
    acc[1] = 0.0;
    if (stop) st[0] = 1;
}

__global__ void conv32_init_kernel(double* acc, int* st) {
    acc[0] = 0.0; acc[1] = 0.0; acc[2] = -1.0;
    st[0] = 0; st[1] = 0; st[2] = 0;
}

__global__ void extract_q_kernel(const float* QA, const float* QB, const int* st, int npad, int n, float* Q0) {
    const float* Q32 = st[1] ? QB : QA;
    // Q0 (n x n, ld n).  After whole sweeps (npad-1 rounds each) every
    // player is back at its own position, so the first n positions are the
    // real indices; padding indices are zero rows/columns that only ever
    // take identity rotations, so their columns of Q are unit vectors of
    // padding rows and are dropped.
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)n * n;
    for (; e < tot; e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e % n), c = (int)(e / n);
        Q0[e] = Q32[r + (long long)c * npad];
    }
}

size_t diag_fp32_ws_floats(int n) {
    long long npad = ((n + 31) / 32) * 32;
    return (size_t)(4 * npad * npad + 64);
}


// off^2 / ||A||^2 of the current buffer, skipped once converged.
__global__ void off32_gated_kernel(const float* A, int npad, double* acc, const int* done) {
    if (*done) return;
    __shared__ double s_off[8], s_all[8];
    double off = 0.0, all = 0.0;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)npad * npad;
    for (; e < tot; e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e % npad), c = (int)(e / npad);
        double v = (double)A[e];
        all += v * v;
        if (r != c) off += v * v;
    }
    for (int o = 16; o > 0; o >>= 1) {
        off += __shfl_xor_sync(0xffffffffu, off, o);
        all += __shfl_xor_sync(0xffffffffu, all, o);
    }
    if ((threadIdx.x & 31) == 0) { s_off[threadIdx.x >> 5] = off; s_all[threadIdx.x >> 5] = all; }
    __syncthreads();
    if (threadIdx.x == 0) {
        double a = 0, b = 0;
        for (int w = 0; w < 8; ++w) { a += s_off[w]; b += s_all[w]; }
        atomicAdd(acc, a);
        atomicAdd(acc + 1, b);
    }
}

// Q0 <- eigenvectors of fl32(A) (approximately).  ws: diag_fp32_ws_floats(n)
// floats.  Entirely asynchronous: after every sweep a device-side test sets
// a flag that turns the remaining launches into no-ops.
cudaError_t diag_fp32(const double* A, long long lda, int n, float* Q0, float* ws, int* iws,
                      int max_sweeps, cudaStream_t st) {
    (void)iws;
    int npad = ((n + 31) / 32) * 32;
    long long nn = (long long)npad * npad;
    float* Ab[2] = {ws, ws + nn};
    float* Qb[2] = {ws + 2 * nn, ws + 3 * nn};
    double* acc = reinterpret_cast<double*>(ws + 4 * nn);   // 3 doubles (8-byte aligned: nn even)
    int* flags = reinterpret_cast<int*>(acc + 4);           // 3 ints
    init32_kernel<<<592, 256, 0, st>>>(A, lda, n, npad, Ab[0], Qb[0]);
    conv32_init_kernel<<<1, 1, 0, st>>>(acc, flags);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int cur = 0;
    const int T = npad / 32;
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        for (int r = 0; r < npad - 1; ++r) {
            round_kernel<<<2 * T * T, 256, 0, st>>>(Ab[cur], Ab[cur ^ 1], Qb[cur], Qb[cur ^ 1], npad, n, flags);
            cur ^= 1;
        }
        off32_gated_kernel<<<296, 256, 0, st>>>(Ab[cur], npad, acc, flags);
        conv32_kernel<<<1, 1, 0, st>>>(acc, flags, cur);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    extract_q_kernel<<<592, 256, 0, st>>>(Qb[0], Qb[1], flags, npad, n, Q0);
    return cudaGetLastError();
}

}  // namespace pjac
