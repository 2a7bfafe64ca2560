// Dense products of the preconditioner (Shao & Nakatsukasa, Sec. 2.1):
// the Newton--Schulz reorthogonalisation X <- X (3I - X^T X)/2 and the
// preconditioned matrix A1 = Q^T A Q.  This file holds the plain FP64
// product on the CUDA cores and the element-wise helpers; the tensor-core
// split-precision product is in gemm_tc.cu.
#include <cuda_runtime.h>
#include <cstdint>
#include "internal.h"

namespace pjac {

// C = alpha * op(A) * op(B) + beta * C, column-major, FP64 FMA accumulation.
// 64x64 tile per CTA, 16-deep K slices staged in shared memory, 4x4 outputs
// per thread.
constexpr int GB = 64, GK = 16;

__global__ void __launch_bounds__(256) gemm_f64_kernel(bool ta, bool tb, int m, int n, int k,
                                                       double alpha, const double* __restrict__ A,
                                                       long long lda, const double* __restrict__ B,
                                                       long long ldb, double beta, double* C,
                                                       long long ldc) {
    __shared__ double As[GK][GB + 1];
    __shared__ double Bs[GK][GB + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.x * GB, n0 = blockIdx.y * GB;
    double acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
    for (int k0 = 0; k0 < k; k0 += GK) {
        // load op(A)[m0:m0+64, k0:k0+16] into As[kk][mm]
        for (int e = threadIdx.x; e < GB * GK; e += 256) {
            int mm, kk;
            double v = 0.0;
            if (!ta) {  // A is m x k: element (i, kk) at A[i + kk*lda]; consecutive threads along m
                mm = e % GB; kk = e / GB;
                int gi = m0 + mm, gk = k0 + kk;
                if (gi < m && gk < k) v = A[gi + (long long)gk * lda];
            } else {    // op(A) = A^T, A is k x m: element (i, kk) at A[kk + i*lda]; along k
                kk = e % GK; mm = e / GK;
                int gi = m0 + mm, gk = k0 + kk;
                if (gi < m && gk < k) v = A[gk + (long long)gi * lda];
            }
            As[kk][mm] = v;
        }
        for (int e = threadIdx.x; e < GB * GK; e += 256) {
            int nn, kk;
            double v = 0.0;
            if (!tb) {  // B is k x n: element (kk, j) at B[kk + j*ldb]; along k
                kk = e % GK; nn = e / GK;
                int gk = k0 + kk, gj = n0 + nn;
                if (gk < k && gj < n) v = B[gk + (long long)gj * ldb];
            } else {    // op(B) = B^T, B is n x k: element (kk, j) at B[j + kk*ldb]; along n
                nn = e % GB; kk = e / GB;
                int gk = k0 + kk, gj = n0 + nn;
                if (gk < k && gj < n) v = B[gj + (long long)gk * ldb];
            }
            Bs[kk][nn] = v;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
            double av[4], bv[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) av[a] = As[kk][tx + 16 * a];
#pragma unroll
            for (int b = 0; b < 4; ++b) bv[b] = Bs[kk][ty + 16 * b];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = __fma_rn(av[a], bv[b], acc[a][b]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            int gi = m0 + tx + 16 * a, gj = n0 + ty + 16 * b;
            if (gi < m && gj < n) {
                double* c = C + gi + (long long)gj * ldc;
                double r = alpha * acc[a][b];
                if (beta != 0.0) r = __fma_rn(beta, *c, r);
                *c = r;
            }
        }
}

cudaError_t gemm_f64(bool ta, bool tb, int m, int n, int k, double alpha, const double* A,
                     long long lda, const double* B, long long ldb, double beta, double* C,
                     long long ldc, cudaStream_t st) {
    dim3 g((m + GB - 1) / GB, (n + GB - 1) / GB);
    gemm_f64_kernel<<<g, 256, 0, st>>>(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc);
    return cudaGetLastError();
}

// A <- (A + A^T)/2 (upper and lower written from the same pair).
__global__ void symmetrize_kernel(double* A, long long lda, int n) {
    int i = blockIdx.x * 32 + threadIdx.x;
    int j = blockIdx.y * 32 + threadIdx.y;
    if (i >= n || j >= n || i > j) return;
    double a = A[i + (long long)j * lda], b = A[j + (long long)i * lda];
    double v = 0.5 * (a + b);
    A[i + (long long)j * lda] = v;
    A[j + (long long)i * lda] = v;
}

cudaError_t symmetrize(double* A, long long lda, int n, cudaStream_t st) {
    dim3 g((n + 31) / 32, (n + 31) / 32), b(32, 32);
    symmetrize_kernel<<<g, b, 0, st>>>(A, lda, n);
    return cudaGetLastError();
}

__global__ void copy_f32_f64_kernel(const float* s, long long lds, double* d, long long ldd, int n) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)n * n;
    for (; e < tot; e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e % n), c = (int)(e / n);
        d[r + c * ldd] = (double)s[r + c * lds];
    }
}

cudaError_t copy_f32_to_f64(const float* src, long long lds, double* dst, long long ldd, int n,
                            cudaStream_t st) {
    copy_f32_f64_kernel<<<592, 256, 0, st>>>(src, lds, dst, ldd, n);
    return cudaGetLastError();
}

__global__ void copy_f64_kernel(const double* s, long long lds, double* d, long long ldd, int m, int n) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)m * n;
    for (; e < tot; e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e % m), c = (int)(e / m);
        d[r + c * ldd] = s[r + c * lds];
    }
}

cudaError_t copy_f64(const double* src, long long lds, double* dst, long long ldd, int m, int n,
                     cudaStream_t st) {
    copy_f64_kernel<<<592, 256, 0, st>>>(src, lds, dst, ldd, m, n);
    return cudaGetLastError();
}

__global__ void copy_f64_f32_kernel(const double* s, long long lds, float* d, long long ldd, int n) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long nn = (long long)n * n;
    for (; e < nn; e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e % n), c = (int)(e / n);
        d[(long long)c * ldd + r] = __double2float_rn(s[(long long)c * lds + r]);
    }
}

cudaError_t copy_f64_to_f32(const double* src, long long lds, float* dst, long long ldd, int n, cudaStream_t st) {
    long long nn = (long long)n * n;
    int blocks = (int)((nn + 255) / 256);
    if (blocks > 4096) blocks = 4096;
    copy_f64_f32_kernel<<<blocks, 256, 0, st>>>(src, lds, dst, ldd, n);
    return cudaGetLastError();
}

// First-order refinement (see pjac_opts.refine_steps): Z = D with
// D_ij = e_ij / (d_j - d_i) where |e_ij| <= tau |d_j - d_i|, else 0, for the
// nearly diagonal A1 = diag(d) + E.  One CTA per column j; the column's
// absolute sum (the row sum of the antisymmetric D) goes into a running
// maximum (non-negative doubles order like their bit patterns).
__global__ void refine_build_kernel(const double* A1, long long lda1, int n, double tau, double* Z,
                                    unsigned long long* maxsum) {
    const int j = blockIdx.x;
    __shared__ double red[8];
    const double dj = A1[(long long)j * lda1 + j];
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        double v = 0.0;
        if (i != j) {
            const double e = A1[(long long)j * lda1 + i];
            const double dl = __dadd_rn(dj, -A1[(long long)i * lda1 + i]);
            if (fabs(e) <= __dmul_rn(tau, fabs(dl)) && dl != 0.0) v = __ddiv_rn(e, dl);
        }
        Z[(long long)j * n + i] = v;
        acc = __dadd_rn(acc, fabs(v));
    }
    for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = __dadd_rn(t, red[w]);
        atomicMax(maxsum, (unsigned long long)__double_as_longlong(t));
    }
}

// E <- s D with s = min(1, limit / max row sum)  (Z = I + E).
__global__ void refine_scale_kernel(double* Z, int n, const unsigned long long* maxsum, double limit) {
    const double m = __longlong_as_double((long long)*maxsum);
    const double s = (m > limit) ? __ddiv_rn(limit, m) : 1.0;
    const long long nn = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
         e += (long long)gridDim.x * blockDim.x)
        Z[e] = __dmul_rn(s, Z[e]);
}

// The refinement works on E = Z - I, so that every product involves only
// the small E (and the split product's error, relative to the operands'
// row and column scales, stays relative to |E|).
// R = E^T E + E + E^T: Y holds E^T E on entry.
__global__ void refine_r_kernel(double* Y, const double* E, int n) {
    const long long nn = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e % n), c = (int)(e / n);
        Y[e] = __dadd_rn(Y[e], __dadd_rn(E[e], E[(long long)r * n + c]));
    }
}

// Newton--Schulz on Z = I + E, Z <- Z (I - R/2): E <- E - R/2 + T with
// T = -E R / 2 on entry.
__global__ void refine_ns_kernel(double* E, const double* R, const double* T, int n) {
    const long long nn = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
         e += (long long)gridDim.x * blockDim.x)
        E[e] = __dadd_rn(E[e], __dadd_rn(__dmul_rn(-0.5, R[e]), T[e]));
}

// Z^T A1 Z = A1 + (T + T^T + E^T T) with T = A1 E; Y holds E^T T.
__global__ void refine_a1_kernel(double* A1, long long lda1, const double* T, const double* Y, int n) {
    const long long nn = (long long)n * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nn;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e % n), c = (int)(e / n);
        const double d = __dadd_rn(__dadd_rn(T[e], T[(long long)r * n + c]), Y[e]);
        A1[(long long)c * lda1 + r] = __dadd_rn(A1[(long long)c * lda1 + r], d);
    }
}

cudaError_t refine_r(double* Y, const double* E, int n, cudaStream_t st) {
    refine_r_kernel<<<592, 256, 0, st>>>(Y, E, n);
    return cudaGetLastError();
}
cudaError_t refine_ns(double* E, const double* R, const double* T, int n, cudaStream_t st) {
    refine_ns_kernel<<<592, 256, 0, st>>>(E, R, T, n);
    return cudaGetLastError();
}
cudaError_t refine_a1(double* A1, long long lda1, const double* T, const double* Y, int n, cudaStream_t st) {
    refine_a1_kernel<<<592, 256, 0, st>>>(A1, lda1, T, Y, n);
    return cudaGetLastError();
}

cudaError_t refine_build(const double* A1, long long lda1, int n, double tau, double* Z,
                         unsigned long long* maxsum, double limit, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(maxsum, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    refine_build_kernel<<<n, 256, 0, st>>>(A1, lda1, n, tau, Z, maxsum);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    refine_scale_kernel<<<592, 256, 0, st>>>(Z, n, maxsum, limit);
    return cudaGetLastError();
}

__global__ void identity_kernel(double* d, long long ldd, int n) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)n * n;
    for (; e < tot; e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e % n), c = (int)(e / n);
        d[r + c * ldd] = (r == c) ? 1.0 : 0.0;
    }
}

cudaError_t set_identity(double* dst, long long ldd, int n, cudaStream_t st) {
    identity_kernel<<<592, 256, 0, st>>>(dst, ldd, n);
    return cudaGetLastError();
}

// dst = fl64(fl32(src)): the matrix the FP32 decomposition describes
__global__ void round_fp32_kernel(const double* s, long long lds, double* d, long long ldd, int n) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)n * n;
    for (; e < tot; e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e % n), c = (int)(e / n);
        d[r + c * ldd] = (double)__double2float_rn(s[r + c * lds]);
    }
}

cudaError_t round_to_fp32(const double* src, long long lds, double* dst, long long ldd, int n, cudaStream_t st) {
    round_fp32_kernel<<<592, 256, 0, st>>>(src, lds, dst, ldd, n);
    return cudaGetLastError();
}

// X <- X + Y
__global__ void add_f64_kernel(double* X, long long ldx, const double* Y, long long ldy, int n) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)n * n;
    for (; e < tot; e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e % n), c = (int)(e / n);
        X[r + c * ldx] += Y[r + c * ldy];
    }
}

cudaError_t add_f64(double* X, long long ldx, const double* Y, long long ldy, int n, cudaStream_t st) {
    add_f64_kernel<<<592, 256, 0, st>>>(X, ldx, Y, ldy, n);
    return cudaGetLastError();
}

// Y <- 3I - Y
__global__ void three_i_minus_kernel(double* Y, long long ldy, int n) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)n * n;
    for (; e < tot; e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e % n), c = (int)(e / n);
        double* p = Y + r + c * ldy;
        *p = ((r == c) ? 3.0 : 0.0) - *p;
    }
}

cudaError_t three_i_minus(double* Y, long long ldy, int n, cudaStream_t st) {
    three_i_minus_kernel<<<592, 256, 0, st>>>(Y, ldy, n);
    return cudaGetLastError();
}

// Sets *flag = 1 if any entry is NaN or Inf, 2 if A is not exactly symmetric.
__global__ void check_finite_kernel(const double* A, long long lda, int n, int* flag) {
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long tot = (long long)n * n;
    for (; e < tot; e += (long long)gridDim.x * blockDim.x) {
        int r = (int)(e % n), c = (int)(e / n);
        double v = A[r + c * lda];
        if (!isfinite(v)) atomicOr(flag, 1);
        else if (r < c && v != A[c + (long long)r * lda]) atomicOr(flag, 2);
    }
}

cudaError_t check_finite(const double* A, long long lda, int n, int* d_flag, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(d_flag, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    check_finite_kernel<<<592, 256, 0, st>>>(A, lda, n, d_flag);
    return cudaGetLastError();
}

// Loads this file's kernels on the current device: asking for a kernel's
// attributes loads it, where a first launch would otherwise do so later.
cudaError_t preload_gemm_kernels() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, gemm_f64_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, symmetrize_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, copy_f32_f64_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, copy_f64_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, identity_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, round_fp32_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, add_f64_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, three_i_minus_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, check_finite_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, copy_f64_f32_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, refine_build_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, refine_scale_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, refine_r_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, refine_ns_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, refine_a1_kernel);
    return e;
}

}  // namespace pjac
