// Readout of the one-sided Jacobi SVD (Shao & Nakatsukasa, Alg. 2 and the
// SVD paragraph of Sec. 2.1): the singular values are the norms of the
// columns of the rotated matrix B V, sorted descending; U holds those
// columns normalised, V the rotations' columns in the same order.
#include <cuda_runtime.h>
#include <climits>
#include "devmath.cuh"
#include "internal.h"

namespace pjac {

// ||x_k||_2 of every column of X (m x n, ld ldx): one CTA per column, the
// maximum first, then the sum of squares of the entries scaled by the exact
// power of two 2^-e, e = ilogb(max), so that no square overflows or
// underflows.
__global__ void colnorm_kernel(const double* X, long long ldx, int m, double* out) {
    const int k = blockIdx.x;
    const double* x = X + (long long)k * ldx;
    __shared__ double red[8];
    __shared__ double sm;
    double mx = 0.0;
    for (int r = threadIdx.x; r < m; r += blockDim.x) mx = fmax(mx, fabs(x[r]));
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
        sm = t;
    }
    __syncthreads();
    const double m0 = sm;
    if (m0 == 0.0) {
        if (threadIdx.x == 0) out[k] = 0.0;
        return;
    }
    const int e = ilogb(m0);
    double acc = 0.0;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        const double v = ldexp(x[r], -e);
        acc = __fma_rn(v, v, acc);
    }
    for (int o = 16; o > 0; o >>= 1) acc = __dadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t = __dadd_rn(t, red[w]);
        out[k] = ldexp(__dsqrt_rn(t), e);
    }
}

// rank of sigma_k in descending order, ties by index
__global__ void svd_rank_kernel(const double* sig, int n, int* rank) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const double s = sig[k];
    int r = 0;
    for (int l = 0; l < n; ++l) {
        const double o = sig[l];
        r += (o > s) || (o == s && l < k);
    }
    rank[k] = r;
}

__global__ void svd_gather_kernel(const double* sig, const int* rank, const double* BF, long long ldbf, int m,
                                  const double* Vw, long long ldvw, int n, double* S, double* U, long long ldu,
                                  double* V, long long ldv) {
    const int k = blockIdx.y;
    const int r = rank[k];
    const double s = sig[k];
    if (blockIdx.x == 0 && threadIdx.x == 0) S[r] = s;
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < m; row += gridDim.x * blockDim.x) {
        if (U) U[(long long)r * ldu + row] = (s > 0.0) ? __ddiv_rn(BF[(long long)k * ldbf + row], s) : 0.0;
        if (V && row < n) V[(long long)r * ldv + row] = Vw[(long long)k * ldvw + row];
    }
}

__global__ void check_finite_rect_kernel(const double* A, long long lda, int m, int n, int* flag) {
    const long long tot = (long long)m * n;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < tot;
         e += (long long)gridDim.x * blockDim.x) {
        const int r = (int)(e % m), c = (int)(e / m);
        if (!isfinite(A[r + (long long)c * lda])) atomicOr(flag, 1);
    }
}

cudaError_t check_finite_rect(const double* A, long long lda, int m, int n, int* d_flag, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(d_flag, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    check_finite_rect_kernel<<<592, 256, 0, st>>>(A, lda, m, n, d_flag);
    return cudaGetLastError();
}

cudaError_t launch_svd_readout(const double* BF, long long ldbf, int m, const double* Vw, long long ldvw, int n,
                               double* sig, int* rank, double* S, double* U, long long ldu, double* V,
                               long long ldv, cudaStream_t st) {
    colnorm_kernel<<<n, 256, 0, st>>>(BF, ldbf, m, sig);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    svd_rank_kernel<<<(n + 255) / 256, 256, 0, st>>>(sig, n, rank);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 g((m + 255) / 256, n);
    svd_gather_kernel<<<g, 256, 0, st>>>(sig, rank, BF, ldbf, m, Vw, ldvw, n, S, U, ldu, V, ldv);
    return cudaGetLastError();
}

cudaError_t preload_svd_kernels() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, colnorm_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, svd_rank_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, svd_gather_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, check_finite_rect_kernel);
    return e;
}


// ---------------------------------------------------------------------------
// One-sided Jacobi with inner products recomputed from the columns (Alg. 2
// in Sec. 4.2's relative-accuracy setting, no preconditioner).  One CTA.
// B (m x n, ld m) is rotated in place; G = B^T B of the current columns is
// kept in global memory, formed once and then refreshed in rows/columns i, j
// after every rotation, each entry a dot product accumulated in row order
// with fma (so every value is the oracle's bit for bit).  A per-row best
// score (value, column) lives in shared memory and is updated as in Sec. 3.2.
// ---------------------------------------------------------------------------
namespace {
constexpr int OS_NT = 256;

__device__ __forceinline__ double os_dot(const double* x, const double* y, int m) {
    double acc = 0.0;
    for (int r = 0; r < m; ++r) acc = __fma_rn(__ldcg(x + r), __ldcg(y + r), acc);
    return acc;
}

__device__ __forceinline__ double os_score(int pivot, const double* G, int n, int k, int l) {
    const double gkl = __ldcg(G + (long long)k * n + l);
    if (pivot == PJAC_PIVOT_GREEDY) return fabs(gkl);
    const double gkk = __ldcg(G + (long long)k * n + k), gll = __ldcg(G + (long long)l * n + l);
    const double L = gap_exact(gkk, gll, gkl);
    if (pivot == PJAC_PIVOT_GAP) return L;
    // Sec. 4.2: (1/g_kk + 1/g_ll) L_kl
    if (gkl == 0.0 || gkk == 0.0 || gll == 0.0) return 0.0;
    return __dmul_rn(__dadd_rn(__ddiv_rn(1.0, gkk), __ddiv_rn(1.0, gll)), L);
}

// a larger value wins; equal values go to the smaller column
__device__ __forceinline__ void warp_argmax(double& v, int& c) {
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, v, o);
        const int oc = __shfl_xor_sync(0xffffffffu, c, o);
        if (ov > v || (ov == v && oc < c)) { v = ov; c = oc; }
    }
}

// row k's best (value, column) over l != k, by one warp
__device__ void os_rescan_warp(int pivot, const double* G, int n, int k, double* bv, int* bc) {
    const int lane = threadIdx.x & 31;
    double best = -1.0;
    int col = INT_MAX;
    for (int l = lane; l < n; l += 32) {
        if (l == k) continue;
        const double v = os_score(pivot, G, n, k, l);
        if (v > best) { best = v; col = l; }
    }
    warp_argmax(best, col);
    if (lane == 0) {
        bv[k] = best;
        bc[k] = (col == INT_MAX) ? ((k == 0) ? 1 : 0) : col;
    }
}
}  // namespace

__global__ void __launch_bounds__(OS_NT) svd_onesided_kernel(double* B, int m, int n, double* V, double* G,
                                                             int pivot, double tol, long long max_rot,
                                                             unsigned long long seed, long long budget_ns,
                                                             DevInfo* info) {
    extern __shared__ __align__(16) unsigned char dyn[];
    double* bv = reinterpret_cast<double*>(dyn);
    int* bc = reinterpret_cast<int*>(bv + n);
    int* resc = bc + n;
    __shared__ double red_v[OS_NT / 32];
    __shared__ int red_k[OS_NT / 32];
    __shared__ double s_c, s_s, s_thr;
    __shared__ int s_i, s_j, s_dec, s_nresc;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned long long start = now_ns();
    const int score_pivot = (pivot == PJAC_PIVOT_RANDOM) ? PJAC_PIVOT_GAP_REL : pivot;
    // the Gram matrix of the columns
    const long long npair = (long long)n * (n + 1) / 2;
    for (long long p = tid; p < npair; p += OS_NT) {
        int k = (int)((sqrt(8.0 * (double)p + 1.0) - 1.0) * 0.5);
        while ((long long)k * (k + 1) / 2 > p) --k;
        while ((long long)(k + 1) * (k + 2) / 2 <= p) ++k;
        const int l = (int)(p - (long long)k * (k + 1) / 2);
        const double g = os_dot(B + (long long)k * m, B + (long long)l * m, m);
        __stcg(G + (long long)k * n + l, g);
        __stcg(G + (long long)l * n + k, g);
    }
    __syncthreads();
    // ||G||_F (scaled) for the absolute thresholds
    if (tid == 0) {
        double mx = 0.0;
        for (long long e = 0; e < (long long)n * n; ++e) mx = fmax(mx, fabs(__ldcg(G + e)));
        double nf = 0.0;
        if (mx > 0.0) {
            const int ex = ilogb(mx);
            double acc = 0.0;
            for (long long e = 0; e < (long long)n * n; ++e) {
                const double x = ldexp(__ldcg(G + e), -ex);
                acc = __dadd_rn(acc, __dmul_rn(x, x));
            }
            nf = ldexp(sqrt(acc), ex);
        }
        s_thr = (score_pivot == PJAC_PIVOT_GAP_REL) ? tol : tol * nf;
    }
    for (int k = warp; k < n; k += OS_NT / 32) os_rescan_warp(score_pivot, G, n, k, bv, bc);
    __syncthreads();
    const double thr = s_thr;
    long long rot = 0;
    int status = PJAC_ENOCONV;
    double last = 0.0;
    for (;;) {
        // pivot: the best row (ties to the smallest row), or a draw
        if (pivot == PJAC_PIVOT_RANDOM) {
            if (rot % n == 0) {
                double mx = 0.0;
                for (int k = tid; k < n; k += OS_NT) mx = fmax(mx, bv[k]);
                for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
                if (lane == 0) red_v[warp] = mx;
                __syncthreads();
                if (tid == 0) {
                    double t = 0.0;
                    for (int w = 0; w < OS_NT / 32; ++w) t = fmax(t, red_v[w]);
                    s_dec = (t <= thr) ? 1 : 0;
                }
                __syncthreads();
                if (s_dec) { status = PJAC_OK; break; }
            }
            if (rot >= max_rot) break;
            if (tid == 0) {
                int i, j;
                random_pair(seed, rot, n, i, j);
                s_i = i;
                s_j = j;
            }
        } else {
            double v = -2.0;
            int kk = INT_MAX;
            for (int k = tid; k < n; k += OS_NT)
                if (bv[k] > v) { v = bv[k]; kk = k; }
            warp_argmax(v, kk);
            if (lane == 0) { red_v[warp] = v; red_k[warp] = kk; }
            __syncthreads();
            if (tid == 0) {
                double bvv = red_v[0];
                int bk = red_k[0];
                for (int w = 1; w < OS_NT / 32; ++w)
                    if (red_v[w] > bvv || (red_v[w] == bvv && red_k[w] < bk)) { bvv = red_v[w]; bk = red_k[w]; }
                int dec = 0;
                if (bvv <= thr || bvv == 0.0) dec = 1;
                else if (rot >= max_rot) dec = 3;
                if (budget_ns > 0 && (long long)(now_ns() - start) > budget_ns) dec = 2;
                s_dec = dec;
                last = bvv;
                const int l = bc[bk];
                s_i = min(bk, l);
                s_j = max(bk, l);
            }
            __syncthreads();
            const int dec = s_dec;
            if (dec == 1) { status = PJAC_OK; break; }
            if (dec == 3) break;
            if (dec == 2) { status = PJAC_ETIMEOUT; break; }
        }
        if (tid == 0) {
            const int i = s_i, j = s_j;
            const Rot rp = rot_params(__ldcg(G + (long long)i * n + i), __ldcg(G + (long long)j * n + j),
                                      __ldcg(G + (long long)i * n + j));
            s_c = rp.c;
            s_s = rp.s;
            s_nresc = 0;
        }
        __syncthreads();
        const int i = s_i, j = s_j;
        const double c = s_c, s = s_s;
        double* bi = B + (long long)i * m;
        double* bj = B + (long long)j * m;
        for (int r = tid; r < m; r += OS_NT) {
            const double x = __ldcg(bi + r), y = __ldcg(bj + r);
            __stcg(bi + r, __fma_rn(c, x, __dmul_rn(s, y)));
            __stcg(bj + r, __fma_rn(c, y, -__dmul_rn(s, x)));
        }
        if (V) {
            double* vi = V + (long long)i * n;
            double* vj = V + (long long)j * n;
            for (int r = tid; r < n; r += OS_NT) {
                const double x = vi[r], y = vj[r];
                vi[r] = __fma_rn(c, x, __dmul_rn(s, y));
                vj[r] = __fma_rn(c, y, -__dmul_rn(s, x));
            }
        }
        __syncthreads();
        // rows and columns i, j of G from the rotated columns
        for (int k = tid; k < n; k += OS_NT) {
            const double* bk = B + (long long)k * m;
            double gi = 0.0, gj = 0.0;
            for (int r = 0; r < m; ++r) {
                const double y = __ldcg(bk + r);
                gi = __fma_rn(__ldcg(bi + r), y, gi);
                gj = __fma_rn(__ldcg(bj + r), y, gj);
            }
            __stcg(G + (long long)i * n + k, gi);
            __stcg(G + (long long)k * n + i, gi);
            __stcg(G + (long long)j * n + k, gj);
            __stcg(G + (long long)k * n + j, gj);
        }
        rot++;
        __syncthreads();
        // row-best cache: rows i, j and rows whose best was in column i or j
        // are rescanned; the others compare their entries (k,i), (k,j)
        for (int k = tid; k < n; k += OS_NT) {
            if (k == i || k == j || bc[k] == i || bc[k] == j) {
                resc[atomicAdd(&s_nresc, 1)] = k;
                continue;
            }
            double b = bv[k];
            int col = bc[k];
            const double vi2 = os_score(score_pivot, G, n, k, i);
            if (vi2 > b || (vi2 == b && i < col)) { b = vi2; col = i; }
            const double vj2 = os_score(score_pivot, G, n, k, j);
            if (vj2 > b || (vj2 == b && j < col)) { b = vj2; col = j; }
            bv[k] = b;
            bc[k] = col;
        }
        __syncthreads();
        const int nr = s_nresc;
        for (int q = warp; q < nr; q += OS_NT / 32) os_rescan_warp(score_pivot, G, n, resc[q], bv, bc);
        __syncthreads();
    }
    if (tid == 0 && info) {
        DevInfo d;
        d.rotations = rot;
        d.sweeps = 0;
        d.off = 0.0;
        d.normf = 0.0;
        d.max_score = last;
        d.status = status;
        d.n = n;
        d.steps = rot;
        *info = d;
    }
}

__global__ void os_sigma_kernel(const double* G, int n, double* sig) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n) sig[k] = __dsqrt_rn(fmax(G[(long long)k * n + k], 0.0));
}

cudaError_t launch_svd_onesided(double* B, int m, int n, double* V, double* G, int pivot, double tol,
                                long long max_rot, unsigned long long seed, long long budget_ns, DevInfo* info,
                                cudaStream_t st) {
    const size_t smem = (size_t)n * (sizeof(double) + 2 * sizeof(int));
    cudaError_t e = cudaFuncSetAttribute(svd_onesided_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    svd_onesided_kernel<<<1, OS_NT, smem, st>>>(B, m, n, V, G, pivot, tol, max_rot, seed, budget_ns, info);
    return cudaGetLastError();
}

cudaError_t launch_os_readout(const double* G, const double* Brot, int m, const double* Vw, int n, double* sig,
                              int* rank, double* S, double* U, long long ldu, double* V, long long ldv,
                              cudaStream_t st) {
    os_sigma_kernel<<<(n + 255) / 256, 256, 0, st>>>(G, n, sig);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    svd_rank_kernel<<<(n + 255) / 256, 256, 0, st>>>(sig, n, rank);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    dim3 g((m + 255) / 256, n);
    svd_gather_kernel<<<g, 256, 0, st>>>(sig, rank, Brot, m, m, Vw, n, n, S, U, ldu, V, ldv);
    return cudaGetLastError();
}

cudaError_t preload_os_kernels() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, svd_onesided_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, os_sigma_kernel);
    return e;
}

}  // namespace pjac
