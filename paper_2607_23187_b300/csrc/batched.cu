// Batched form: thousands of independent eigenproblems of mixed orders in
// one stream of device work, without host synchronisation (so a call can be
// captured in a CUDA graph).  Every problem follows the single-problem
// pipeline: FP32 diagonalisation of fl32(A) (Sec. 2.1, u_l = single),
// Newton--Schulz reorthogonalisation, A1 = Q^T A Q, Algorithm 1, readout.
//
// Each stage is one launch of persistent CTAs that take problems from a
// device work queue, largest order first.
#include <cuda_runtime.h>
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <map>
#include <vector>
#include "internal.h"

namespace pjac {

int set_err(int code, const char* fmt, ...);
int cuda_err(cudaError_t e, const char* what);

constexpr int BT = 256;          // threads per CTA of the batched stages
constexpr int SMEM_N32 = 128;    // FP32 diagonaliser state in shared memory up to this order

__device__ __forceinline__ int take_problem(int* counter, int* sh_next) {
    if (threadIdx.x == 0) *sh_next = atomicAdd(counter, 1);
    __syncthreads();
    int t = *sh_next;
    __syncthreads();
    return t;
}

__device__ __forceinline__ void rot32b(float app, float aqq, float apq, float& c, float& s) {
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

// Z = G_a^T X G_b for one 2x2 block with the products summed in the same
// pairs for the block and its transpose, so the matrix stays exactly
// symmetric (see diag32.cu).
__device__ __forceinline__ void rot2x2_symb(float ca, float sa, float cb, float sb, float x00, float x01,
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

// Round-robin tournament (circle method) on N players (N even): in round r
// pair 0 is (N-1, r) and pair k >= 1 is ((r+k) mod (N-1), (r-k) mod (N-1)).
__device__ __forceinline__ void rr_pair(int r, int k, int N, int& p, int& q) {
    if (k == 0) { p = N - 1; q = r; }
    else {
        p = (r + k) % (N - 1);
        q = (r - k + (N - 1)) % (N - 1);
    }
    if (p > q) { int t = p; p = q; q = t; }
}

// Stage 1: FP32 parallel-order Jacobi on fl32(A) per problem.
__global__ void __launch_bounds__(BT) b_diag32_kernel(const BatchDesc* desc, int nb, const int* order,
                                                      int* counter, int max_sweeps) {
    extern __shared__ __align__(16) unsigned char dyn[];
    __shared__ int next;
    __shared__ float cs[512][2];
    __shared__ short pp[512][2];
    __shared__ double red[BT / 32][2];
    __shared__ int stop;
    for (;;) {
        int t = take_problem(counter, &next);
        if (t >= nb) break;
        BatchDesc d = desc[order[t]];
        const int n = d.n;
        const int N = n + (n & 1);
        const int npairs = N / 2;
        float* A = (n <= SMEM_N32) ? reinterpret_cast<float*>(dyn) : d.A32;
        float* Q = (n <= SMEM_N32) ? reinterpret_cast<float*>(dyn) + n * n : d.Q32;
        for (int e = threadIdx.x; e < n * n; e += BT) {
            int r = e % n, c = e / n;
            A[e] = (float)d.Ain[e];
            Q[e] = (r == c) ? 1.0f : 0.0f;
        }
        __syncthreads();
        double prev = -1.0;
        const int nsw = d.sweeps32 > 0 ? d.sweeps32 : max_sweeps;
        for (int sweep = 0; sweep < nsw; ++sweep) {
            for (int r = 0; r < N - 1; ++r) {
                for (int k = threadIdx.x; k < npairs; k += BT) {
                    int p, q;
                    rr_pair(r, k, N, p, q);
                    float c = 1.0f, s = 0.0f;
                    if (q < n) rot32b(A[p + p * n], A[q + q * n], A[p + q * n], c, s);
                    cs[k][0] = c; cs[k][1] = s;
                    pp[k][0] = (short)p; pp[k][1] = (short)q;
                }
                __syncthreads();
                // A <- G^T A G on 2x2 blocks (pair a rows, pair b cols), in place
                for (int e = threadIdx.x; e < npairs * npairs; e += BT) {
                    int a = e % npairs, b = e / npairs;
                    int pa = pp[a][0], qa = pp[a][1], pb = pp[b][0], qb = pp[b][1];
                    // for odd n the dummy player (index n) is always the second of
                    // its pair; its row/column does not exist and its rotation is
                    // the identity, but the real partner is still rotated
                    const bool ra = qa < n, rb = qb < n;
                    float ca = cs[a][0], sa = cs[a][1], cb = cs[b][0], sb = cs[b][1];
                    float x00 = A[pa + pb * n];
                    float x10 = ra ? A[qa + pb * n] : 0.0f;
                    float x01 = rb ? A[pa + qb * n] : 0.0f;
                    float x11 = (ra && rb) ? A[qa + qb * n] : 0.0f;
                    float z00, z01, z10, z11;
                    rot2x2_symb(ca, sa, cb, sb, x00, x01, x10, x11, z00, z01, z10, z11);
                    if (a == b && sa != 0.0f) { z01 = 0.0f; z10 = 0.0f; }
                    A[pa + pb * n] = z00;
                    if (ra) A[qa + pb * n] = z10;
                    if (rb) A[pa + qb * n] = z01;
                    if (ra && rb) A[qa + qb * n] = z11;
                }
                // Q <- Q G on column pairs
                for (int e = threadIdx.x; e < n * npairs; e += BT) {
                    int row = e % n, k = e / n;
                    int p = pp[k][0], q = pp[k][1];
                    if (q >= n) continue;
                    float c = cs[k][0], s = cs[k][1];
                    float q0 = Q[row + p * n], q1 = Q[row + q * n];
                    Q[row + p * n] = q0 * c + q1 * s;
                    Q[row + q * n] = -q0 * s + q1 * c;
                }
                __syncthreads();
            }
            // convergence: off^2 vs ||A||^2 (FP64 accumulation)
            double off = 0.0, all = 0.0;
            for (int e = threadIdx.x; e < n * n; e += BT) {
                double v = (double)A[e];
                all += v * v;
                if (e % n != e / n) off += v * v;
            }
            for (int o = 16; o > 0; o >>= 1) {
                off += __shfl_xor_sync(0xffffffffu, off, o);
                all += __shfl_xor_sync(0xffffffffu, all, o);
            }
            if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5][0] = off; red[threadIdx.x >> 5][1] = all; }
            __syncthreads();
            if (threadIdx.x == 0) {
                double o2 = 0, a2 = 0;
                for (int w = 0; w < BT / 32; ++w) { o2 += red[w][0]; a2 += red[w][1]; }
                int st = 0;
                if (a2 == 0.0 || o2 <= 1e-15 * a2) st = 1;
                else if (prev >= 0.0 && sweep >= 4 && o2 > 0.9 * prev) st = 1;
                prev = o2;
                stop = st;
            }
            __syncthreads();
            if (stop) break;
        }
        for (int e = threadIdx.x; e < n * n; e += BT) d.Q32[e] = Q[e];
        __syncthreads();
    }
}

// C = alpha * op(X) * op(Y), n x n, all leading dimensions n, inside one CTA.
__device__ void cta_gemm(bool tx, bool ty, int n, double alpha, const double* X, const double* Y,
                         double* C, double (*Xs)[65], double (*Ys)[65]) {
    const int ti = threadIdx.x & 15, tj = threadIdx.x >> 4;
    for (int m0 = 0; m0 < n; m0 += 64)
        for (int n0 = 0; n0 < n; n0 += 64) {
            double acc[4][4];
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) acc[a][b] = 0.0;
            for (int k0 = 0; k0 < n; k0 += 16) {
                for (int e = threadIdx.x; e < 64 * 16; e += BT) {
                    int mm = e % 64, kk = e / 64;
                    int gi = m0 + mm, gk = k0 + kk;
                    double v = 0.0;
                    if (gi < n && gk < n) v = tx ? X[gk + gi * n] : X[gi + gk * n];
                    Xs[kk][mm] = v;
                    int nn = e % 64;
                    int gj = n0 + nn;
                    double w = 0.0;
                    if (gj < n && gk < n) w = ty ? Y[gj + gk * n] : Y[gk + gj * n];
                    Ys[kk][nn] = w;
                }
                __syncthreads();
#pragma unroll
                for (int kk = 0; kk < 16; ++kk) {
                    double av[4], bv[4];
#pragma unroll
                    for (int a = 0; a < 4; ++a) av[a] = Xs[kk][ti + 16 * a];
#pragma unroll
                    for (int b = 0; b < 4; ++b) bv[b] = Ys[kk][tj + 16 * b];
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
                    int gi = m0 + ti + 16 * a, gj = n0 + tj + 16 * b;
                    if (gi < n && gj < n) C[gi + gj * n] = alpha * acc[a][b];
                }
        }
    __syncthreads();
}

// Stage 2: Newton--Schulz X <- X(3I - X^T X)/2 from X = fl64(Q0), then
// A1 = X^T A X symmetrised.  V holds X (it becomes V0 = Q of the iteration).
__global__ void __launch_bounds__(BT) b_precond_kernel(const BatchDesc* desc, int nb, const int* order,
                                                       int* counter, int ns_steps) {
    __shared__ double Xs[16][65], Ys[16][65];
    __shared__ int next;
    for (;;) {
        int t = take_problem(counter, &next);
        if (t >= nb) break;
        BatchDesc d = desc[order[t]];
        const int n = d.n;
        for (int e = threadIdx.x; e < n * n; e += BT) d.V[e] = (double)d.Q32[e];
        __syncthreads();
        for (int it = 0; it < ns_steps; ++it) {
            cta_gemm(true, false, n, 1.0, d.V, d.V, d.Y, Xs, Ys);
            for (int e = threadIdx.x; e < n * n; e += BT) {
                int r = e % n, c = e / n;
                d.Y[e] = ((r == c) ? 3.0 : 0.0) - d.Y[e];
            }
            __syncthreads();
            cta_gemm(false, false, n, 0.5, d.V, d.Y, d.T, Xs, Ys);
            for (int e = threadIdx.x; e < n * n; e += BT) d.V[e] = d.T[e];
            __syncthreads();
        }
        cta_gemm(false, false, n, 1.0, d.Ain, d.V, d.T, Xs, Ys);
        cta_gemm(true, false, n, 1.0, d.V, d.T, d.A, Xs, Ys);
        for (int e = threadIdx.x; e < n * n; e += BT) {
            int r = e % n, c = e / n;
            if (r < c) {
                double v = 0.5 * (d.A[r + c * n] + d.A[c + r * n]);
                d.A[r + c * n] = v;
                d.A[c + r * n] = v;
            }
        }
        __syncthreads();
    }
}

// Stage 2b: first-order refinement steps of (A1, V) (see pjac_opts.
// refine_steps): Z = I + s D with D_ij = a_ij/(a_jj - a_ii) for the pairs
// with |a_ij| <= tau |a_jj - a_ii| (else 0), s scaling the largest absolute
// row sum of D to at most 1/4; Z made orthogonal by Newton--Schulz (steps
// until the bound on ||Z^T Z - I|| falls below 1e-20, at most 5); then
// A1 <- Z^T A1 Z symmetrised, V <- V Z.  The parallel FP32 pass of stage 1
// leaves its basis off orthogonality by the rounding of its rotation layers,
// which Newton--Schulz turns into off-diagonal entries of A1 near that
// level; one step brings them back to FP32 accuracy.
__global__ void __launch_bounds__(BT) b_refine_kernel(const BatchDesc* desc, int nb, const int* order,
                                                      int* counter, int steps) {
    __shared__ double Xs[16][65], Ys[16][65];
    __shared__ double red[BT / 32];
    __shared__ int next;
    for (;;) {
        int t = take_problem(counter, &next);
        if (t >= nb) break;
        BatchDesc d = desc[order[t]];
        const int n = d.n;
        const int nsteps = d.refine > 0 ? d.refine : steps;
        for (int step = 0; step < nsteps; ++step) {
            // D, and its largest absolute row (= column) sum
            double mx = 0.0;
            for (int j = threadIdx.x; j < n; j += BT) {
                const double dj = d.A[j + j * n];
                double acc = 0.0;
                for (int i = 0; i < n; ++i) {
                    double v = 0.0;
                    if (i != j) {
                        const double e = d.A[i + j * n];
                        const double dl = __dadd_rn(dj, -d.A[i + i * n]);
                        if (fabs(e) <= __dmul_rn(REFINE_TAU, fabs(dl)) && dl != 0.0) v = __ddiv_rn(e, dl);
                    }
                    d.Z[i + j * n] = v;
                    acc = __dadd_rn(acc, fabs(v));
                }
                mx = fmax(mx, acc);
            }
            for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
            __syncthreads();
            double m = 0.0;
            for (int w = 0; w < BT / 32; ++w) m = fmax(m, red[w]);
            const double sc = (m > REFINE_MAX_ROWSUM) ? __ddiv_rn(REFINE_MAX_ROWSUM, m) : 1.0;
            const double rho = fmin(m, REFINE_MAX_ROWSUM);
            for (int e = threadIdx.x; e < n * n; e += BT) {
                const int r = e % n, c = e / n;
                d.Z[e] = (r == c) ? 1.0 : __dmul_rn(sc, d.Z[e]);
            }
            __syncthreads();
            // Newton--Schulz: ||Z^T Z - I|| <= rho^2 = e0, e_{k+1} <= 3/4 e_k^2 + e_k^3/4
            int ns = 0;
            for (double eb = rho * rho; eb > 1e-20 && ns < REFINE_NS_STEPS; eb = 0.75 * eb * eb + 0.25 * eb * eb * eb)
                ++ns;
            for (int it = 0; it < ns; ++it) {
                cta_gemm(true, false, n, 1.0, d.Z, d.Z, d.Y, Xs, Ys);
                for (int e = threadIdx.x; e < n * n; e += BT) {
                    int r = e % n, c = e / n;
                    d.Y[e] = ((r == c) ? 3.0 : 0.0) - d.Y[e];
                }
                __syncthreads();
                cta_gemm(false, false, n, 0.5, d.Z, d.Y, d.T, Xs, Ys);
                for (int e = threadIdx.x; e < n * n; e += BT) d.Z[e] = d.T[e];
                __syncthreads();
            }
            cta_gemm(false, false, n, 1.0, d.A, d.Z, d.T, Xs, Ys);   // T = A1 Z
            cta_gemm(true, false, n, 1.0, d.Z, d.T, d.A, Xs, Ys);    // A1 = Z^T T
            for (int e = threadIdx.x; e < n * n; e += BT) {
                int r = e % n, c = e / n;
                if (r < c) {
                    double v = 0.5 * (d.A[r + c * n] + d.A[c + r * n]);
                    d.A[r + c * n] = v;
                    d.A[c + r * n] = v;
                }
            }
            __syncthreads();
            cta_gemm(false, false, n, 1.0, d.V, d.Z, d.T, Xs, Ys);   // T = V Z
            for (int e = threadIdx.x; e < n * n; e += BT) d.V[e] = d.T[e];
            __syncthreads();
        }
    }
}

// Without the preconditioner: A1 = A and V0 = I for every problem.
__global__ void __launch_bounds__(BT) b_copyin_kernel(const BatchDesc* desc, int nb) {
    const int p = blockIdx.x;
    if (p >= nb) return;
    const BatchDesc d = desc[p];
    const int n = d.n;
    for (int e = threadIdx.x; e < n * n; e += BT) {
        const int r = e % n, c = e / n;
        d.A[e] = d.Ain[e];
        d.V[e] = (r == c) ? 1.0 : 0.0;
    }
}

// Loads this file's kernels on the current device: asking for a kernel's
// attributes loads it, where a first launch would otherwise do so later.
cudaError_t preload_batched_kernels() {
    cudaFuncAttributes fa;
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, b_diag32_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, b_precond_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, b_copyin_kernel);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, b_refine_kernel);
    return e;
}

// Kernel launches of one pjac_solve_batched call: FP32 diagonaliser,
// preconditioner, refinement, Jacobi, readout, report (without the
// preconditioner: the copy-in replaces the first three).
int batched_launch_count(int no_precondition) { return no_precondition ? 4 : 6; }

}  // namespace pjac

using namespace pjac;

// the autotuner's choice for one (order bucket, pivot rule)
struct TuneChoice { int refine, sweeps; float solves_per_s; };

struct BatchState {
    void* dbuf = nullptr;     // device: descriptors, order, counters, per-problem workspace
    size_t dbytes = 0;
    void* hbuf = nullptr;     // pinned host staging
    size_t hbytes = 0;
    std::vector<void*> held;  // staging buffers read by captured graphs (freed on release)
    cudaEvent_t ev[6] = {};   // stage boundaries of the last call made outside a capture
    bool ev_made = false, ev_valid = false;
    std::map<int, TuneChoice> tuned;   // autotuner: (order bucket, pivot) -> choice
};

// The batched workspace lives in a handle-independent cache keyed by the
// handle pointer (kept simple: one per handle, grown on demand).
#include <mutex>
#include <unordered_map>
static std::mutex g_bmu;
static std::unordered_map<const void*, BatchState> g_bstate;

void pjac_batched_release(const void* h) {
    std::lock_guard<std::mutex> lk(g_bmu);
    auto it = g_bstate.find(h);
    if (it == g_bstate.end()) return;
    if (it->second.ev_made)
        for (cudaEvent_t e : it->second.ev) cudaEventDestroy(e);
    if (it->second.dbuf) cudaFree(it->second.dbuf);
    if (it->second.hbuf) cudaFreeHost(it->second.hbuf);
    for (void* q : it->second.held) cudaFreeHost(q);
    g_bstate.erase(it);
}

static size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

namespace pjac {
int handle_opts(const pjac_handle* h, pjac_opts* o);
}

// The batched pipeline on nb problems, problem q with refinement steps
// refine[q] and FP32 sweep cap sweeps[q].  Called with g_bmu held.
static int batched_core(pjac_handle* h, const pjac_opts& opts, BatchState& bs, int nb, const int* n,
                        const int64_t* a_off, const double* A, const int64_t* w_off, double* W,
                        const int64_t* v_off, double* V, pjac_pivot pivot, double tol, pjac_info* infos,
                        const int* refine, const int* sweeps, cudaStream_t st) {
    (void)h;
    int max_n = 0;
    size_t ws = 0;
    for (int p = 0; p < nb; ++p) {
        max_n = std::max(max_n, n[p]);
        size_t nn = (size_t)n[p] * n[p];
        ws += a256(nn * 8) * 5 + a256((size_t)n[p] * 8) + a256(nn * 4) * 2 + a256(sizeof(DevInfo));
    }
    size_t hdr = a256(sizeof(BatchDesc) * nb) + a256(sizeof(int) * nb) + 256;
    size_t need = hdr + ws;
    if (bs.dbytes < need) {
        // stream-ordered: growing never waits for other streams' work
        if (bs.dbuf) cudaFreeAsync(bs.dbuf, st);
        bs.dbuf = nullptr;
        bs.dbytes = 0;
        cudaError_t e = cudaMallocAsync(&bs.dbuf, need, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_err(PJAC_ENOMEM, "batched workspace of %zu bytes: %s", need, cudaGetErrorString(e));
        }
        bs.dbytes = need;
    }
    size_t hneed = a256(sizeof(BatchDesc) * nb) + a256(sizeof(int) * nb);
    // Inside a stream capture nothing runs now: the copies below become graph
    // nodes that read the staging buffer at every replay, so that buffer is
    // handed to the graph (kept until the handle is destroyed) and later
    // calls stage elsewhere.  Outside a capture the stream is synchronised
    // before the staging buffer is rewritten.
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t ec = cudaStreamIsCapturing(st, &cap);
    if (ec != cudaSuccess) return cuda_err(ec, "cudaStreamIsCapturing");
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    if (bs.hbytes < hneed) {
        // retired, not freed: cudaFreeHost would wait for the whole device
        if (bs.hbuf) bs.held.push_back(bs.hbuf);
        bs.hbuf = nullptr;
        bs.hbytes = 0;
        cudaError_t e = cudaMallocHost(&bs.hbuf, hneed);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_err(PJAC_ENOMEM, "pinned staging of %zu bytes: %s", hneed, cudaGetErrorString(e));
        }
        bs.hbytes = hneed;
    }
    if (!capturing) {
        // the staging buffer may still be read by an earlier call's copy
        cudaError_t e0 = cudaStreamSynchronize(st);
        if (e0 != cudaSuccess) return cuda_err(e0, "cudaStreamSynchronize");
    }
    char* dbase = static_cast<char*>(bs.dbuf);
    BatchDesc* d_desc = reinterpret_cast<BatchDesc*>(dbase);
    int* d_order = reinterpret_cast<int*>(dbase + a256(sizeof(BatchDesc) * nb));
    int* d_counters = reinterpret_cast<int*>(dbase + a256(sizeof(BatchDesc) * nb) + a256(sizeof(int) * nb));
    BatchDesc* h_desc = static_cast<BatchDesc*>(bs.hbuf);
    int* h_order = reinterpret_cast<int*>(static_cast<char*>(bs.hbuf) + a256(sizeof(BatchDesc) * nb));
    char* p = dbase + hdr;
    for (int q = 0; q < nb; ++q) {
        size_t m = (size_t)n[q], nn = m * m;
        BatchDesc d;
        memset(&d, 0, sizeof(d));
        d.Ain = A + a_off[q];
        d.A = reinterpret_cast<double*>(p); p += a256(nn * 8);
        d.V = reinterpret_cast<double*>(p); p += a256(nn * 8);
        d.T = reinterpret_cast<double*>(p); p += a256(nn * 8);
        d.Y = reinterpret_cast<double*>(p); p += a256(nn * 8);
        d.Z = reinterpret_cast<double*>(p); p += a256(nn * 8);
        d.Wd = reinterpret_cast<double*>(p); p += a256(m * 8);
        d.A32 = reinterpret_cast<float*>(p); p += a256(nn * 4);
        d.Q32 = reinterpret_cast<float*>(p); p += a256(nn * 4);
        d.info = reinterpret_cast<DevInfo*>(p); p += a256(sizeof(DevInfo));
        d.Wout = W + w_off[q];
        d.Vout = V ? V + v_off[q] : nullptr;
        d.n = (int)m;
        d.refine = refine[q];
        d.sweeps32 = sweeps[q];
        h_desc[q] = d;
        h_order[q] = q;
    }
    std::stable_sort(h_order, h_order + nb, [&](int x, int y) { return n[x] > n[y]; });
    cudaError_t e;
#define BK(call) do { e = (call); if (e != cudaSuccess) return cuda_err(e, #call); } while (0)
    BK(cudaMemcpyAsync(d_desc, h_desc, sizeof(BatchDesc) * nb, cudaMemcpyHostToDevice, st));
    BK(cudaMemcpyAsync(d_order, h_order, sizeof(int) * nb, cudaMemcpyHostToDevice, st));
    BK(cudaMemsetAsync(d_counters, 0, 8 * sizeof(int), st));
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int ctas = std::min(nb, sms * 2);
    size_t smem32 = (size_t)2 * SMEM_N32 * SMEM_N32 * sizeof(float);
    BK(cudaFuncSetAttribute(b_diag32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem32));
    // stage boundaries, recorded outside a capture (pjac_batched_stage_ms)
    if (!capturing && !bs.ev_made) {
        for (cudaEvent_t& ev : bs.ev) BK(cudaEventCreate(&ev));
        bs.ev_made = true;
    }
    auto mark = [&](int k) -> cudaError_t { return capturing ? cudaSuccess : cudaEventRecord(bs.ev[k], st); };
    bs.ev_valid = false;
    BK(mark(0));
    if (opts.no_precondition) {
        b_copyin_kernel<<<nb, BT, 0, st>>>(d_desc, nb);
        BK(cudaGetLastError());
        BK(mark(1));
        BK(mark(2));
        BK(mark(3));
    } else {
        b_diag32_kernel<<<ctas, BT, smem32, st>>>(d_desc, nb, d_order, d_counters + 0, 40);
        BK(cudaGetLastError());
        BK(mark(1));
        int ns = opts.ns_steps;
        b_precond_kernel<<<std::min(nb, sms * 4), BT, 0, st>>>(d_desc, nb, d_order, d_counters + 1, ns);
        BK(cudaGetLastError());
        BK(mark(2));
        // refinement steps per problem (at least one, which restores the
        // FP32-accurate basis; see b_refine_kernel)
        b_refine_kernel<<<std::min(nb, sms * 4), BT, 0, st>>>(d_desc, nb, d_order, d_counters + 3, 1);
        BK(cudaGetLastError());
        BK(mark(3));
    }
    long long budget = (long long)((opts.time_budget_s > 0 ? opts.time_budget_s : 600.0) * 1e9);   // ns
    BK(launch_jacobi_batched(d_desc, nb, d_order, d_counters + 2, (int)pivot, (int)opts.stop, tol, 25, budget,
                             max_n, std::min(nb, sms * 2), opts.seed, st));
    BK(mark(4));
    BK(launch_readout_batched(d_desc, nb, max_n, st));
    BK(launch_info_batched(d_desc, nb, infos, st));   // keep batched_launch_count() in step
    BK(mark(5));
    bs.ev_valid = !capturing;
#undef BK
    if (capturing) {
        bs.held.push_back(bs.hbuf);
        bs.hbuf = nullptr;
        bs.hbytes = 0;
    }
    return PJAC_OK;
}


// ---------------------------------------------------------------------------
// Autotuner of the batched form.  Per order bucket (n < 32, < 64, < 128,
// <= 256, > 256) and pivot rule it chooses the refinement steps (1, 2 or 3)
// and the FP32 sweep cap (12 or 40) of the problems in that bucket: more
// refinement moves work from the latency-bound Jacobi chain onto the CTA's
// FP64 products, fewer FP32 sweeps shorten stage 1 at the cost of a rougher
// basis.  On the first call outside a stream capture that meets a bucket not
// yet tuned, up to 32 of the call's own problems of that bucket are solved
// with every candidate, timed on the device, and the fastest candidate is
// kept in the handle's cache; later calls (and graphs captured after it)
// reuse it.  opts.autotune = 0 skips it (refinement 1 + opts.refine_steps,
// sweep cap opts.fp32_sweeps or 40).
// ---------------------------------------------------------------------------
static int order_bucket(int n) { return n < 32 ? 0 : n < 64 ? 1 : n < 128 ? 2 : n <= 256 ? 3 : 4; }

static const int kCands[6][2] = {{1, 40}, {2, 40}, {3, 40}, {1, 12}, {2, 12}, {3, 12}};

static int tune_bucket(pjac_handle* h, const pjac_opts& opts, BatchState& bs, const std::vector<int>& idx,
                       const int* n, const int64_t* a_off, const double* A, pjac_pivot pivot, double tol,
                       cudaStream_t st, TuneChoice* out) {
    const int m = (int)idx.size();
    std::vector<int> ns(m);
    std::vector<int64_t> ao(m), wo(m), vo(m);
    int64_t wsum = 0, vsum = 0;
    for (int q = 0; q < m; ++q) {
        ns[q] = n[idx[q]];
        ao[q] = a_off[idx[q]];
        wo[q] = wsum;
        vo[q] = vsum;
        wsum += ns[q];
        vsum += (int64_t)ns[q] * ns[q];
    }
    double* W = nullptr;
    double* V = nullptr;
    pjac_info* inf = nullptr;
    cudaError_t e = cudaMallocAsync(&W, sizeof(double) * wsum, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&V, sizeof(double) * vsum, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&inf, sizeof(pjac_info) * m, st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (W) cudaFreeAsync(W, st);
        if (V) cudaFreeAsync(V, st);
        return set_err(PJAC_ENOMEM, "autotuner buffers: %s", cudaGetErrorString(e));
    }
    float best_ms = -1.f;
    int best = 0;
    int r = PJAC_OK;
    for (int c = 0; c < 6 && r == PJAC_OK; ++c) {
        std::vector<int> rf(m, kCands[c][0]), sw(m, kCands[c][1]);
        r = batched_core(h, opts, bs, m, ns.data(), ao.data(), A, wo.data(), W, vo.data(), V, pivot, tol, inf,
                         rf.data(), sw.data(), st);
        if (r) break;
        if (cudaEventSynchronize(bs.ev[5]) != cudaSuccess) { r = cuda_err(cudaGetLastError(), "tuning"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, bs.ev[0], bs.ev[5]);
        if (best_ms < 0.f || ms < best_ms) { best_ms = ms; best = c; }
    }
    cudaFreeAsync(W, st);
    cudaFreeAsync(V, st);
    cudaFreeAsync(inf, st);
    if (r) return r;
    out->refine = kCands[best][0];
    out->sweeps = kCands[best][1];
    out->solves_per_s = best_ms > 0.f ? 1000.f * m / best_ms : 0.f;
    return PJAC_OK;
}

extern "C" int pjac_solve_batched(pjac_handle* h, int nb, const int* n, const int64_t* a_off, const double* A,
                                  const int64_t* w_off, double* W, const int64_t* v_off, double* V,
                                  pjac_pivot pivot, double tol, pjac_info* infos, void* stream) {
    if (!h || !n || !a_off || !A || !w_off || !W || !infos) return set_err(PJAC_EINVAL, "NULL argument");
    if (V && !v_off) return set_err(PJAC_EINVAL, "v_off is NULL while V is not");
    if (nb < 1) return set_err(PJAC_EINVAL, "nb = %d < 1", nb);
    if (pivot < PJAC_PIVOT_GAP || pivot > PJAC_PIVOT_RANDOM) return set_err(PJAC_EINVAL, "bad pivot");
    if (!(tol >= 0.0)) return set_err(PJAC_EINVAL, "tol must be >= 0");
    pjac_opts opts;
    handle_opts(h, &opts);
    if (opts.stop == PJAC_STOP_LIBOUND && pivot != PJAC_PIVOT_GAP)
        return set_err(PJAC_EINVAL, "PJAC_STOP_LIBOUND needs the gap rule");
    for (int p = 0; p < nb; ++p) {
        if (n[p] < 2 || n[p] > 1024) return set_err(PJAC_EINVAL, "n[%d] = %d outside [2, 1024]", p, n[p]);
        if (a_off[p] < 0 || w_off[p] < 0 || (V && v_off[p] < 0)) return set_err(PJAC_EINVAL, "negative offset");
    }
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t ec = cudaStreamIsCapturing(st, &cap);
    if (ec != cudaSuccess) return cuda_err(ec, "cudaStreamIsCapturing");
    std::lock_guard<std::mutex> lk(g_bmu);
    BatchState& bs = g_bstate[h];
    const int base_refine = 1 + opts.refine_steps;
    const int base_sweeps = opts.fp32_sweeps > 0 ? opts.fp32_sweeps : 40;
    if (opts.autotune && !opts.no_precondition && cap == cudaStreamCaptureStatusNone) {
        std::vector<int> members[5];
        for (int p = 0; p < nb; ++p) members[order_bucket(n[p])].push_back(p);
        for (int b = 0; b < 5; ++b) {
            const int key = b * 16 + (int)pivot;
            if (members[b].size() < 8 || bs.tuned.count(key)) continue;
            std::vector<int> sample;
            const size_t step = std::max<size_t>(1, members[b].size() / 32);
            for (size_t q = 0; q < members[b].size() && sample.size() < 32; q += step) sample.push_back(members[b][q]);
            TuneChoice c;
            int r = tune_bucket(h, opts, bs, sample, n, a_off, A, pivot, tol, st, &c);
            if (r) return r;
            bs.tuned[key] = c;
        }
    }
    std::vector<int> rf(nb), sw(nb);
    for (int p = 0; p < nb; ++p) {
        auto it = opts.autotune ? bs.tuned.find(order_bucket(n[p]) * 16 + (int)pivot) : bs.tuned.end();
        rf[p] = (it != bs.tuned.end()) ? it->second.refine : base_refine;
        sw[p] = (it != bs.tuned.end()) ? it->second.sweeps : base_sweeps;
    }
    return batched_core(h, opts, bs, nb, n, a_off, A, w_off, W, v_off, V, pivot, tol, infos, rf.data(), sw.data(),
                        st);
}

extern "C" int pjac_batched_tuning(pjac_handle* h, int bucket, pjac_pivot pivot, int* refine, int* fp32_sweeps,
                                   float* sample_solves_per_s) {
    if (!h || bucket < 0 || bucket > 4) return set_err(PJAC_EINVAL, "bad argument");
    std::lock_guard<std::mutex> lk(g_bmu);
    auto it = g_bstate.find(h);
    if (it == g_bstate.end()) return set_err(PJAC_EINVAL, "no batched call on this handle yet");
    auto c = it->second.tuned.find(bucket * 16 + (int)pivot);
    if (c == it->second.tuned.end()) return set_err(PJAC_EINVAL, "bucket %d not tuned", bucket);
    if (refine) *refine = c->second.refine;
    if (fp32_sweeps) *fp32_sweeps = c->second.sweeps;
    if (sample_solves_per_s) *sample_solves_per_s = c->second.solves_per_s;
    return PJAC_OK;
}

extern "C" int pjac_batched_stage_ms(pjac_handle* h, float* ms) {
    if (!h || !ms) return set_err(PJAC_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(g_bmu);
    auto it = g_bstate.find(h);
    if (it == g_bstate.end() || !it->second.ev_valid)
        return set_err(PJAC_EINVAL, "no batched call outside a stream capture on this handle yet");
    BatchState& bs = it->second;
    cudaError_t e = cudaEventSynchronize(bs.ev[5]);
    if (e != cudaSuccess) return cuda_err(e, "cudaEventSynchronize");
    for (int k = 0; k < 5; ++k) {
        e = cudaEventElapsedTime(&ms[k], bs.ev[k], bs.ev[k + 1]);
        if (e != cudaSuccess) return cuda_err(e, "cudaEventElapsedTime");
    }
    return PJAC_OK;
}
