// C ABI of libpjac: handle, argument checks, and the single-problem pipeline
// (Sec. 2.1 preconditioner, then Algorithm 1, then the readout).
#include <cuda_runtime.h>
#include <cstdarg>
#include <cstdio>
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>
#include "internal.h"

using namespace pjac;

namespace pjac {
static thread_local char g_err[512] = "";

int set_err(int code, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_err(cudaError_t e, const char* what) {
    return set_err(PJAC_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}
}  // namespace pjac

#define CK(call)                                                     \
    do {                                                             \
        cudaError_t e_ = (call);                                     \
        if (e_ != cudaSuccess) return pjac::cuda_err(e_, #call);    \
    } while (0)

// Grow-only device buffer.  Growth is stream-ordered (cudaFreeAsync /
// cudaMallocAsync on the caller's stream), so it never waits for work of
// other streams.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    int ensure(size_t need, cudaStream_t st) {
        if (need <= bytes) return PJAC_OK;
        if (p) cudaFreeAsync(p, st);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMallocAsync(&p, need, st);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return set_err(PJAC_ENOMEM, "cudaMalloc(%zu bytes) failed: %s", need, cudaGetErrorString(e));
        }
        bytes = need;
        return PJAC_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
};

struct pjac_handle {
    pjac_opts opts;
    int device;
    DevBuf ws;          // main workspace
    DevBuf tcws;        // tensor-core product workspace
    DevBuf svdws;       // SVD: the m x n rotated matrix
    int coop_cap = 0;   // cap of the cooperative grids (0: the whole GPU)
    int last_n = 0;     // order of the last workspace layout
    // refinement steps of the last solve: order, steps applied, their
    // Newton--Schulz steps in all (for pjac_solve_launch_count)
    int ref_n = 0, ref_done = 0, ref_ns = 0;
    // set while a solve must not wait on the host (the server's lanes): the
    // refinement then takes the largest Newton--Schulz count instead of
    // reading the correction's size back
    bool no_host_wait = false;
    cudaEvent_t ev[4];
    std::mutex mu;
};

extern "C" void pjac_default_opts(pjac_opts* o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->stop = PJAC_STOP_OFFDIAG;
    o->tol = 1e-15;
    o->max_rotations = 0;
    o->check_every = 0;
    o->transform = PJAC_TRANSFORM_SPLIT_BF16;
    o->ns_steps = 3;
    o->cluster_size = 0;
    o->time_budget_s = 600.0;
    o->no_precondition = 0;
    o->seed = 0;
    o->refine_steps = 0;
    o->fp32_sweeps = 0;
    o->multi_pivot = 0;
    o->multi_ratio = 0.0;
    o->autotune = 1;
}

static int validate_opts(const pjac_opts* o) {
    if (o->stop != PJAC_STOP_OFFDIAG && o->stop != PJAC_STOP_LIBOUND)
        return set_err(PJAC_EINVAL, "opts.stop must be PJAC_STOP_OFFDIAG or PJAC_STOP_LIBOUND");
    if (!(o->tol >= 0.0) || o->tol != o->tol) return set_err(PJAC_EINVAL, "opts.tol must be >= 0");
    if (o->max_rotations < 0 || o->check_every < 0) return set_err(PJAC_EINVAL, "negative budget");
    if (o->transform != PJAC_TRANSFORM_SPLIT_BF16 && o->transform != PJAC_TRANSFORM_FP64)
        return set_err(PJAC_EINVAL, "opts.transform invalid");
    if (o->ns_steps < 0 || o->ns_steps > 10) return set_err(PJAC_EINVAL, "opts.ns_steps must be in [0,10]");
    if (o->cluster_size < 0 || o->cluster_size > 16 || (o->cluster_size & (o->cluster_size - 1)))
        return set_err(PJAC_EINVAL, "opts.cluster_size must be 0 or a power of two <= 16");
    if (o->no_precondition != 0 && o->no_precondition != 1)
        return set_err(PJAC_EINVAL, "opts.no_precondition must be 0 or 1");
    if (o->refine_steps < 0 || o->refine_steps > 8) return set_err(PJAC_EINVAL, "opts.refine_steps must be in [0,8]");
    if (o->fp32_sweeps < 0 || o->fp32_sweeps > 100) return set_err(PJAC_EINVAL, "opts.fp32_sweeps must be in [0,100]");
    if (o->multi_pivot < 0 || o->multi_pivot > 64) return set_err(PJAC_EINVAL, "opts.multi_pivot must be in [0,64]");
    if (!(o->multi_ratio >= 0.0 && o->multi_ratio <= 1.0))
        return set_err(PJAC_EINVAL, "opts.multi_ratio must be in [0,1]");
    if (o->autotune != 0 && o->autotune != 1) return set_err(PJAC_EINVAL, "opts.autotune must be 0 or 1");
    return PJAC_OK;
}

extern "C" int pjac_create(pjac_handle** h, const pjac_opts* o) {
    if (!h) return set_err(PJAC_EINVAL, "h is NULL");
    *h = nullptr;
    pjac_opts d;
    pjac_default_opts(&d);
    if (o) d = *o;
    int r = validate_opts(&d);
    if (r) return r;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    pjac_handle* p = new pjac_handle();
    p->opts = d;
    p->device = dev;
    for (int k = 0; k < 4; ++k) {
        cudaError_t e = cudaEventCreate(&p->ev[k]);
        if (e != cudaSuccess) {
            delete p;
            return cuda_err(e, "cudaEventCreate");
        }
    }
    *h = p;
    return PJAC_OK;
}

void pjac_batched_release(const void* h);

namespace pjac {
void handle_set_coop_cap(pjac_handle* h, int max_grid) { h->coop_cap = max_grid; }
int handle_opts(const pjac_handle* h, pjac_opts* o) {
    *o = h->opts;
    return PJAC_OK;
}
}  // namespace pjac

extern "C" int pjac_destroy(pjac_handle* h) {
    if (!h) return PJAC_OK;
    cudaDeviceSynchronize();
    pjac_batched_release(h);
    h->ws.release();
    h->tcws.release();
    h->svdws.release();
    for (int k = 0; k < 4; ++k) cudaEventDestroy(h->ev[k]);
    delete h;
    return PJAC_OK;
}

extern "C" int pjac_set_opts(pjac_handle* h, const pjac_opts* o) {
    if (!h || !o) return set_err(PJAC_EINVAL, "NULL argument");
    int r = validate_opts(o);
    if (r) return r;
    h->opts = *o;
    return PJAC_OK;
}

static int check_dims(int n, int ld, const char* name) {
    if (n < 1 || n > PJAC_MAX_N) return set_err(PJAC_EINVAL, "n = %d out of range [1, %d]", n, PJAC_MAX_N);
    if (ld < n) return set_err(PJAC_EINVAL, "%s = %d < n = %d", name, ld, n);
    return PJAC_OK;
}

static int check_input(pjac_handle* h, const double* A, long long lda, int n, cudaStream_t st, int* flag) {
    CK(check_finite(A, lda, n, flag, st));
    int hflag = 0;
    CK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    (void)h;
    if (hflag & 1) return set_err(PJAC_EINVAL, "input contains NaN or Inf");
    if (hflag & 2) return set_err(PJAC_EINVAL, "input is not exactly symmetric");
    return PJAC_OK;
}

// Workspace layout of one single-problem solve (doubles unless noted).
struct SolveWs {
    double* A1;    // n x n
    double* Vw;    // n x n
    double* T;     // n x n
    double* Y;     // n x n
    double* Wd;    // n
    float* Q0;     // n x n
    float* d32;    // diag_fp32 workspace
    int* rank;     // n
    int* flag;     // 1
    DevInfo* info; // 1
    double* Z;     // n x n (refinement)
    unsigned long long* maxsum;   // 1 (refinement)
    int* K;        // n x n screening keys of the Jacobi iteration
};

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

static int layout_ws(pjac_handle* h, int n, SolveWs* w, cudaStream_t st) {
    size_t nn = (size_t)n * n;
    h->last_n = n;
    const size_t nz = h->opts.refine_steps > 0 ? nn * 8 : 8;
    size_t sz[13] = {nn * 8, nn * 8, nn * 8, nn * 8, (size_t)n * 8, nn * 4,
                     diag_fp32_ws_floats(n) * 4, (size_t)n * 4, 16, sizeof(DevInfo), nz, 8, nn * 4};
    size_t tot = 0;
    for (size_t s : sz) tot += align256(s);
    int r = h->ws.ensure(tot, st);
    if (r) return r;
    char* p = static_cast<char*>(h->ws.p);
    void* ptrs[13];
    for (int k = 0; k < 13; ++k) {
        ptrs[k] = p;
        p += align256(sz[k]);
    }
    w->A1 = (double*)ptrs[0];
    w->Vw = (double*)ptrs[1];
    w->T = (double*)ptrs[2];
    w->Y = (double*)ptrs[3];
    w->Wd = (double*)ptrs[4];
    w->Q0 = (float*)ptrs[5];
    w->d32 = (float*)ptrs[6];
    w->rank = (int*)ptrs[7];
    w->flag = (int*)ptrs[8];
    w->info = (DevInfo*)ptrs[9];
    w->Z = (double*)ptrs[10];
    w->maxsum = (unsigned long long*)ptrs[11];
    w->K = (int*)ptrs[12];
    return PJAC_OK;
}

// Tensor-core products: size the workspace for m x n x k products and clear
// their device status word.  Called before a sequence of products.
static int tc_prepare(pjac_handle* h, int m, int n, int k, cudaStream_t st) {
    if (h->opts.transform != PJAC_TRANSFORM_SPLIT_BF16) return PJAC_OK;
    size_t need = gemm_split_bf16_ws(m, n, k);
    if (need == 0)
        return set_err(PJAC_ENOTIMPL, "split-BF16 product not available for inner dimension %d", k);
    int r = h->tcws.ensure(need, st);
    if (r) return r;
    CK(cudaMemsetAsync(gemm_split_bf16_errflag(h->tcws.p), 0, sizeof(int), st));
    return PJAC_OK;
}

// Device status of the tensor-core products since tc_prepare (synchronises).
static int tc_status(pjac_handle* h, cudaStream_t st) {
    if (h->opts.transform != PJAC_TRANSFORM_SPLIT_BF16) return PJAC_OK;
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, gemm_split_bf16_errflag(h->tcws.p), sizeof(int), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (flag) return set_err(PJAC_ETIMEOUT, "tensor-core product pipeline timed out (code %d)", flag);
    return PJAC_OK;
}

// C = alpha op(A) op(B) + beta C with the product chosen by the options
// (the split-BF16 workspace was prepared by tc_prepare for this shape).
// sym (m == n): the caller knows op(A) op(B) to be symmetric in exact
// arithmetic; C comes out exactly symmetric (the split product computes the
// tiles on and above the diagonal and mirrors them, the FP64 product is
// symmetrised).
static int product_mnk(pjac_handle* h, bool ta, bool tb, int m, int n, int k, double alpha, const double* A,
                       long long lda, const double* B, long long ldb, double beta, double* C, long long ldc,
                       cudaStream_t st, bool sym = false) {
    if (h->opts.transform == PJAC_TRANSFORM_SPLIT_BF16) {
        cudaError_t e = gemm_split_bf16(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, h->tcws.p,
                                        h->tcws.bytes, st, sym);
        if (e == cudaErrorNotSupported) {
            cudaGetLastError();
            return set_err(PJAC_ENOTIMPL, "split-BF16 tensor-core product not available for this shape");
        }
        CK(e);
        return PJAC_OK;
    }
    CK(gemm_f64(ta, tb, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, st));
    if (sym) CK(symmetrize(C, ldc, n, st));
    return PJAC_OK;
}

static int product(pjac_handle* h, bool ta, bool tb, int n, double alpha, const double* A, long long lda,
                   const double* B, long long ldb, double beta, double* C, long long ldc, cudaStream_t st) {
    return product_mnk(h, ta, tb, n, n, n, alpha, A, lda, B, ldb, beta, C, ldc, st);
}

// A product whose exact value is symmetric (X^T X, X^T (S X) with S symmetric).
static int product_sym(pjac_handle* h, bool ta, bool tb, int n, double alpha, const double* A, long long lda,
                       const double* B, long long ldb, double beta, double* C, long long ldc, cudaStream_t st) {
    return product_mnk(h, ta, tb, n, n, n, alpha, A, lda, B, ldb, beta, C, ldc, st, true);
}

// X <- X (3I - X^T X) / 2, steps times (Newton--Schulz; Sec. 2.1 names it
// as one way to restore orthogonality to working precision).
static int newton_schulz(pjac_handle* h, double* Q, long long ldq, int n, int steps, SolveWs& w,
                         cudaStream_t st) {
    for (int it = 0; it < steps; ++it) {
        int r = product_sym(h, true, false, n, 1.0, Q, ldq, Q, ldq, 0.0, w.Y, n, st);
        if (r) return r;
        CK(three_i_minus(w.Y, n, n, st));
        r = product(h, false, false, n, 0.5, Q, ldq, w.Y, n, 0.0, w.T, n, st);
        if (r) return r;
        CK(copy_f64(w.T, n, Q, ldq, n, n, st));
    }
    return PJAC_OK;
}

// The low-precision spectral decomposition of Sec. 2.1 (u_l = single, as in
// Sec. 4) into Q (FP64 storage, ld ldq): an FP32 eigenbasis X of fl32(A).
// The parallel-order FP32 Jacobi pass leaves its basis off by the rounding of
// its many rotation layers, in the eigenvectors and in orthogonality (each
// FP32 rotation moves column norms by a rounding unit).  So: X = fl64(Q0)
// made orthogonal (Newton--Schulz), then a refinement pass on
// B = X^T fl32(A) X that diagonalises it further, X <- X (I + D).  With
// fp32_refine == false that pass is left out.
static int lowprec_basis(pjac_handle* h, const double* A, int n, long long lda, double* Q, long long ldq,
                         SolveWs& w, cudaStream_t st, bool fp32_refine = true) {
    CK(diag_fp32(A, lda, n, w.Q0, w.d32, nullptr, h->opts.fp32_sweeps > 0 ? h->opts.fp32_sweeps : 40, h->coop_cap,
                 st));
    CK(copy_f32_to_f64(w.Q0, n, Q, ldq, n, st));                        // X = fl64(Q0)
    if (!fp32_refine) return PJAC_OK;
    int r = newton_schulz(h, Q, ldq, n, 2, w, st);
    if (r) return r;
    CK(round_to_fp32(A, lda, w.Y, n, n, st));                             // Y = fl32(A)
    r = product(h, false, false, n, 1.0, w.Y, n, Q, ldq, 0.0, w.T, n, st);    // T = fl32(A) X
    if (r) return r;
    r = product_sym(h, true, false, n, 1.0, Q, ldq, w.T, n, 0.0, w.Y, n, st); // B = X^T T, symmetric
    if (r) return r;
    const int rsw = h->opts.fp32_sweeps > 0 && h->opts.fp32_sweeps < 20 ? h->opts.fp32_sweeps : 20;
    CK(refine_fp32(w.Y, n, w.Q0, w.d32, rsw, h->coop_cap, st));                        // D
    CK(copy_f32_to_f64(w.Q0, n, w.T, n, n, st));
    r = product(h, false, false, n, 1.0, Q, ldq, w.T, n, 0.0, w.Y, n, st);    // X D
    if (r) return r;
    CK(add_f64(Q, ldq, w.Y, n, n, st));                                   // X (I + D)
    return PJAC_OK;
}

// One first-order refinement step of (A1, Q) (pjac_opts.refine_steps, an
// extension beyond the paper): Z = I + E with E = s D from A1, made
// orthogonal by Newton--Schulz, then A1 <- Z^T A1 Z (symmetrised) and
// Q <- Q Z.  Everything is written in terms of the small E, so that each
// product's error is relative to |E| rather than to |Z| ~ 1:
//   R = E^T E + E + E^T,  E <- E - R/2 - E R/2              (Newton--Schulz)
//   T = A1 E,  A1 <- A1 + (T + T^T + E^T T),  Q <- Q + Q E.
// Newton--Schulz steps that make Z = I + E orthogonal (E antisymmetric,
// ||E||_2 <= rho <= 1/4, bounded by its largest absolute row sum): the defect
// Z^T Z - I = E^T E starts at most rho^2 and a step maps r to
// 3/4 r^2 + 1/4 r^3 <= r^2, so k steps leave rho^(2^(k+1)); the least k >= 1
// with rho^(2^(k+1)) <= 2^-56, at most REFINE_NS_STEPS.
static int refine_ns_count(double rho) {
    if (!(rho > 0.0)) return 0;
    const double bits = -std::log2(rho);
    int k = 1;
    while (k < REFINE_NS_STEPS && std::ldexp(1.0, k + 1) * bits < 56.0) ++k;
    return k;
}

static int refine_step(pjac_handle* h, double* A1, long long lda1, double* Q, long long ldq, int n, SolveWs& w,
                       cudaStream_t st) {
    double* E = w.Z;
    CK(refine_build(A1, lda1, n, REFINE_TAU, E, w.maxsum, REFINE_MAX_ROWSUM, st));
    int ns = REFINE_NS_STEPS;
    if (!h->no_host_wait) {
        // the largest absolute row sum of D before scaling: the step count of
        // the orthogonalisation (one small copy; the solve is not captured)
        unsigned long long bits = 0;
        CK(cudaMemcpyAsync(&bits, w.maxsum, sizeof(bits), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        double rowsum = 0.0;
        std::memcpy(&rowsum, &bits, sizeof(rowsum));
        ns = refine_ns_count(std::min(rowsum, REFINE_MAX_ROWSUM));
        if (ns == 0) return PJAC_OK;   // D = 0: nothing to refine
    }
    // (without the read-back: the largest count, and a zero correction goes
    // through the steps unchanged, E = 0 staying 0)
    h->ref_done++;
    h->ref_ns += ns;
    int r;
    for (int it = 0; it < ns; ++it) {
        r = product_sym(h, true, false, n, 1.0, E, n, E, n, 0.0, w.Y, n, st);     // Y = E^T E
        if (r) return r;
        CK(refine_r(w.Y, E, n, st));                                               // R = Y + E + E^T
        r = product(h, false, false, n, -0.5, E, n, w.Y, n, 0.0, w.T, n, st);     // T = -E R / 2
        if (r) return r;
        CK(refine_ns(E, w.Y, w.T, n, st));                                         // E <- E - R/2 + T
    }
    r = product(h, false, false, n, 1.0, A1, lda1, E, n, 0.0, w.T, n, st);       // T = A1 E
    if (r) return r;
    r = product_sym(h, true, false, n, 1.0, E, n, w.T, n, 0.0, w.Y, n, st);      // Y = E^T A1 E
    if (r) return r;
    CK(refine_a1(A1, lda1, w.T, w.Y, n, st));
    CK(symmetrize(A1, lda1, n, st));
    r = product(h, false, false, n, 1.0, Q, ldq, E, n, 0.0, w.T, n, st);         // T = Q E
    if (r) return r;
    CK(add_f64(Q, ldq, w.T, n, n, st));                                          // Q <- Q + T
    return PJAC_OK;
}

// Sec. 2.1 into workspace: Q (ld n) and A1 (ld n).  Records ev[0..2].
static int precondition_ws(pjac_handle* h, const double* A, int n, long long lda, const float* Q0,
                           double* Q, long long ldq, double* A1, long long lda1, SolveWs& w, cudaStream_t st) {
    int rp = tc_prepare(h, n, n, n, st);
    if (rp) return rp;
    CK(cudaEventRecord(h->ev[0], st));
    if (Q0) {
        // X = fl64(Q0) as given
        CK(copy_f32_to_f64(Q0, n, Q, ldq, n, st));
    } else {
        // after the final reorthogonalisation below, fl32(A) = Q Lambda Q^T
        // to FP32 accuracy
        int r = lowprec_basis(h, A, n, lda, Q, ldq, w, st);
        if (r) return r;
    }
    int r = newton_schulz(h, Q, ldq, n, h->opts.ns_steps, w, st);
    if (r) return r;
    CK(cudaEventRecord(h->ev[1], st));
    // A1 = Q^T (A Q), symmetrised
    r = product(h, false, false, n, 1.0, A, lda, Q, ldq, 0.0, w.T, n, st);
    if (r) return r;
    r = product_sym(h, true, false, n, 1.0, Q, ldq, w.T, n, 0.0, A1, lda1, st);
    if (r) return r;
    h->ref_n = n;
    h->ref_done = h->ref_ns = 0;
    for (int k = 0; k < h->opts.refine_steps; ++k) {
        r = refine_step(h, A1, lda1, Q, ldq, n, w, st);
        if (r) return r;
    }
    CK(cudaEventRecord(h->ev[2], st));
    return PJAC_OK;
}

extern "C" int pjac_precondition(pjac_handle* h, const double* A, int n, int lda, const float* Q0,
                                 double* Q, int ldq, double* A1, int lda1, void* stream) {
    if (!h || !A || !Q || !A1) return set_err(PJAC_EINVAL, "NULL argument");
    int r = check_dims(n, lda, "lda");
    if (!r) r = check_dims(n, ldq, "ldq");
    if (!r) r = check_dims(n, lda1, "lda1");
    if (r) return r;
    std::lock_guard<std::mutex> lk(h->mu);
    cudaStream_t st = (cudaStream_t)stream;
    SolveWs w;
    r = layout_ws(h, n, &w, st);
    if (r) return r;
    r = check_input(h, A, lda, n, st, w.flag);
    if (r) return r;
    r = precondition_ws(h, A, n, lda, Q0, Q, ldq, A1, lda1, w, st);
    if (r) return r;
    return tc_status(h, st);
}

extern "C" int pjac_eig_lowprec(pjac_handle* h, const double* A, int n, int lda, float* Q0, int ldq0,
                                void* stream) {
    if (!h || !A || !Q0) return set_err(PJAC_EINVAL, "NULL argument");
    int r = check_dims(n, lda, "lda");
    if (!r) r = check_dims(n, ldq0, "ldq0");
    if (r) return r;
    std::lock_guard<std::mutex> lk(h->mu);
    cudaStream_t st = (cudaStream_t)stream;
    SolveWs w;
    r = layout_ws(h, n, &w, st);
    if (r) return r;
    r = check_input(h, A, lda, n, st, w.flag);
    if (r) return r;
    r = tc_prepare(h, n, n, n, st);
    if (r) return r;
    r = lowprec_basis(h, A, n, lda, w.Vw, n, w, st);
    if (r) return r;
    CK(copy_f64_to_f32(w.Vw, n, Q0, ldq0, n, st));
    r = tc_status(h, st);
    if (r) return r;
    CK(cudaStreamSynchronize(st));
    return PJAC_OK;
}

extern "C" int pjac_product(pjac_handle* h, int transa, int transb, int m, int n, int k, double alpha,
                            const double* A, int lda, const double* B, int ldb, double beta, double* C, int ldc,
                            void* stream) {
    if (!h || !A || !B || !C) return set_err(PJAC_EINVAL, "NULL argument");
    if (m < 1 || n < 1 || k < 1 || m > PJAC_MAX_N || n > PJAC_MAX_N || k > PJAC_MAX_N)
        return set_err(PJAC_EINVAL, "m, n, k = %d, %d, %d out of range [1, %d]", m, n, k, PJAC_MAX_N);
    if ((transa != 0 && transa != 1) || (transb != 0 && transb != 1))
        return set_err(PJAC_EINVAL, "transa and transb must be 0 or 1");
    if (lda < (transa ? k : m) || ldb < (transb ? n : k) || ldc < m)
        return set_err(PJAC_EINVAL, "leading dimension too small");
    std::lock_guard<std::mutex> lk(h->mu);
    cudaStream_t st = (cudaStream_t)stream;
    int r = tc_prepare(h, m, n, k, st);
    if (r) return r;
    r = product_mnk(h, transa != 0, transb != 0, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, st);
    if (r) return r;
    return tc_status(h, st);
}

extern "C" int pjac_product_symmetric(pjac_handle* h, int transa, int transb, int n, int k, double alpha,
                                      const double* A, int lda, const double* B, int ldb, double beta, double* C,
                                      int ldc, void* stream) {
    if (!h || !A || !B || !C) return set_err(PJAC_EINVAL, "NULL argument");
    if (n < 1 || k < 1 || n > PJAC_MAX_N || k > PJAC_MAX_N)
        return set_err(PJAC_EINVAL, "n, k = %d, %d out of range [1, %d]", n, k, PJAC_MAX_N);
    if ((transa != 0 && transa != 1) || (transb != 0 && transb != 1))
        return set_err(PJAC_EINVAL, "transa and transb must be 0 or 1");
    if (lda < (transa ? k : n) || ldb < (transb ? n : k) || ldc < n)
        return set_err(PJAC_EINVAL, "leading dimension too small");
    std::lock_guard<std::mutex> lk(h->mu);
    cudaStream_t st = (cudaStream_t)stream;
    int r = tc_prepare(h, n, n, k, st);
    if (r) return r;
    r = product_mnk(h, transa != 0, transb != 0, n, n, k, alpha, A, lda, B, ldb, beta, C, ldc, st, true);
    if (r) return r;
    return tc_status(h, st);
}

// The device checks its time budget against the GPU's global nanosecond
// timer (%globaltimer), so the budget is wall time whatever the SM clock.
static long long budget_ns(const pjac_opts& o) {
    double s = o.time_budget_s > 0 ? o.time_budget_s : 600.0;
    return (long long)(s * 1e9);
}

static int run_jacobi(pjac_handle* h, double* A1, long long lda1, int n, double* Vw, long long ldvw,
                      pjac_pivot pivot, double tol, double* Wd, DevInfo* dinfo, int* K, cudaStream_t st) {
    JacArgs a;
    a.K = K;
    a.ldk = n;
    a.A = A1;
    a.lda = lda1;
    a.V = Vw;
    a.ldv = ldvw;
    a.Wd = Wd;
    a.n = n;
    a.pivot = (int)pivot;
    a.stop = (int)h->opts.stop;
    a.tol = tol;
    long long pairs = (long long)n * (n - 1) / 2;
    a.max_rot = h->opts.max_rotations > 0 ? h->opts.max_rotations : 50 * pairs;
    a.check_every = h->opts.check_every > 0 ? h->opts.check_every : n;
    a.budget_ns = budget_ns(h->opts);
    a.info = dinfo;
    a.seed = h->opts.seed;
    if (h->opts.multi_pivot >= 2) {
        if (pivot != PJAC_PIVOT_GAP && pivot != PJAC_PIVOT_GREEDY)
            return set_err(PJAC_EINVAL, "the multi-pivot variant needs the gap or the greedy rule");
        if (n > 4096) return set_err(PJAC_EINVAL, "the multi-pivot variant takes n <= 4096 (n = %d)", n);
        CK(launch_jacobi_multi(a, h->opts.multi_pivot, h->opts.multi_ratio, nullptr, st));
        return PJAC_OK;
    }
    int P = h->opts.cluster_size > 0 ? h->opts.cluster_size : jacobi_auto_cluster(n);
    while (P > 1 && (n + P - 1) / P < 8) P >>= 1;
    if ((n + P - 1) / P > 1024) return set_err(PJAC_EINVAL, "n = %d needs a larger cluster", n);
    CK(launch_jacobi(a, P, st));
    return PJAC_OK;
}

static int finish_info(pjac_handle* h, DevInfo* dinfo, pjac_info* info, cudaStream_t st, bool timed) {
    DevInfo d;
    CK(cudaMemcpyAsync(&d, dinfo, sizeof(d), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (info) {
        info->rotations = d.rotations;
        double pairs = 0.5 * (double)d.n * (double)(d.n - 1);
        info->sweeps = d.sweeps > 0 ? (double)d.sweeps : (pairs > 0 ? d.rotations / pairs : 0.0);
        info->off_rel = d.normf > 0 ? d.off / d.normf : 0.0;
        info->max_score = d.max_score;
        info->status = d.status;
        info->n = d.n;
        info->steps = d.steps;
        info->ms_precond = info->ms_transform = info->ms_jacobi = 0.f;
        if (timed) {
            cudaEventElapsedTime(&info->ms_precond, h->ev[0], h->ev[1]);
            cudaEventElapsedTime(&info->ms_transform, h->ev[1], h->ev[2]);
            cudaEventElapsedTime(&info->ms_jacobi, h->ev[2], h->ev[3]);
        }
    }
    return d.status == PJAC_OK ? PJAC_OK
                               : set_err(d.status, "solve ended with status %d after %lld rotations", d.status,
                                         (long long)d.rotations);
}

static int trivial_n1(const double* A, double* W, double* V, cudaStream_t st, pjac_info* info) {
    CK(cudaMemcpyAsync(W, A, sizeof(double), cudaMemcpyDeviceToDevice, st));
    if (V) {
        double one = 1.0;
        CK(cudaMemcpyAsync(V, &one, sizeof(double), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    }
    if (info) {
        memset(info, 0, sizeof(*info));
        info->n = 1;
    }
    return PJAC_OK;
}

static int solve_checks(pjac_handle* h, const double* A, int n, int lda, pjac_pivot pivot, double tol,
                        const double* W, const double* V, int ldv) {
    if (!h || !A || !W) return set_err(PJAC_EINVAL, "NULL argument");
    int r = check_dims(n, lda, "lda");
    if (!r && V) r = check_dims(n, ldv, "ldv");
    if (r) return r;
    if (pivot < PJAC_PIVOT_GAP || pivot > PJAC_PIVOT_RANDOM) return set_err(PJAC_EINVAL, "bad pivot");
    if (!(tol >= 0.0)) return set_err(PJAC_EINVAL, "tol must be >= 0");
    if (h->opts.stop == PJAC_STOP_LIBOUND && pivot != PJAC_PIVOT_GAP)
        return set_err(PJAC_EINVAL, "PJAC_STOP_LIBOUND needs the gap rule");
    return PJAC_OK;
}

// Preconditioner, Jacobi, readout: all enqueued on st, no host round trip.
// Without the preconditioner (opts.no_precondition) Algorithm 1 starts from
// A1 = A and V0 = I.
static int solve_pipeline(pjac_handle* h, const double* A, int n, int lda, pjac_pivot pivot, double tol,
                          double* W, double* V, int ldv, SolveWs& w, cudaStream_t st) {
    int r;
    if (h->opts.no_precondition) {
        CK(cudaEventRecord(h->ev[0], st));
        CK(cudaEventRecord(h->ev[1], st));
        CK(copy_f64(A, lda, w.A1, n, n, n, st));
        CK(set_identity(w.Vw, n, n, st));
        CK(cudaEventRecord(h->ev[2], st));
    } else {
        r = precondition_ws(h, A, n, lda, nullptr, w.Vw, n, w.A1, n, w, st);
        if (r) return r;
    }
    r = run_jacobi(h, w.A1, n, n, w.Vw, n, pivot, tol, w.Wd, w.info, w.K, st);
    if (r) return r;
    CK(launch_readout(w.Wd, w.Vw, n, n, W, V, ldv, w.rank, st));
    if (h->opts.transform == PJAC_TRANSFORM_SPLIT_BF16 && !h->opts.no_precondition)
        CK(gemm_split_bf16_fold_status(h->tcws.p, w.info, st));   // a timed-out product fails the solve
    CK(cudaEventRecord(h->ev[3], st));
    return PJAC_OK;
}

extern "C" int pjac_solve(pjac_handle* h, const double* A, int n, int lda, pjac_pivot pivot, double tol,
                          double* W, double* V, int ldv, pjac_info* info, void* stream) {
    int r = solve_checks(h, A, n, lda, pivot, tol, W, V, ldv);
    if (r) return r;
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 1) return trivial_n1(A, W, V, st, info);
    std::lock_guard<std::mutex> lk(h->mu);
    SolveWs w;
    r = layout_ws(h, n, &w, st);
    if (r) return r;
    r = check_input(h, A, lda, n, st, w.flag);
    if (r) return r;
    r = solve_pipeline(h, A, n, lda, pivot, tol, W, V, ldv, w, st);
    if (r) return r;
    return finish_info(h, w.info, info, st, true);
}

namespace pjac {
// Asynchronous single-problem solve for the serving lanes: the input was
// validated on the host; the report is written to device memory (dinfo)
// by the device.  Nothing here waits for the device.
int solve_async_dev(pjac_handle* h, const double* A, int n, int lda, pjac_pivot pivot, double tol, double* W,
                    double* V, int ldv, pjac_info* dinfo, cudaStream_t st) {
    int r = solve_checks(h, A, n, lda, pivot, tol, W, V, ldv);
    if (r) return r;
    std::lock_guard<std::mutex> lk(h->mu);
    SolveWs w;
    r = layout_ws(h, n, &w, st);
    if (r) return r;
    // nothing in this call waits for the device (the server runs it on the
    // thread that also admits and polls every other request)
    h->no_host_wait = true;
    r = solve_pipeline(h, A, n, lda, pivot, tol, W, V, ldv, w, st);
    h->no_host_wait = false;
    if (r) return r;
    CK(launch_info_single(w.info, dinfo, st));
    return PJAC_OK;
}
}  // namespace pjac

extern "C" int pjac_solve_preconditioned(pjac_handle* h, double* A1, int n, int lda1, const double* V0,
                                         int ldv0, pjac_pivot pivot, double tol, double* W, double* V,
                                         int ldv, pjac_info* info, void* stream) {
    if (!h || !A1 || !W) return set_err(PJAC_EINVAL, "NULL argument");
    int r = check_dims(n, lda1, "lda1");
    if (!r && V0) r = check_dims(n, ldv0, "ldv0");
    if (!r && V) r = check_dims(n, ldv, "ldv");
    if (r) return r;
    if (pivot < PJAC_PIVOT_GAP || pivot > PJAC_PIVOT_RANDOM) return set_err(PJAC_EINVAL, "bad pivot");
    if (!(tol >= 0.0)) return set_err(PJAC_EINVAL, "tol must be >= 0");
    if (h->opts.stop == PJAC_STOP_LIBOUND && pivot != PJAC_PIVOT_GAP)
        return set_err(PJAC_EINVAL, "PJAC_STOP_LIBOUND needs the gap rule");
    cudaStream_t st = (cudaStream_t)stream;
    if (n == 1) return trivial_n1(A1, W, V, st, info);
    std::lock_guard<std::mutex> lk(h->mu);
    SolveWs w;
    r = layout_ws(h, n, &w, st);
    if (r) return r;
    r = check_input(h, A1, lda1, n, st, w.flag);
    if (r) return r;
    CK(cudaEventRecord(h->ev[0], st));
    CK(cudaEventRecord(h->ev[1], st));
    if (V0) {
        CK(copy_f64(V0, ldv0, w.Vw, n, n, n, st));
    } else {
        CK(set_identity(w.Vw, n, n, st));
    }
    CK(cudaEventRecord(h->ev[2], st));
    r = run_jacobi(h, A1, lda1, n, w.Vw, n, pivot, tol, w.Wd, w.info, w.K, st);
    if (r) return r;
    CK(launch_readout(w.Wd, w.Vw, n, n, W, V, ldv, w.rank, st));
    CK(cudaEventRecord(h->ev[3], st));
    return finish_info(h, w.info, info, st, true);
}

extern "C" int pjac_svd(pjac_handle* h, const double* B, int m, int n, int ldb, const float* Vl, int ldvl,
                        pjac_pivot pivot, double tol, double* S, double* U, int ldu, double* V, int ldv,
                        pjac_info* info, void* stream) {
    if (!h || !B || !S) return set_err(PJAC_EINVAL, "NULL argument");
    if (n < 1 || m < n || m > PJAC_MAX_N) return set_err(PJAC_EINVAL, "need 1 <= n <= m <= %d (m = %d, n = %d)",
                                                           PJAC_MAX_N, m, n);
    if (ldb < m || (U && ldu < m) || (V && ldv < n) || (Vl && ldvl < n))
        return set_err(PJAC_EINVAL, "leading dimension too small");
    if (pivot < PJAC_PIVOT_GAP || pivot > PJAC_PIVOT_RANDOM) return set_err(PJAC_EINVAL, "bad pivot");
    if (!(tol >= 0.0)) return set_err(PJAC_EINVAL, "tol must be >= 0");
    if (h->opts.stop == PJAC_STOP_LIBOUND && pivot != PJAC_PIVOT_GAP)
        return set_err(PJAC_EINVAL, "PJAC_STOP_LIBOUND needs the gap rule");
    std::lock_guard<std::mutex> lk(h->mu);
    cudaStream_t st = (cudaStream_t)stream;
    SolveWs w;
    int r = layout_ws(h, n, &w, st);
    if (r) return r;
    r = h->svdws.ensure(align256((size_t)m * n * 8), st);
    if (r) return r;
    double* BF = static_cast<double*>(h->svdws.p);
    CK(check_finite_rect(B, ldb, m, n, w.flag, st));
    {
        int hflag = 0;
        CK(cudaMemcpyAsync(&hflag, w.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (hflag) return set_err(PJAC_EINVAL, "input contains NaN or Inf");
    }
    if (h->opts.transform == PJAC_TRANSFORM_SPLIT_BF16) {
        size_t need = 0;
        const int shapes[3][3] = {{m, n, n}, {n, n, m}, {n, n, n}};
        for (const auto& sh : shapes) {
            size_t b = gemm_split_bf16_ws(sh[0], sh[1], sh[2]);
            if (b == 0) return set_err(PJAC_ENOTIMPL, "split-BF16 product not available for m = %d", m);
            need = need > b ? need : b;
        }
        r = h->tcws.ensure(need, st);
        if (r) return r;
        CK(cudaMemsetAsync(gemm_split_bf16_errflag(h->tcws.p), 0, sizeof(int), st));
    }
    CK(cudaEventRecord(h->ev[0], st));
    // V0: Newton--Schulz of the low-precision right singular vectors
    if (h->opts.no_precondition) {
        CK(set_identity(w.Vw, n, n, st));
    } else {
        if (Vl) {
            CK(copy_f32_to_f64(Vl, ldvl, w.Vw, n, n, st));
        } else {
            // FP32 eigenbasis of G = B^T B (its eigenvectors are B's right
            // singular vectors)
            r = product_mnk(h, true, false, n, n, m, 1.0, B, ldb, B, ldb, 0.0, w.A1, n, st);
            if (r) return r;
            CK(symmetrize(w.A1, n, n, st));
            r = lowprec_basis(h, w.A1, n, n, w.Vw, n, w, st);
            if (r) return r;
        }
        r = newton_schulz(h, w.Vw, n, n, h->opts.ns_steps, w, st);
        if (r) return r;
    }
    CK(cudaEventRecord(h->ev[1], st));
    // B1 = B V0, A = B1^T B1
    r = product_mnk(h, false, false, m, n, n, 1.0, B, ldb, w.Vw, n, 0.0, BF, m, st);
    if (r) return r;
    r = product_mnk(h, true, false, n, n, m, 1.0, BF, m, BF, m, 0.0, w.A1, n, st);
    if (r) return r;
    CK(symmetrize(w.A1, n, n, st));
    h->ref_n = n;
    h->ref_done = h->ref_ns = 0;
    for (int k = 0; k < h->opts.refine_steps; ++k) {
        r = refine_step(h, w.A1, n, w.Vw, n, n, w, st);
        if (r) return r;
    }
    CK(cudaEventRecord(h->ev[2], st));
    r = run_jacobi(h, w.A1, n, n, w.Vw, n, pivot, tol, w.Wd, w.info, w.K, st);
    if (r) return r;
    // the rotated matrix B V, its column norms, the sorted factors
    r = product_mnk(h, false, false, m, n, n, 1.0, B, ldb, w.Vw, n, 0.0, BF, m, st);
    if (r) return r;
    CK(launch_svd_readout(BF, m, m, w.Vw, n, n, w.Wd, w.rank, S, U, ldu, V, ldv, st));
    if (h->opts.transform == PJAC_TRANSFORM_SPLIT_BF16)
        CK(gemm_split_bf16_fold_status(h->tcws.p, w.info, st));
    CK(cudaEventRecord(h->ev[3], st));
    if (!info) return PJAC_OK;
    return finish_info(h, w.info, info, st, true);
}

extern "C" int pjac_svd_onesided(pjac_handle* h, const double* B, int m, int n, int ldb, pjac_pivot pivot,
                                 double tol, double* S, double* U, int ldu, double* V, int ldv, pjac_info* info,
                                 void* stream) {
    if (!h || !B || !S) return set_err(PJAC_EINVAL, "NULL argument");
    if (n < 2 || n > 1024 || m < n || m > PJAC_MAX_N)
        return set_err(PJAC_EINVAL, "need 2 <= n <= 1024 and n <= m <= %d (m = %d, n = %d)", PJAC_MAX_N, m, n);
    if (ldb < m || (U && ldu < m) || (V && ldv < n)) return set_err(PJAC_EINVAL, "leading dimension too small");
    if (pivot != PJAC_PIVOT_GAP_REL && pivot != PJAC_PIVOT_GAP && pivot != PJAC_PIVOT_GREEDY &&
        pivot != PJAC_PIVOT_RANDOM)
        return set_err(PJAC_EINVAL, "pjac_svd_onesided: pivot must be GAP_REL, GAP, GREEDY or RANDOM");
    if (!(tol >= 0.0)) return set_err(PJAC_EINVAL, "tol must be >= 0");
    std::lock_guard<std::mutex> lk(h->mu);
    cudaStream_t st = (cudaStream_t)stream;
    SolveWs w;
    int r = layout_ws(h, n, &w, st);
    if (r) return r;
    r = h->svdws.ensure(align256((size_t)m * n * 8), st);
    if (r) return r;
    double* Bw = static_cast<double*>(h->svdws.p);
    CK(check_finite_rect(B, ldb, m, n, w.flag, st));
    {
        int hflag = 0;
        CK(cudaMemcpyAsync(&hflag, w.flag, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        if (hflag) return set_err(PJAC_EINVAL, "input contains NaN or Inf");
    }
    CK(cudaEventRecord(h->ev[0], st));
    CK(cudaEventRecord(h->ev[1], st));
    CK(copy_f64(B, ldb, Bw, m, m, n, st));
    CK(set_identity(w.Vw, n, n, st));
    CK(cudaEventRecord(h->ev[2], st));
    long long pairs = (long long)n * (n - 1) / 2;
    long long max_rot = h->opts.max_rotations > 0 ? h->opts.max_rotations : 50 * pairs;
    CK(launch_svd_onesided(Bw, m, n, w.Vw, w.A1, (int)pivot, tol, max_rot, h->opts.seed, budget_ns(h->opts),
                           w.info, st));
    CK(launch_os_readout(w.A1, Bw, m, w.Vw, n, w.Wd, w.rank, S, U, ldu, V, ldv, st));
    CK(cudaEventRecord(h->ev[3], st));
    if (!info) return PJAC_OK;
    return finish_info(h, w.info, info, st, true);
}

extern "C" int pjac_fp32_sweeps_done(pjac_handle* h, int* diag, int* refine) {
    if (!h || h->last_n < 1) return set_err(PJAC_EINVAL, "no solve on this handle yet");
    std::lock_guard<std::mutex> lk(h->mu);
    SolveWs w;
    int r = layout_ws(h, h->last_n, &w, 0);
    if (r) return r;
    CK(fp32_sweeps_done(w.d32, h->last_n, diag, refine));
    return PJAC_OK;
}

extern "C" int pjac_solve_launch_count(pjac_handle* h, int n) {
    if (!h || n < 1 || n > PJAC_MAX_N) return -1;
    if (n == 1) return 0;
    // without the preconditioner: input check, copy of A, V0 = I, Jacobi,
    // readout (two kernels)
    if (h->opts.no_precondition) return 6;
    const bool split = h->opts.transform == PJAC_TRANSFORM_SPLIT_BF16;
    const int P = split ? gemm_split_bf16_launches(n, n, n) : 1;   // launches per product
    // launches per symmetric product (the FP64 product is symmetrised after)
    const int Ps = split ? gemm_split_bf16_launches(n, n, n, true) : 2;
    const int ns = h->opts.ns_steps;
    // input check, FP32 diagonaliser, copy to FP64
    int c = 3;
    // Newton--Schulz before the refinement (2 steps) and after it (ns steps):
    // two products (one symmetric), 3I - Y and a copy per step
    c += (2 + ns) * (P + Ps + 2);
    // fl32(A), T = fl32(A) X, B = X^T T (symmetric), refinement, copy, X D, add
    c += 1 + P + Ps + 1 + 1 + P + 1;
    // transform (two products, one symmetric), Jacobi, readout (two kernels)
    c += P + Ps + 1 + 2;
    // refinement steps: build and scale (every step), then for the steps
    // with a nonzero correction its Newton--Schulz steps (two products, one
    // symmetric, and two element-wise steps each), three products (one
    // symmetric), the A1 update, symmetrise, the Q update.  The Newton--Schulz count depends on the
    // correction's size: the handle's last solve of this order gives it,
    // else the largest count is assumed.
    if (h->opts.refine_steps > 0) {
        int done = h->opts.refine_steps, nss = h->opts.refine_steps * REFINE_NS_STEPS;
        if (h->ref_n == n) {
            done = h->ref_done;
            nss = h->ref_ns;
        }
        c += 2 * h->opts.refine_steps + nss * (P + Ps + 2) + done * (2 * P + Ps + 3);
    }
    if (split) c += 1;  // product status folded into the solve record
    return c;
}

extern "C" int pjac_product_launch_count(pjac_handle* h, int m, int n, int k) {
    if (!h || m < 1 || n < 1 || k < 1 || m > PJAC_MAX_N || n > PJAC_MAX_N || k > PJAC_MAX_N) return -1;
    if (h->opts.transform != PJAC_TRANSFORM_SPLIT_BF16) return 1;
    int c = gemm_split_bf16_launches(m, n, k);
    return c > 0 ? c : -1;
}

extern "C" int pjac_product_plan(int m, int n, int k, int symmetric, int sms, int* info, int* pairs,
                                 int pairs_cap) {
    if (!info || m < 1 || n < 1 || k < 1 || m > PJAC_MAX_N || n > PJAC_MAX_N || k > PJAC_MAX_N ||
        (symmetric != 0 && symmetric != 1) || (symmetric && m != n) || pairs_cap < 0 || sms < 0)
        return set_err(PJAC_EINVAL, "invalid product plan query");
    if (gemm_split_bf16_plan(m, n, k, symmetric != 0, sms, info, pairs, pairs_cap) != 0)
        return set_err(PJAC_ENOTIMPL, "split-BF16 product not available for inner dimension %d", k);
    return PJAC_OK;
}

extern "C" const char* pjac_status_string(int s) {
    switch (s) {
        case PJAC_OK: return "PJAC_OK";
        case PJAC_PENDING: return "PJAC_PENDING";
        case PJAC_EINVAL: return "PJAC_EINVAL: invalid argument";
        case PJAC_ENOMEM: return "PJAC_ENOMEM: device allocation failed";
        case PJAC_EAGAIN: return "PJAC_EAGAIN: queue full";
        case PJAC_ENOCONV: return "PJAC_ENOCONV: rotation budget reached";
        case PJAC_ETIMEOUT: return "PJAC_ETIMEOUT: device time budget ran out";
        case PJAC_ECUDA: return "PJAC_ECUDA: CUDA runtime error";
        case PJAC_ENOTIMPL: return "PJAC_ENOTIMPL: not available";
        default: return "unknown status";
    }
}

extern "C" const char* pjac_last_error(void) { return pjac::g_err; }
