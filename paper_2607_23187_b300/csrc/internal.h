// Internal declarations shared by the CUDA translation units of libpjac.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/pjac.h"

namespace pjac {

// Device-side report of one Jacobi solve (written by the kernel).
struct DevInfo {
    long long rotations;
    long long sweeps;      // cyclic: sweeps started
    double off;            // off(A) at exit (absolute)
    double normf;          // ||A1||_F at entry
    double max_score;      // last selected score
    int status;            // pjac_status
    int n;
    long long steps;       // selection steps (rotations, except for the multi-pivot variant)
};

struct JacArgs {
    double* A;             // working matrix, overwritten (column-major == row-major, symmetric)
    long long lda;
    double* V;             // accumulated V (column-major), may be null
    long long ldv;
    double* Wd;            // out: final diagonal (unsorted), n
    int n;
    int pivot;             // pjac_pivot
    int stop;              // pjac_stop
    double tol;
    long long max_rot;
    long long check_every;
    long long budget_ns;
    DevInfo* info;
    unsigned long long seed;   // PJAC_PIVOT_RANDOM
    int* K = nullptr;      // optional: screening key of every entry (n x n, ld ldk), kept current
    long long ldk = 0;
};

// One problem of the batched form, as the device sees it.  All matrices
// have leading dimension n.
struct BatchDesc {
    const double* Ain;     // caller's A (read only)
    double* A;             // A1 working copy, overwritten by the iteration
    double* V;             // Q, then the accumulated V
    double* T;             // product temporaries
    double* Y;
    double* Z;             // refinement rotation
    double* Wd;            // unsorted diagonal
    float* A32;            // FP32 diagonaliser state (used when n > 128)
    float* Q32;            // FP32 eigenvector estimate Q0
    double* Wout;          // caller's W of this problem
    double* Vout;          // caller's V of this problem (may be null)
    DevInfo* info;
    int n;
    int refine;            // refinement steps (stage 2b)
    int sweeps32;          // FP32 sweep cap (stage 1)
    int pad;
};

// jacobi.cu
cudaError_t launch_jacobi(const JacArgs& a, int cluster, cudaStream_t st);
int jacobi_auto_cluster(int n);
cudaError_t launch_jacobi_batched(const BatchDesc* d_desc, int nb, const int* d_order,
                                  int* d_counter, int pivot, int stop, double tol,
                                  long long max_rot_per_n2, long long budget_ns, int max_n,
                                  int ctas, unsigned long long seed, cudaStream_t st);
cudaError_t launch_readout(const double* Wd, const double* Vws, long long ldvws, int n,
                           double* W, double* V, long long ldv, int* rank_ws, cudaStream_t st);
cudaError_t launch_readout_batched(const BatchDesc* d_desc, int nb, int max_n, cudaStream_t st);
cudaError_t launch_info_batched(const BatchDesc* d_desc, int nb, pjac_info* infos, cudaStream_t st);
cudaError_t launch_info_single(const DevInfo* src, pjac_info* dst, cudaStream_t st);
int solve_async_dev(pjac_handle* h, const double* A, int n, int lda, pjac_pivot pivot, double tol, double* W,
                    double* V, int ldv, pjac_info* dinfo, cudaStream_t st);

// gemm.cu (transform and Newton--Schulz)
cudaError_t gemm_f64(bool ta, bool tb, int m, int n, int k, double alpha, const double* A,
                     long long lda, const double* B, long long ldb, double beta, double* C,
                     long long ldc, cudaStream_t st);
cudaError_t symmetrize(double* A, long long lda, int n, cudaStream_t st);
cudaError_t copy_f32_to_f64(const float* src, long long lds, double* dst, long long ldd, int n,
                            cudaStream_t st);
cudaError_t copy_f64(const double* src, long long lds, double* dst, long long ldd, int m, int n,
                     cudaStream_t st);
cudaError_t set_identity(double* dst, long long ldd, int n, cudaStream_t st);
cudaError_t copy_f64_to_f32(const double* src, long long lds, float* dst, long long ldd, int n, cudaStream_t st);
// first-order refinement (pjac_opts.refine_steps): Z = I + s D built from A1
constexpr double REFINE_TAU = 0.01;
constexpr double REFINE_MAX_ROWSUM = 0.25;
constexpr int REFINE_NS_STEPS = 5;
cudaError_t refine_build(const double* A1, long long lda1, int n, double tau, double* Z,
                         unsigned long long* maxsum, double limit, cudaStream_t st);
cudaError_t refine_r(double* Y, const double* E, int n, cudaStream_t st);
cudaError_t refine_ns(double* E, const double* R, const double* T, int n, cudaStream_t st);
cudaError_t refine_a1(double* A1, long long lda1, const double* T, const double* Y, int n, cudaStream_t st);
cudaError_t three_i_minus(double* Y, long long ldy, int n, cudaStream_t st);
cudaError_t check_finite(const double* A, long long lda, int n, int* d_flag, cudaStream_t st);

// Split-precision products on the tensor cores (BF16 slices, FP32 accumulation).
// sym (m == n, op(A) op(B) symmetric in exact arithmetic): only the tiles on
// and above the diagonal are computed; entry (i, j), i <= j, is written to
// (i, j) and (j, i), so C comes out exactly symmetric.
cudaError_t gemm_split_bf16(bool ta, bool tb, int m, int n, int k, double alpha, const double* A,
                            long long lda, const double* B, long long ldb, double beta, double* C,
                            long long ldc, void* ws, size_t ws_bytes, cudaStream_t st, bool sym = false);
size_t gemm_split_bf16_ws(int m, int n, int k);          // 0: k too large for the exact split product
int* gemm_split_bf16_errflag(void* ws);                 // device status word (0 = ok), sticky until cleared
int gemm_split_bf16_launches(int m, int n, int k, bool sym = false);   // kernel launches per product
// Host-only plan of a product (info: b, S, units, splits, CTAs, pairs; pairs
// as (s, t, unit, split) quadruples, at most cap); -1 when k is too large.
int gemm_split_bf16_plan(int m, int n, int k, bool sym, int sms, int* info, int* pairs, int cap);
cudaError_t gemm_split_bf16_fold_status(void* ws, DevInfo* info, cudaStream_t st);

// diag32.cu: FP32 parallel-order Jacobi diagonalisation of fl32(A); Q0 out (ld n)
// max_grid > 0 caps the cooperative grid (so that it can start beside other work)
cudaError_t diag_fp32(const double* A, long long lda, int n, float* Q0, float* ws, int* iws,
                      int max_sweeps, int max_grid, cudaStream_t st);
size_t diag_fp32_ws_floats(int n);
cudaError_t fp32_sweeps_done(float* ws, int n, int* diag, int* refine);
// refinement of an FP32 eigenbasis on B = X^T fl32(A) X; Dout: X (I + D)
cudaError_t refine_fp32(const double* B, int n, float* Dout, float* ws, int max_sweeps, int max_grid,
                        cudaStream_t st);
// serving lanes: cap of the cooperative grids of a handle's preconditioner
void handle_set_coop_cap(pjac_handle* h, int max_grid);
cudaError_t round_to_fp32(const double* src, long long lds, double* dst, long long ldd, int n, cudaStream_t st);
cudaError_t add_f64(double* X, long long ldx, const double* Y, long long ldy, int n, cudaStream_t st);

// multi.cu: the multi-pivot variant (one CTA per problem)
cudaError_t launch_jacobi_multi(const JacArgs& a, int K, double ratio, long long* steps_out, cudaStream_t st);
cudaError_t preload_multi_kernels();

// svd.cu: readout of the one-sided Jacobi SVD
cudaError_t check_finite_rect(const double* A, long long lda, int m, int n, int* d_flag, cudaStream_t st);
cudaError_t launch_svd_readout(const double* BF, long long ldbf, int m, const double* Vw, long long ldvw, int n,
                               double* sig, int* rank, double* S, double* U, long long ldu, double* V,
                               long long ldv, cudaStream_t st);
cudaError_t preload_svd_kernels();
cudaError_t launch_svd_onesided(double* B, int m, int n, double* V, double* G, int pivot, double tol,
                                long long max_rot, unsigned long long seed, long long budget_ns, DevInfo* info,
                                cudaStream_t st);
cudaError_t launch_os_readout(const double* G, const double* Brot, int m, const double* Vw, int n, double* sig,
                              int* rank, double* S, double* U, long long ldu, double* V, long long ldv,
                              cudaStream_t st);
cudaError_t preload_os_kernels();

// Kernel preloading (one function per source file), for the serving form.
cudaError_t preload_batched_kernels();
cudaError_t preload_diag32_kernels();
cudaError_t preload_gemm_kernels();
cudaError_t preload_tc_kernels();
cudaError_t preload_jacobi_kernels();

int batched_launch_count(int no_precondition);

}  // namespace pjac
