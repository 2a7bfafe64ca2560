// Allocation-free variant of pjac_solve_preconditioned.
//
// Some callers must not allocate device memory while they solve: a process
// that reserves its whole device-memory budget when it starts (a serving or
// real-time process whose own allocator holds all free memory, so a
// cudaMalloc at solve time fails or fragments that budget), or a plug-in
// that runs inside a host application and has no access to the allocator
// that application uses.  pjac_solve_preconditioned_noalloc gives them the
// Jacobi iteration and the readout without any device allocation: the
// scratch it needs beyond the caller's inputs and outputs (the working
// eigenvector matrix, the unsorted diagonal, the sort ranks, the input-check
// flag and the solve record) lives in one file-scope __device__ array of
// fixed size.  Every GPU that loads the library holds that array
// (PJAC_NOALLOC_SCRATCH_BYTES, about 2 MiB) until the process exits.
//
// Host code cannot use the array's name as a device address (in host code it
// is only a host-side stand-in), so the device address is looked up once per
// device with cudaGetSymbolAddress, with that device current, on the first
// call made on that device.  Under CUDA's lazy module loading that lookup is
// also when the array is placed in device memory, and a kernel's first launch
// is when its code is loaded: both take device memory.  So the first call on
// a device does all of it at once -- the lookup and the loading of every
// kernel the entry point launches -- and callers make that first call before
// they reserve the device's memory.
#include <cuda_runtime.h>
#include <cstring>
#include <mutex>
#include "internal.h"

namespace pjac {
int set_err(int code, const char* fmt, ...);
int cuda_err(cudaError_t e, const char* what);
}
using namespace pjac;

namespace {

constexpr size_t kVBytes = (size_t)PJAC_NOALLOC_MAX_N * PJAC_NOALLOC_MAX_N * sizeof(double);
constexpr size_t kWdOff = kVBytes;
constexpr size_t kRankOff = kWdOff + (size_t)PJAC_NOALLOC_MAX_N * sizeof(double);
constexpr size_t kInfoOff = kRankOff + (size_t)PJAC_NOALLOC_MAX_N * sizeof(int);
constexpr size_t kFlagOff = kInfoOff + 256;
static_assert(kFlagOff + 256 <= PJAC_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the array");

static __device__ __align__(256) unsigned char g_noalloc_scratch[PJAC_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up on
// the first call per device).
int scratch_address(void** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) return set_err(PJAC_EINVAL, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress(scratch)");
        // load the kernels this entry point launches (Jacobi, readout, input
        // check, copies) now rather than at their first launch
        e = preload_jacobi_kernels();
        if (e == cudaSuccess) e = preload_gemm_kernels();
        if (e != cudaSuccess) return cuda_err(e, "loading the kernels");
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return PJAC_OK;
}

}  // namespace

extern "C" int pjac_solve_preconditioned_noalloc(double* A1, int n, int lda1, const double* V0, int ldv0,
                                                 pjac_pivot pivot, double tol, double* W, double* V, int ldv,
                                                 pjac_info* info, void* stream) {
    if (!A1 || !W) return set_err(PJAC_EINVAL, "NULL argument");
    if (n < 1) return set_err(PJAC_EINVAL, "n = %d < 1", n);
    if (n > PJAC_NOALLOC_MAX_N)
        return set_err(PJAC_EINVAL, "n = %d exceeds the allocation-free limit of %d (use pjac_solve_preconditioned)",
                       n, PJAC_NOALLOC_MAX_N);
    if (lda1 < n || (V0 && ldv0 < n) || (V && ldv < n)) return set_err(PJAC_EINVAL, "leading dimension < n");
    if (pivot < PJAC_PIVOT_GAP || pivot > PJAC_PIVOT_CYCLIC) return set_err(PJAC_EINVAL, "bad pivot");
    if (!(tol >= 0.0)) return set_err(PJAC_EINVAL, "tol must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    void* base = nullptr;
    int r = scratch_address(&base);
    if (r) return r;
    char* sp = static_cast<char*>(base);
    double* Vw = reinterpret_cast<double*>(sp);
    double* Wd = reinterpret_cast<double*>(sp + kWdOff);
    int* rank = reinterpret_cast<int*>(sp + kRankOff);
    DevInfo* dinfo = reinterpret_cast<DevInfo*>(sp + kInfoOff);
    int* flag = reinterpret_cast<int*>(sp + kFlagOff);
    cudaError_t e;
#define NK(call) do { e = (call); if (e != cudaSuccess) return cuda_err(e, #call); } while (0)
    if (n == 1) {
        static const double one = 1.0;
        NK(cudaMemcpyAsync(W, A1, sizeof(double), cudaMemcpyDeviceToDevice, st));
        if (V) NK(cudaMemcpyAsync(V, &one, sizeof(double), cudaMemcpyHostToDevice, st));
        NK(cudaStreamSynchronize(st));
        if (info) {
            memset(info, 0, sizeof(*info));
            info->n = 1;
        }
        return PJAC_OK;
    }
    // input check (the flag is cleared by check_finite before use)
    NK(check_finite(A1, lda1, n, flag, st));
    int hflag = 0;
    NK(cudaMemcpyAsync(&hflag, flag, sizeof(int), cudaMemcpyDeviceToHost, st));
    NK(cudaStreamSynchronize(st));
    if (hflag & 1) return set_err(PJAC_EINVAL, "input contains NaN or Inf");
    if (hflag & 2) return set_err(PJAC_EINVAL, "input is not exactly symmetric");
    if (V0) NK(copy_f64(V0, ldv0, Vw, n, n, n, st));
    else NK(set_identity(Vw, n, n, st));
    pjac_opts o;
    pjac_default_opts(&o);
    JacArgs a;
    a.A = A1;
    a.lda = lda1;
    a.V = Vw;
    a.ldv = n;
    a.Wd = Wd;
    a.n = n;
    a.pivot = (int)pivot;
    a.stop = (int)o.stop;
    a.tol = tol;
    a.max_rot = 50LL * n * (n - 1) / 2;
    a.check_every = n;
    a.budget_ns = (long long)(o.time_budget_s * 1e9);
    a.info = dinfo;
    a.seed = o.seed;
    int P = jacobi_auto_cluster(n);
    while (P > 1 && (n + P - 1) / P < 8) P >>= 1;
    NK(launch_jacobi(a, P, st));
    NK(launch_readout(Wd, Vw, n, n, W, V, ldv, rank, st));
    DevInfo d;
    NK(cudaMemcpyAsync(&d, dinfo, sizeof(d), cudaMemcpyDeviceToHost, st));
    NK(cudaStreamSynchronize(st));
#undef NK
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
    }
    return d.status == PJAC_OK ? PJAC_OK
                               : set_err(d.status, "solve ended with status %d after %lld rotations", d.status,
                                         (long long)d.rotations);
}
