// FP64 arithmetic peak of the device, measured: the denominator of the
// roofline of the FP64-bound kernels (the Jacobi iteration, the FP32
// diagonaliser's refinement).  A grid of several CTAs per SM runs eight
// independent fused multiply-add chains per thread; the rate is
// 2 * 8 * iterations * threads / time.
#include <cuda_runtime.h>
#include "internal.h"

namespace pjac {

__global__ void __launch_bounds__(256) dfma_probe_kernel(double* out, long long iters, double a, double b) {
    double x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = 1.0 + 1e-3 * (threadIdx.x + u);
    for (long long it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < 8; ++u) x[u] = __fma_rn(x[u], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int u = 0; u < 8; ++u) s += x[u];
    if (s == 12345.678) out[blockIdx.x] = s;   // keeps the chains live
}

}  // namespace pjac

extern "C" int pjac_probe_fp64(double* tflops, void* stream) {
    using namespace pjac;
    if (!tflops) return PJAC_EINVAL;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) != cudaSuccess) return PJAC_ECUDA;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double* out = nullptr;
    if (cudaMallocAsync(&out, sizeof(double) * sms * 8, st) != cudaSuccess) return PJAC_ENOMEM;
    const int blocks = sms * 8, threads = 256;
    const long long iters = 4096;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    dfma_probe_kernel<<<blocks, threads, 0, st>>>(out, iters, 0.9999999, 1e-9);   // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < 5; ++r) dfma_probe_kernel<<<blocks, threads, 0, st>>>(out, iters, 0.9999999, 1e-9);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(out, st);
    if (e != cudaSuccess) return PJAC_ECUDA;
    const double flops = 5.0 * 2.0 * 8.0 * (double)iters * blocks * threads;
    *tflops = flops / (ms * 1e-3) / 1e12;
    return PJAC_OK;
}
