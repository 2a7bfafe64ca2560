// Split-precision products on the tensor cores (placeholder until the
// tcgen05 kernel lands): reports "not supported" so callers return
// PJAC_ENOTIMPL instead of computing anything else.
#include <cuda_runtime.h>
#include "internal.h"

namespace pjac {
size_t gemm_split_bf16_ws(int, int, int) { return 0; }
cudaError_t gemm_split_bf16(bool, bool, int, int, int, double, const double*, long long, const double*,
                            long long, double, double*, long long, void*, size_t, cudaStream_t) {
    return cudaErrorNotSupported;
}
}  // namespace pjac
