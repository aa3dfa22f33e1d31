// Tensor-core (tcgen05) form of the gathered GEMM: not built yet.
#include "fmm_internal.h"

namespace fmm {
cudaError_t gemm_tc(const fmm_ctx *, const GemmCall &, int, cudaStream_t) { return cudaErrorNotSupported; }
cudaError_t tc_upload_operators(fmm_ctx *) { return cudaErrorNotSupported; }
void tc_free(fmm_ctx *) {}
}  // namespace fmm
