// Tensor-core regeneration passes (placeholder until the tcgen05 kernels land).
#include "tc.h"

namespace rff {
cudaError_t tc_write_z(const TcView&, int64_t, int64_t, int64_t, int64_t, float*, int64_t) { return cudaErrorNotSupported; }
cudaError_t tc_pass1(const TcView&, float*) { return cudaErrorNotSupported; }
cudaError_t tc_pass2(const TcView&, const __nv_bfloat16*, const __nv_bfloat16*, int64_t, float*, int) {
  return cudaErrorNotSupported;
}
cudaError_t tc_predict(const TcView&, const __nv_bfloat16*, const __nv_bfloat16*, int64_t, const __nv_bfloat16*,
                       const __nv_bfloat16*, float*) {
  return cudaErrorNotSupported;
}
}  // namespace rff
