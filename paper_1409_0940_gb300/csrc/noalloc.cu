// Scoring that allocates no device memory.
//
// Some callers cannot call cudaMalloc at the moment they need scores: serving loops
// whose device memory is handed out entirely by another allocator's pool (a cudaMalloc
// of their own fails, or fragments that pool), and loops that must not take the
// device-wide synchronisation an allocation or a free can cost in the middle of a
// request.  rff_admm_predict_noalloc serves them: it runs the same kernels as
// rff_admm_predict, but its scratch (the slot-padded queries in FP32, their FP16 hi/lo
// split and the padded scores) lives in one fixed array in device global memory that
// the library defines once, so a call allocates nothing.  The price: every GPU that
// loads the library holds the array (32 MiB) until the process exits, a call can score
// at most as many queries as fit in it, and all calls share it (calls that overlap on
// the GPU race on it).  A call synchronises the handle's stream.
#include <mutex>
#include <string>

#include "../../include/rff_admm.h"

namespace rff {
rff_status predict_into_scratch(rff_admm_t h, const float* Xq, int64_t q, float* scores, void* scratch,
                                size_t scratch_bytes);
}  // namespace rff

namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;   // 32 MiB per device

// The scratch itself.  In host code the name stands for a host-side shadow, not a
// device address: the device address is looked up once per device below.
static __device__ __align__(256) unsigned char g_predict_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up on first use.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_predict_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" rff_status rff_admm_predict_noalloc(rff_admm_t h, const float* Xq, int64_t q, float* scores) {
  if (!h) return RFF_EINVAL;
  void* p = nullptr;
  const cudaError_t e = scratch_address(&p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return RFF_ECUDA;
  }
  return rff::predict_into_scratch(h, Xq, q, scores, p, kScratchBytes);
}
