// Device-side bounds checks of the bounds-checked build of the library (nvcc -DRFF_CHECK,
// built beside the ordinary library as librff_admm_check.so).
//
// At a global access a kernel tests
//   RFF_IN(i, n)           0 <= i < n: element i of a buffer (or layout) of n elements,
//   RFF_SPAN(i, k, n)      elements i .. i+k-1 all inside [0, n),
//   RFF_TMA_X(x)           a TMA box's innermost coordinate on a 16-byte boundary (every
//                          tensor map of this library holds 2-byte elements: x % 8 == 0),
// and skips the access when the test fails, after counting the failure in the record of its
// translation unit (the first failure's source line, index and bound are kept).  A skipped
// TMA copy never completes its barrier: the bounded wait on that barrier then gives up and
// sets the kernel's error word, so a failed check ends as an error status, not a fault.
// rff_check_report reads and clears the records of every unit.
//
// In the ordinary build every test is the constant true, and neither the record nor any
// instruction of the tests exists.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace rff {

struct CheckHit {
  unsigned long long count;   // failed tests since the record was last cleared
  long long line, index, bound;
};

#ifdef RFF_CHECK

static __device__ CheckHit g_check_hit;   // one per translation unit

static __device__ __noinline__ bool check_failed(long long i, long long n, int line) {
  if (atomicAdd(&g_check_hit.count, 1ull) == 0ull) {
    g_check_hit.line = line;
    g_check_hit.index = i;
    g_check_hit.bound = n;
  }
  return false;
}

static __device__ __forceinline__ bool check_in(long long i, long long n, int line) {
  return (i >= 0 && i < n) ? true : check_failed(i, n, line);
}

static __device__ __forceinline__ bool check_span(long long i, long long k, long long n, int line) {
  return (i >= 0 && k >= 0 && i + k <= n) ? true : check_failed(i + k - 1, n, line);
}

#define RFF_IN(i, n) ::rff::check_in((long long)(i), (long long)(n), __LINE__)
#define RFF_SPAN(i, k, n) ::rff::check_span((long long)(i), (long long)(k), (long long)(n), __LINE__)
#define RFF_TMA_X(x) (((x) & 7) == 0 ? true : ::rff::check_failed((long long)(x), 8, __LINE__))

// host side: read this unit's record into *h and clear it (the caller synchronises first)
#define RFF_CHECK_UNIT(name)                                                        \
  cudaError_t check_collect_##name(CheckHit* h) {                                   \
    cudaError_t e = cudaMemcpyFromSymbol(h, g_check_hit, sizeof(CheckHit));         \
    if (e != cudaSuccess) return e;                                                 \
    const CheckHit zero{};                                                          \
    return cudaMemcpyToSymbol(g_check_hit, &zero, sizeof(CheckHit));                \
  }

#else

#define RFF_IN(i, n) true
#define RFF_SPAN(i, k, n) true
#define RFF_TMA_X(x) true
#define RFF_CHECK_UNIT(name)                                                        \
  cudaError_t check_collect_##name(CheckHit* h) {                                   \
    *h = CheckHit{};                                                                \
    return cudaSuccess;                                                             \
  }

#endif

}  // namespace rff
