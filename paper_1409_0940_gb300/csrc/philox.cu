// Philox4x32-10 generation of the random Fourier feature parameters (Sec. 4:
// omega kept implicit as the state of a pseudo-random generator; the generator
// itself is Salmon et al., SC'11).
//
// Stream layout (identical on every device and independent of the block grid):
//   key            (seed mod 2^32, seed >> 32)
//   G[r, k]        counter (k, r/4, 0, 0); words 0,1 -> Box-Muller pair for rows
//                  4q, 4q+1 (cos, sin); words 2,3 -> rows 4q+2, 4q+3
//   b[k]           counter (k, 0, 1, 0), word 0
//   block mask     counter (b, k, 2, 0), word 0: block b = i C + j active in iteration k
//                  of the stochastic variant iff (w >> 8) < floor(p 2^24)
//   uniform        ((w >> 8) + 0.5) 2^-24 in float64
//   G = float32(sqrt(-2 ln u1) {cos,sin}(2 pi u2) / sigma), b = float32(pi u)
//   random Laplace map: W = float32(1 / (2 sigma^2 g^2)) from the same standard normals
//   g (a Levy(0, 1/(2 sigma^2)) draw), b = 0
#include "common.cuh"
#include "internal.h"

namespace rff {

// map 0 (random Fourier): g / sigma; map 1 (random Laplace): 1 / (2 sigma^2 g^2)
__device__ __forceinline__ float from_normal(double g, double sigma, int map) {
  return map ? (float)(1.0 / (2.0 * sigma * sigma * g * g)) : (float)(g / sigma);
}

__device__ __forceinline__ void gauss4(uint32_t k, uint32_t q, uint32_t k0, uint32_t k1, double sigma,
                                       float g[4], int map = 0) {
  const U4 w = philox4x32_10(U4{k, q, 0u, 0u}, k0, k1);
  const double two_pi = 6.283185307179586;  // float64 nearest to 2 pi
  const double r0 = sqrt(-2.0 * log(uniform01(w.x)));
  const double t0 = two_pi * uniform01(w.y);
  const double r1 = sqrt(-2.0 * log(uniform01(w.z)));
  const double t1 = two_pi * uniform01(w.w);
  g[0] = from_normal(r0 * cos(t0), sigma, map);
  g[1] = from_normal(r0 * sin(t0), sigma, map);
  g[2] = from_normal(r1 * cos(t1), sigma, map);
  g[3] = from_normal(r1 * sin(t1), sigma, map);
}

__device__ __forceinline__ float phase(uint32_t k, uint32_t k0, uint32_t k1) {
  const U4 w = philox4x32_10(U4{k, 0u, 1u, 0u}, k0, k1);
  return (float)(uniform01(w.x) * 3.141592653589793);
}

__global__ void k_philox_raw(const uint32_t* __restrict__ ctr, uint32_t k0, uint32_t k1, int64_t n,
                             uint32_t* __restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const U4 c{ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
  const U4 o = philox4x32_10(c, k0, k1);
  out[4 * i] = o.x;
  out[4 * i + 1] = o.y;
  out[4 * i + 2] = o.z;
  out[4 * i + 3] = o.w;
}

// API layout: G (d x nk row-major), one thread per (row group q, feature).
__global__ void k_params_rowmajor(uint32_t k0, uint32_t k1, double sigma, int64_t d, int64_t k_lo, int64_t nk,
                                  float* __restrict__ G, float* __restrict__ b, int map) {
  const int64_t kk = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t q = blockIdx.y;
  if (kk >= nk) return;
  const uint32_t k = (uint32_t)(k_lo + kk);
  float g[4];
  gauss4(k, (uint32_t)q, k0, k1, sigma, g, map);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int64_t r = 4 * q + e;
    if (r < d) G[r * nk + kk] = g[e];
  }
  if (q == 0 && b) b[kk] = map ? 0.f : phase(k, k0, k1);
}

// Slot layout: Gt (D_slots x ld, feature-major) in float32 and/or split BF16.
// Padding features and the columns d..ld-1 are written as zeros.
__global__ void k_params_slots(uint32_t k0, uint32_t k1, double sigma, int64_t d, int64_t ld, int64_t nslots,
                               const int32_t* __restrict__ feat_of_slot, float* __restrict__ Gt,
                               __half* __restrict__ Ghi, __half* __restrict__ Glo, float gscale,
                               float* __restrict__ bias, int64_t bias_col, int map) {
  const int64_t nq = ld / 4;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nslots * nq) return;
  const int64_t p = t / nq, q = t % nq;
  const int32_t k = feat_of_slot[p];
  float g[4] = {0.f, 0.f, 0.f, 0.f};
  if (k >= 0 && 4 * q < d) gauss4((uint32_t)k, (uint32_t)q, k0, k1, sigma, g, map);
  const bool has_bias_col = bias_col >= 4 * q && bias_col < 4 * q + 4;
  const float ph = (!map && k >= 0 && (q == 0 || has_bias_col)) ? phase((uint32_t)k, k0, k1) : 0.f;
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int64_t r = 4 * q + e;
    const float v = (r < d) ? g[e] : 0.f;
    if (Gt) Gt[p * ld + r] = v;
    if (Ghi) {
      // the FP16 copies may carry the phase b in column bias_col (the input then
      // carries a column of ones there), so the product X G already includes b
      __half hi, lo;
      split_f16(r == bias_col ? ph : v, gscale, hi, lo);
      Ghi[p * ld + r] = hi;
      Glo[p * ld + r] = lo;
    }
  }
  if (q == 0 && bias) bias[p] = ph;
}

// One CTA: the mask of iteration *ctr, then the counter moves on (so a captured iteration
// replays with the right k)
__global__ void k_block_mask(uint32_t k0, uint32_t k1, uint32_t thr, int nb, int64_t* __restrict__ ctr,
                             uint8_t* __restrict__ mask) {
  const int64_t k = *ctr;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    const U4 w = philox4x32_10(U4{(uint32_t)b, (uint32_t)k, 2u, 0u}, k0, k1);
    mask[b] = (w.x >> 8) < thr ? 1 : 0;
  }
  __syncthreads();
  if (threadIdx.x == 0) *ctr = k + 1;
}

cudaError_t launch_block_mask(uint64_t seed, uint32_t thr, int nblocks, int64_t* ctr, uint8_t* mask,
                              cudaStream_t st) {
  if (nblocks <= 0) return cudaSuccess;
  k_block_mask<<<1, 256, 0, st>>>((uint32_t)seed, (uint32_t)(seed >> 32), thr, nblocks, ctr, mask);
  return cudaGetLastError();
}

cudaError_t launch_philox_raw(const uint32_t* ctr, uint64_t seed, int64_t n, uint32_t* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_philox_raw<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(ctr, (uint32_t)seed, (uint32_t)(seed >> 32), n, out);
  return cudaGetLastError();
}

cudaError_t launch_params_rowmajor(uint64_t seed, double sigma, int64_t d, int64_t k_lo, int64_t nk, float* G,
                                   float* b, cudaStream_t st, int map) {
  if (nk <= 0 || d <= 0) return cudaSuccess;
  dim3 grid((unsigned)ceil_div(nk, 128), (unsigned)ceil_div(d, 4));
  k_params_rowmajor<<<grid, 128, 0, st>>>((uint32_t)seed, (uint32_t)(seed >> 32), sigma, d, k_lo, nk, G, b, map);
  return cudaGetLastError();
}

cudaError_t launch_params_slots(uint64_t seed, double sigma, int64_t d, int64_t ld, int64_t nslots,
                                const int32_t* feat_of_slot, float* Gt, __half* Ghi, __half* Glo, float gscale,
                                float* bias, int64_t bias_col, cudaStream_t st, int map) {
  const int64_t total = nslots * (ld / 4);
  if (total <= 0) return cudaSuccess;
  k_params_slots<<<(unsigned)ceil_div(total, 256), 256, 0, st>>>((uint32_t)seed, (uint32_t)(seed >> 32), sigma,
                                                                   d, ld, nslots, feat_of_slot, Gt, Ghi, Glo, gscale, bias,
                                                                   bias_col, map);
  return cudaGetLastError();
}

}  // namespace rff
