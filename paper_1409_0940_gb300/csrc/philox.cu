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
//   Fastfood map (blocks of d' = 2^p >= d features, block beta = k / d', row i = k mod d'):
//     V = (1/(sigma sqrt d')) S H diag(g) P H diag(B) per block, H Walsh-Hadamard (Sylvester)
//     B[beta, j]  counter (beta, j, 3, 0), word 0: -1 if its top bit is set
//     g[beta, m]  counter (beta, m, 4, 0): Box-Muller normal of words 0, 1 (the cos one)
//     P           Fisher-Yates from the identity, i = d'-1 .. 1: j = (w (i + 1)) >> 32 for word 0
//                 w of counter (beta, i, 5, 0), swap pi[i], pi[j]; (P y)[m] = y[pi(m)]
//     S[k]        |n| / |g|, n the d' normals of counters (k, q, 6, 0), q < d'/2 (both of a pair)
//     b[k]        as for the Fourier map
#include "common.cuh"
#include "internal.h"

namespace rff {

// map 0 (random Fourier): g / sigma; map 1 (random Laplace): 1 / (2 sigma^2 g^2)
__device__ __forceinline__ float from_normal(double g, double sigma, int map) {
  return map == 1 ? (float)(1.0 / (2.0 * sigma * sigma * g * g)) : (float)(g / sigma);
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
  if (q == 0 && b) b[kk] = map == 1 ? 0.f : phase(k, k0, k1);
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
  const float ph = (map != 1 && k >= 0 && (q == 0 || has_bias_col)) ? phase((uint32_t)k, k0, k1) : 0.f;
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

// ---- Fastfood
__device__ __forceinline__ double normal_cos(const U4& w) {
  const double two_pi = 6.283185307179586;
  return sqrt(-2.0 * log(uniform01(w.x))) * cos(two_pi * uniform01(w.y));
}

template <int NT>
__device__ __forceinline__ double block_sum_d(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int o = NT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// One CTA per block beta: signs, normals, |g| and the permutation (Fisher-Yates by one thread)
__global__ void __launch_bounds__(256) k_fastfood_blocks(uint32_t k0, uint32_t k1, int dp, float* __restrict__ Bt,
                                                       double* __restrict__ gt, int32_t* __restrict__ perm,
                                                       double* __restrict__ gnorm) {
  __shared__ double red[256];
  const uint32_t beta = blockIdx.x;
  double acc = 0.0;
  for (int j = threadIdx.x; j < dp; j += 256) {
    const U4 wb = philox4x32_10(U4{beta, (uint32_t)j, 3u, 0u}, k0, k1);
    Bt[(int64_t)beta * dp + j] = (wb.x >> 31) ? -1.f : 1.f;
    const double g = normal_cos(philox4x32_10(U4{beta, (uint32_t)j, 4u, 0u}, k0, k1));
    gt[(int64_t)beta * dp + j] = g;
    acc += g * g;
    perm[(int64_t)beta * dp + j] = j;
  }
  acc = block_sum_d<256>(acc, red);
  if (threadIdx.x == 0) {
    gnorm[beta] = sqrt(acc);
    int32_t* pb = perm + (int64_t)beta * dp;
    for (int i = dp - 1; i > 0; --i) {
      const uint32_t w = philox4x32_10(U4{beta, (uint32_t)i, 5u, 0u}, k0, k1).x;
      const int j = (int)(((uint64_t)w * (uint64_t)(i + 1)) >> 32);
      const int32_t t = pb[i];
      pb[i] = pb[j];
      pb[j] = t;
    }
  }
}

// One CTA per feature slot: row i of V_beta = c B .* (H v), v[pi(m)] = H[i, m] g[m], by one
// in-place Walsh-Hadamard transform of length d' in float64 (shared memory); then b.
// maxbits receives max |V| (float bits).
__global__ void __launch_bounds__(256) k_fastfood_rows(uint32_t k0, uint32_t k1, double sigma, int64_t d, int64_t ld,
                                                     int dp, const int32_t* __restrict__ feat_of_slot,
                                                     const float* __restrict__ Bt, const double* __restrict__ gt,
                                                     const int32_t* __restrict__ perm,
                                                     const double* __restrict__ gnorm, float* __restrict__ Gt,
                                                     float* __restrict__ bias, unsigned* __restrict__ maxbits) {
  extern __shared__ double ff_v[];
  __shared__ double red[256];
  const int64_t p = blockIdx.x;
  const int32_t k = feat_of_slot[p];
  if (k < 0) {
    for (int64_t j = threadIdx.x; j < ld; j += 256) Gt[p * ld + j] = 0.f;
    if (threadIdx.x == 0 && bias) bias[p] = 0.f;
    return;
  }
  const int64_t beta = k / dp;
  const int i = (int)(k % dp);
  for (int m = threadIdx.x; m < dp; m += 256) {
    const double h = (__popc(i & m) & 1) ? -1.0 : 1.0;
    ff_v[perm[beta * dp + m]] = h * gt[beta * dp + m];
  }
  __syncthreads();
  for (int h = 1; h < dp; h *= 2) {
    for (int t = threadIdx.x; t < dp / 2; t += 256) {
      const int i1 = (t / h) * 2 * h + (t % h), i2 = i1 + h;
      const double a = ff_v[i1], b = ff_v[i2];
      ff_v[i1] = a + b;
      ff_v[i2] = a - b;
    }
    __syncthreads();
  }
  // the row length: a chi(d') draw
  double s2 = 0.0;
  for (int q = threadIdx.x; q < max(dp / 2, 1); q += 256) {
    const U4 w = philox4x32_10(U4{(uint32_t)k, (uint32_t)q, 6u, 0u}, k0, k1);
    const double r = sqrt(-2.0 * log(uniform01(w.x))), t = 6.283185307179586 * uniform01(w.y);
    const double a = r * cos(t), b = r * sin(t);
    s2 += a * a + (2 * q + 1 < dp ? b * b : 0.0);
  }
  s2 = block_sum_d<256>(s2, red);
  const double c = sqrt(s2) / (gnorm[beta] * sigma * sqrt((double)dp));
  float mx = 0.f;
  for (int64_t j = threadIdx.x; j < ld; j += 256) {
    const float v = j < d ? (float)(c * (double)Bt[beta * dp + j] * ff_v[j]) : 0.f;
    Gt[p * ld + j] = v;
    mx = fmaxf(mx, fabsf(v));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0 && maxbits && mx > 0.f) atomicMax(maxbits, __float_as_uint(mx));
  if (threadIdx.x == 0 && bias) bias[p] = phase((uint32_t)k, k0, k1);
}

// FP16 hi/lo split of rows of Gt scaled by gscale, with b in column bias_col (>= 0)
__global__ void k_split_g_bias(const float* __restrict__ Gt, int64_t n, int64_t ld, const float* __restrict__ bias,
                               int64_t bias_col, float gscale, __half* __restrict__ hi, __half* __restrict__ lo) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n * ld) return;
  const int64_t r = t / ld, c = t % ld;
  split_f16(c == bias_col ? bias[r] : Gt[t], gscale, hi[t], lo[t]);
}

size_t fastfood_table_bytes(int64_t D, int dp) {
  const int64_t nb = ceil_div(D, dp);
  return (size_t)nb * dp * (sizeof(float) + sizeof(double) + sizeof(int32_t)) + (size_t)nb * sizeof(double) + 1024;
}

cudaError_t launch_fastfood_params(uint64_t seed, double sigma, int64_t d, int64_t ld, int64_t D, int64_t nslots,
                                   const int32_t* feat_of_slot, float* Gt, float* bias, unsigned* maxbits,
                                   void* tables, cudaStream_t st) {
  const int dp = fastfood_dim(d);
  if (dp > 4096) return cudaErrorInvalidValue;
  const int64_t nb = ceil_div(D, dp);
  char* base = static_cast<char*>(tables);
  double* gt = reinterpret_cast<double*>(base);
  double* gnorm = gt + nb * dp;
  float* Bt = reinterpret_cast<float*>(gnorm + nb);
  int32_t* perm = reinterpret_cast<int32_t*>(Bt + nb * dp);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  k_fastfood_blocks<<<(unsigned)nb, 256, 0, st>>>(k0, k1, dp, Bt, gt, perm, gnorm);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || nslots <= 0) return e;
  k_fastfood_rows<<<(unsigned)nslots, 256, (size_t)dp * sizeof(double), st>>>(k0, k1, sigma, d, ld, dp, feat_of_slot,
                                                                           Bt, gt, perm, gnorm, Gt, bias, maxbits);
  return cudaGetLastError();
}

cudaError_t launch_split_g_bias(const float* Gt, int64_t n, int64_t ld, const float* bias, int64_t bias_col,
                                float gscale, __half* hi, __half* lo, cudaStream_t st) {
  if (n * ld <= 0) return cudaSuccess;
  k_split_g_bias<<<(unsigned)ceil_div(n * ld, 256), 256, 0, st>>>(Gt, n, ld, bias, bias_col, gscale, hi, lo);
  return cudaGetLastError();
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
