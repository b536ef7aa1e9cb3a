// Shared device helpers of the GB300 solver: Philox4x32-10, the range-reduced
// cosine of the feature map, BF16 hi/lo splitting, and the slot layout that
// every kernel indexes.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "check.cuh"

namespace rff {

// Rows and features live in "slot" space: every row block i (Sec. 3, n_i rows)
// starts at a multiple of SLOT, and so does every column block j (s_j features).
// Tiles therefore never straddle two blocks, and every tensor-memory copy that
// starts at a block boundary is 16-byte aligned.  Padding slots hold zeros.
constexpr int SLOT = 128;

__host__ __device__ inline int64_t round_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }
__host__ __device__ inline int64_t ceil_div(int64_t x, int64_t a) { return (x + a - 1) / a; }

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3",
// SC'11: ten rounds of two 32x32->64-bit multiplies with Weyl-sequence key bumps.
struct U4 {
  uint32_t x, y, z, w;
};

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

__host__ __device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = mulhi32(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = mulhi32(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
  }
  return c;
}

// u = ((w >> 8) + 0.5) 2^-24: 2^24 equally spaced points strictly inside (0, 1),
// exact in float64.
__host__ __device__ __forceinline__ double uniform01(uint32_t w) {
  return ((double)(w >> 8) + 0.5) * (1.0 / 16777216.0);
}

// ------------------------------------------------------------------ cosine
// cos(x) for the feature map z = sqrt(2/D) cos(w.x + b).  Range reduction by
// Cody-Waite with a two-term pi (x = k pi + r, |r| <= pi/2, the products k*pi
// fused into FMAs), cos(x) = (-1)^k cos(r), and cos(r) as a polynomial in
// s = r^2 of degree 5 whose coefficients were fitted for this library by
// iteratively reweighted least squares (Lawson's algorithm) on [0, (pi/2)^2]
// (fit_cos_poly.py beside this file).  Fit error 2.2e-10; float32 evaluation
// error <= 1.2e-7 on [-pi/2, pi/2].
__device__ __forceinline__ float cos_rr(float x) {
  const float inv_pi = 0.318309886183790672f;
  const float pi_hi = 3.14159274101257324f;       // float32 nearest to pi
  const float pi_lo = -8.74227765734758577e-08f;  // pi - pi_hi
  const float k = rintf(x * inv_pi);
  float r = fmaf(-k, pi_hi, x);
  r = fmaf(-k, pi_lo, r);
  const float s = r * r;
  float p = -2.605149518331018e-07f;
  p = fmaf(p, s, 2.476016197761055e-05f);
  p = fmaf(p, s, -0.0013888361863791943f);
  p = fmaf(p, s, 0.04166663810610771f);
  p = fmaf(p, s, -0.5f);
  p = fmaf(p, s, 1.0f);
  return (static_cast<int>(k) & 1) ? -p : p;
}

// 2^E cos(x), bit for bit 2^E cos_rr(x), with fewer instructions for the tensor-core
// epilogues (where the cosine's instruction count, not the tensor pipe, bounds the small-d
// workloads): k = rint(x / pi) by adding and subtracting 1.5 2^23 to the rounded quotient
// (exact for |x / pi| < 2^22) instead of a rounding and a float-to-integer conversion on the
// transcendental unit, the parity of k read from the low mantissa bit of the biased sum, the
// sign applied by flipping the sign bit, and 2^E folded into the polynomial's coefficients
// (scaling by a power of two commutes with every rounding of the evaluation).
template <int E>
__device__ __forceinline__ float cos_rr_pow2(float x) {
  constexpr float S = (float)(1u << E);
  const float inv_pi = 0.318309886183790672f;
  const float pi_hi = 3.14159274101257324f;
  const float pi_lo = -8.74227765734758577e-08f;
  const float magic = 12582912.f;   // 1.5 2^23
  const float biased = __fadd_rn(__fmul_rn(x, inv_pi), magic);   // not contracted: rint of the rounded quotient
  const float k = __fsub_rn(biased, magic);
  float r = fmaf(-k, pi_hi, x);
  r = fmaf(-k, pi_lo, r);
  const float s = r * r;
  float p = -2.605149518331018e-07f * S;
  p = fmaf(p, s, 2.476016197761055e-05f * S);
  p = fmaf(p, s, -0.0013888361863791943f * S);
  p = fmaf(p, s, 0.04166663810610771f * S);
  p = fmaf(p, s, -0.5f * S);
  p = fmaf(p, s, 1.0f * S);
  return __int_as_float(__float_as_int(p) ^ (__float_as_int(biased) << 31));
}

// ------------------------------------------------------------------ BF16 split
// x = hi + lo + O(2^-17 |x|): hi = bf16(x), lo = bf16(x - hi).
__device__ __forceinline__ void split_bf16(float x, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(x);
  lo = __float2bfloat16_rn(x - __bfloat162float(hi));
}

// ------------------------------------------------------------------ scaled FP16 split
// The X.G operands: x * scale (scale a power of two, so the product is exact) =
// hi + lo + O(2^-22 |x * scale|) with hi = fp16(x scale), lo = fp16(x scale - hi).
// The scale keeps |x scale| <= 2^8 (far from the FP16 maximum, 65504) while values
// far below the largest keep an absolute error of at most 2^-25 in scaled units.
__device__ __forceinline__ void split_f16(float x, float scale, __half& hi, __half& lo) {
  const float xs = x * scale;
  hi = __float2half_rn(xs);
  lo = __float2half_rn(xs - __half2float(hi));
}

// Scale of the FP16 split of a matrix whose largest |entry| is maxabs: the power of two s
// with maxabs * s in [128, 256) (1 when maxabs is 0), and its inverse.  Computed on the
// device from a maximum that an earlier kernel reduced, so producers and consumers of a
// split agree without a round trip to the host.
__device__ __forceinline__ int f16_scale_exp(float maxabs) {
  if (!(maxabs > 0.f)) return 0;
  int e;
  frexpf(maxabs, &e);                 // maxabs = f 2^e, f in [0.5, 1)
  return 8 - max(e, -100);
}
__device__ __forceinline__ float f16_scale(float maxabs) { return ldexpf(1.f, f16_scale_exp(maxabs)); }
__device__ __forceinline__ float f16_inv_scale(float maxabs) { return ldexpf(1.f, -f16_scale_exp(maxabs)); }

// Fixed scale of the FP16 split of cosines (|cos| <= 1) in the chained products
constexpr float COS_SCALE = 128.f;

// f * 2^k as an FP64 number, built from the exponent and significand fields with integer
// instructions and selects, no branches (this part's FP64 pipe, conversions included, runs at
// 1/64 of the FP32 rate).  Exact for zero and normal f when the result is a normal double;
// subnormal f and results below the normal range give a signed zero, results above it a
// signed infinity.
__device__ __forceinline__ double f32_to_f64_scaled(float f, int k) {
  const uint32_t b = __float_as_uint(f);
  const int e = (int)((b >> 23) & 0xffu);
  const int ed = e + (1023 - 127) + k;
  const uint64_t sign = (uint64_t)(b & 0x80000000u) << 32;
  uint64_t bits = sign | ((uint64_t)(uint32_t)ed << 52) | ((uint64_t)(b & 0x7fffffu) << 29);
  bits = (e == 0 || ed <= 0) ? sign : bits;
  bits = ed >= 2047 ? (sign | 0x7ff0000000000000ull) : bits;
  return __longlong_as_double((long long)bits);
}

// hi + lo += x with the rounding error of the addition kept in lo (Knuth's TwoSum, every
// operation rounded separately: no contraction into FMAs)
__device__ __forceinline__ void two_sum_into(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bb = __fsub_rn(s, hi);
  lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb)));
  hi = s;
}

}  // namespace rff
