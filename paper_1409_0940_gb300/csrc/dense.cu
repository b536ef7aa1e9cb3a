// Batched dense linear algebra on the SIMT pipes: the Gram matrices
// I + Z_ij^T Z_ij of eq. (cache), their FP64 Cholesky factorisation, the cached
// inverse Q_ij = (I + Z_ij^T Z_ij)^-1 (the paper's "Q_ij can be cached"), and the
// per-iteration products with Q_ij and H_ij.
#include "common.cuh"
#include "internal.h"

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <vector>

namespace rff {

namespace {

// ------------------------------------------------------------------ generic GEMM
// D = alpha * op(A) op(B) + beta * Cm for a batch of row-major matrices.
// Tile 64 x 64, 256 threads, 4 x 4 outputs per thread.  Loads are bounds-checked
// so any M, N, K works.  lower_only skips tiles strictly above the diagonal.
template <typename T, int BK>
__global__ void __launch_bounds__(256) k_gemm(const GemmDesc* __restrict__ descs, int transA, int transB, T alpha,
                                              T beta, int lower_only) {
  const GemmDesc g = descs[blockIdx.z];
  const int tm = blockIdx.x, tn = blockIdx.y;
  if (tm * 64 >= g.M || tn * 64 >= g.N) return;
  if (lower_only && tn > tm) return;
  const T* __restrict__ A = static_cast<const T*>(g.A);
  const T* __restrict__ B = static_cast<const T*>(g.B);
  __shared__ T As[BK][64 + 1];
  __shared__ T Bs[BK][64 + 1];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  T acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
  const int m0 = tm * 64, n0 = tn * 64;
  for (int k0 = 0; k0 < g.K; k0 += BK) {
    for (int t = tid; t < 64 * BK; t += 256) {
      int mm, kk;
      if (transA) { mm = t % 64; kk = t / 64; } else { kk = t % BK; mm = t / BK; }
      const int gm = m0 + mm, gk = k0 + kk;
      T v = T(0);
      if (gm < g.M && gk < g.K) v = transA ? A[(int64_t)gk * g.lda + gm] : A[(int64_t)gm * g.lda + gk];
      As[kk][mm] = v;
      int nn, kb;
      if (transB) { kb = t % BK; nn = t / BK; } else { nn = t % 64; kb = t / 64; }
      const int gn = n0 + nn, gkb = k0 + kb;
      T w = T(0);
      if (gn < g.N && gkb < g.K) w = transB ? B[(int64_t)gn * g.ldb + gkb] : B[(int64_t)gkb * g.ldb + gn];
      Bs[kb][nn] = w;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      T a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[k][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[k][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  const T* __restrict__ Cm = static_cast<const T*>(g.Cm);
  T* __restrict__ D = static_cast<T*>(g.D);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= g.N) continue;
      T v = alpha * acc[i][j];
      if (beta != T(0)) v = fma(beta, Cm[(int64_t)gm * g.ldc + gn], v);
      D[(int64_t)gm * g.ldd + gn] = v;
    }
  }
}

// ------------------------------------------------------------------ FP32 NN GEMM
// The per-iteration products x = Q r and r = b - H x: A (M x K) and B (K x N)
// row-major with K-contiguous A rows, N-contiguous B rows; vector loads when the
// tile is interior.  Tile 64 x 64, BK = 32.  descs null: the one product given by value.
__global__ void __launch_bounds__(256) k_gemm_f32_nn(const GemmDesc* __restrict__ descs, const GemmDesc one,
                                                     float alpha, float beta, const uint8_t* __restrict__ bmask) {
  if (bmask && !bmask[blockIdx.z]) return;
  const GemmDesc g = descs ? descs[blockIdx.z] : one;
  const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
  if (m0 >= g.M || n0 >= g.N) return;
  const float* __restrict__ A = static_cast<const float*>(g.A);
  const float* __restrict__ B = static_cast<const float*>(g.B);
  __shared__ __align__(16) float As[32][64 + 4];
  __shared__ __align__(16) float Bs[32][64 + 4];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  // FP32 products summed 32 at a time (acc), each chunk's sum folded into a float-float
  // accumulator (hi, lo) by TwoSum: the error of a K-term dot product is that of one
  // 32-term FP32 sum instead of a K-term one (K = s_j = 4096 for the cached projection)
  float hi[4][4] = {}, lo[4][4] = {};
  for (int k0 = 0; k0 < g.K; k0 += 32) {
    float acc[4][4] = {};
    // A tile: 64 rows x 32 k
    for (int t = tid; t < 64 * 32; t += 256) {
      const int kk = t % 32, mm = t / 32;
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < g.M && gk < g.K) ? A[(int64_t)gm * g.lda + gk] : 0.f;
    }
    // B tile: 32 k x 64 n
    for (int t = tid; t < 64 * 32; t += 256) {
      const int nn = t % 64, kb = t / 64;
      const int gn = n0 + nn, gk = k0 + kb;
      Bs[kb][nn] = (gn < g.N && gk < g.K) ? B[(int64_t)gk * g.ldb + gn] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < 32; ++k) {
      const float4 av = *reinterpret_cast<const float4*>(&As[k][ty * 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&Bs[k][tx * 4]);
      const float a[4] = {av.x, av.y, av.z, av.w}, b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        // TwoSum (Knuth); separately rounded operations, not contracted
        const float sum = __fadd_rn(hi[i][j], acc[i][j]);
        const float bb = __fsub_rn(sum, hi[i][j]);
        lo[i][j] += __fadd_rn(__fsub_rn(hi[i][j], __fsub_rn(sum, bb)), __fsub_rn(acc[i][j], bb));
        hi[i][j] = sum;
      }
  }
  const float* __restrict__ Cm = static_cast<const float*>(g.Cm);
  float* __restrict__ D = static_cast<float*>(g.D);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= g.N) continue;
      float v = alpha * (hi[i][j] + lo[i][j]);
      if (beta != 0.f) v = fmaf(beta, Cm[(int64_t)gm * g.ldc + gn], v);
      D[(int64_t)gm * g.ldd + gn] = v;
    }
  }
}

// ------------------------------------------------------------------ Gram
// H (s x s, f64, lower tiles) += Z^T Z for Z (n x s) float32.  Products and
// 32-row partial sums in FP32; the partial sums are accumulated in a
// float-float pair (Knuth's TwoSum), so the sum over all n rows carries about
// the error of one 32-term FP32 sum.  (An FP32 accumulator over all rows, or
// over chunks of a few hundred rows, perturbs H enough to move the ADMM fixed
// point by ~kappa(H) * 1e-7.)
// ------------------------------------------------------------------ double-float GEMM
// The FP64 GEMM of the set-up factorisation in double-float arithmetic on the FP32 pipes
// (this part issues FP32 FMAs at 64 times its FP64 rate).  Each FP64 input is held as a
// float pair x = hi + lo (48 significant bits); a product a b is formed exactly as
// p + e by p = a_hi b_hi, e = fma(a_hi, b_hi, -p), plus the cross terms a_hi b_lo and
// a_lo b_hi (a_lo b_lo, 2^-48 relative, is dropped); the accumulator is a float pair
// updated by TwoSum (Knuth), the error terms gathered in its low part.  The result is
// hi + lo in FP64: about 2^-44 relative per K = 64 dot product, enough for a factor whose
// inverse feeds FP32 and three-term BF16 iterations.  Same tiling and interface as k_gemm.
// An operand given as float pairs (PA / PB) is read as such; one given in FP64 is split on
// load (that takes FP64-pipe work, so operands that many CTAs read are split once
// beforehand by k_to_pairs).
constexpr int DF_BK = 16;

__device__ __forceinline__ void load_pair(const void* base, int64_t idx, bool paired, float& h, float& l) {
  if (paired) {
    const float2 v = static_cast<const float2*>(base)[idx];
    h = v.x;
    l = v.y;
  } else {
    const double v = static_cast<const double*>(base)[idx];
    h = __double2float_rn(v);
    l = __double2float_rn(v - (double)h);
  }
}

template <bool PA, bool PB>
__global__ void __launch_bounds__(256) k_gemm_df(const GemmDesc* __restrict__ descs, int transA, int transB,
                                                 double alpha, double beta, int lower_only) {
  const GemmDesc g = descs[blockIdx.z];
  const int tm = blockIdx.x, tn = blockIdx.y;
  if (tm * 64 >= g.M || tn * 64 >= g.N) return;
  if (lower_only && tn > tm) return;
  __shared__ float Ah[DF_BK][64 + 1], Al[DF_BK][64 + 1];
  __shared__ float Bh[DF_BK][64 + 1], Bl[DF_BK][64 + 1];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  float hi[4][4], lo[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) hi[i][j] = lo[i][j] = 0.f;
  const int m0 = tm * 64, n0 = tn * 64;
  for (int k0 = 0; k0 < g.K; k0 += DF_BK) {
    for (int t = tid; t < 64 * DF_BK; t += 256) {
      int mm, kk;
      if (transA) { mm = t % 64; kk = t / 64; } else { kk = t % DF_BK; mm = t / DF_BK; }
      const int gm = m0 + mm, gk = k0 + kk;
      float vh = 0.f, vl = 0.f;
      if (gm < g.M && gk < g.K)
        load_pair(g.A, transA ? (int64_t)gk * g.lda + gm : (int64_t)gm * g.lda + gk, PA, vh, vl);
      Ah[kk][mm] = vh;
      Al[kk][mm] = vl;
      int nn, kb;
      if (transB) { kb = t % DF_BK; nn = t / DF_BK; } else { nn = t % 64; kb = t / 64; }
      const int gn = n0 + nn, gkb = k0 + kb;
      float wh = 0.f, wl = 0.f;
      if (gn < g.N && gkb < g.K)
        load_pair(g.B, transB ? (int64_t)gn * g.ldb + gkb : (int64_t)gkb * g.ldb + gn, PB, wh, wl);
      Bh[kb][nn] = wh;
      Bl[kb][nn] = wl;
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < DF_BK; ++k) {
      float ah[4], al[4], bh[4], bl[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        ah[i] = Ah[k][ty * 4 + i];
        al[i] = Al[k][ty * 4 + i];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        bh[j] = Bh[k][tx * 4 + j];
        bl[j] = Bl[k][tx * 4 + j];
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          // the rounded product and the TwoSum steps must not be contracted into FMAs:
          // the exact-error identities hold only for separately rounded operations
          const float p = __fmul_rn(ah[i], bh[j]);
          float e = fmaf(ah[i], bh[j], -p);
          e = fmaf(ah[i], bl[j], e);
          e = fmaf(al[i], bh[j], e);
          const float s = __fadd_rn(hi[i][j], p);
          const float bb = __fsub_rn(s, hi[i][j]);
          const float err = __fadd_rn(__fsub_rn(hi[i][j], __fsub_rn(s, bb)), __fsub_rn(p, bb));
          lo[i][j] += err + e;
          hi[i][j] = s;
        }
    }
    __syncthreads();
  }
  const double* __restrict__ Cm = static_cast<const double*>(g.Cm);
  double* __restrict__ D = static_cast<double*>(g.D);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty * 4 + i;
    if (gm >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx * 4 + j;
      if (gn >= g.N) continue;
      double v = alpha * ((double)hi[i][j] + (double)lo[i][j]);
      if (beta != 0.0) v = fma(beta, Cm[(int64_t)gm * g.ldc + gn], v);
      D[(int64_t)gm * g.ldd + gn] = v;
    }
  }
}

// dst (float pairs, ld ldd) = src (FP64, ld lda), M x N per job (desc.A = src, desc.D = dst)
__global__ void k_to_pairs(const GemmDesc* __restrict__ descs) {
  const GemmDesc g = descs[blockIdx.z];
  const int64_t r = (int64_t)blockIdx.x * 8 + threadIdx.y, c = (int64_t)blockIdx.y * 32 + threadIdx.x;
  if (r >= g.M || c >= g.N) return;
  const double v = static_cast<const double*>(g.A)[r * g.lda + c];
  const float h = __double2float_rn(v);
  static_cast<float2*>(g.D)[r * g.ldd + c] = make_float2(h, __double2float_rn(v - (double)h));
}

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (x - bb);
  hi = s;
  lo += e;
}

// Gram accumulation H (FP64) += Z^T Z over the n rows of Z (n x s, row-major, ld ldz): one CTA
// per 128 x 64 tile of H that reaches the lower triangle, 8 x 4 outputs per thread (rows
// ty*4 + {0..3} and 64 + ty*4 + {0..3}, columns tx*4 + {0..3}: a warp's shared-memory reads are
// broadcasts or consecutive), rows staged 32 at a time through double-buffered shared memory
// (one stage's arithmetic covers the next stage's global loads).
// Products and 64-row partial sums in FP32 (round to nearest, unbiased), folded into a
// float-float accumulator (TwoSum) after every chunk, added to H in FP64 at the end: about
// 2^-44 relative per entry.
constexpr int GR_M = 128, GR_N = 64, GR_K = 32;

__global__ void __launch_bounds__(256) k_gram_tile(const float* __restrict__ Z, int64_t ldz, int64_t n, int64_t s,
                                                   double* __restrict__ H, int64_t ldh) {
  const int64_t a0 = (int64_t)blockIdx.x * GR_M, b0 = (int64_t)blockIdx.y * GR_N;
  if (b0 > a0 + GR_M - 1) return;   // wholly above the diagonal: the mirror fills it
  __shared__ __align__(16) float As[2][GR_K][GR_M];
  __shared__ __align__(16) float Bs[2][GR_K][GR_N];
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  float acc[8][4], hi[8][4], lo[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = hi[i][j] = lo[i][j] = 0.f;
  float ra[16], rb[8];   // the next stage in registers: A element tid + 256 q, B element tid + 256 q
  auto fetch = [&](int64_t r0) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int e = tid + 256 * q, r = e / GR_M, c = e % GR_M;
      ra[q] = (r0 + r < n && a0 + c < s) ? __ldg(Z + (r0 + r) * ldz + a0 + c) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 256 * q, r = e / GR_N, c = e % GR_N;
      rb[q] = (r0 + r < n && b0 + c < s) ? __ldg(Z + (r0 + r) * ldz + b0 + c) : 0.f;
    }
  };
  auto stash = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const int e = tid + 256 * q;
      As[buf][e / GR_M][e % GR_M] = ra[q];
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const int e = tid + 256 * q;
      Bs[buf][e / GR_N][e % GR_N] = rb[q];
    }
  };
  fetch(0);
  stash(0);
  __syncthreads();
  int buf = 0, stage = 0;
  for (int64_t r0 = 0; r0 < n; r0 += GR_K, ++stage) {
    const bool more = r0 + GR_K < n;
    if (more) fetch(r0 + GR_K);
#pragma unroll
    for (int k = 0; k < GR_K; ++k) {
      const float4 a_lo = *reinterpret_cast<const float4*>(&As[buf][k][ty * 4]);
      const float4 a_hi = *reinterpret_cast<const float4*>(&As[buf][k][64 + ty * 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&Bs[buf][k][tx * 4]);
      const float a[8] = {a_lo.x, a_lo.y, a_lo.z, a_lo.w, a_hi.x, a_hi.y, a_hi.z, a_hi.w};
      const float b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if ((stage & 1) || !more) {   // every 64 rows: fold the partial sums into hi + lo
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          two_sum_acc(hi[i][j], lo[i][j], acc[i][j]);
          acc[i][j] = 0.f;
        }
    }
    if (more) {   // nobody reads buf ^ 1 in this stage: the sync below ends the stage that did
      stash(buf ^ 1);
      __syncthreads();
      buf ^= 1;
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t gm = a0 + (i < 4 ? ty * 4 + i : 64 + ty * 4 + i - 4);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t gn = b0 + tx * 4 + j;
      if (gm < s && gn < s) H[gm * ldh + gn] += (double)hi[i][j] + (double)lo[i][j];
    }
  }
}

// ------------------------------------------------------------------ diagonal potrf
// One CTA per matrix: factor the bs x bs diagonal block starting at column kcol
// (bs = min(64, s - kcol)) in shared memory, write L back (upper part zeroed) and
// the inverse of L into inv (64 x 64, zero padded).  info = column+1 of the first
// non-positive pivot (the pivot is replaced by 1 so the factorisation finishes).
// Step c of the right-looking factorisation also takes step c of the forward substitution
// L X = I (X = L^-1, built in place of the identity: row c scaled by 1 / L_cc, then
// X_rq -= L_rc X_cq for r > c, q <= c), so the inverse needs no sweep of its own.  The
// trailing update walks only the pairs (r, q), c < q <= r, in an order where step c's pairs
// are a prefix of one table (pair (r, q) at r'(r'+1)/2 + q', r' = 63 - q, q' = 63 - r): no lane
// of a warp idles on this part's narrow FP64 pipe.  Every element sees the same operations in
// the same order as the column-by-column forms of both sweeps.
__global__ void __launch_bounds__(256) k_potrf_diag(const DiagJob* __restrict__ jobs, int kcol) {
  const DiagJob jb = jobs[blockIdx.x];
  if (kcol >= jb.s) return;
  const int bs = min(64, jb.s - kcol);
  __shared__ double L[64][65];
  __shared__ double Li[64][65];
  __shared__ double rinv[64];   // reciprocals of the pivots (one FP64 division each: this part's
                                // FP64 division is a long sequence on its 1/64-rate pipe)
  __shared__ uint16_t pairs[63 * 64 / 2];   // (r' << 8) | q', 0 <= q' <= r' < 63
  __shared__ int bad;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int t = tid; t < 64 * 64; t += 256) {
    const int r = t / 64, c = t % 64;
    L[r][c] = (r < bs && c < bs) ? jb.A[(int64_t)(kcol + r) * jb.ld + kcol + c] : (r == c ? 1.0 : 0.0);
    Li[r][c] = r == c ? 1.0 : 0.0;
    if (r < 63 && c <= r) pairs[r * (r + 1) / 2 + c] = (uint16_t)((r << 8) | c);
  }
  __syncthreads();
  for (int c = 0; c < bs; ++c) {
    if (tid == 0) {
      double d = L[c][c];
      if (!(d > 0.0)) {
        if (bad == 0) bad = kcol + c + 1;
        d = 1.0;
      }
      L[c][c] = sqrt(d);
      rinv[c] = 1.0 / L[c][c];
    }
    __syncthreads();
    const double ri = rinv[c];
    if (tid < 64) {
      if (c + 1 + tid < 64) L[c + 1 + tid][c] *= ri;
    } else if (tid < 128) {
      if (tid - 64 <= c) Li[c][tid - 64] *= ri;
    }
    __syncthreads();
    const int w = 63 - c, cw = c + 1;
    for (int p = tid; p < w * (w + 1) / 2; p += 256) {
      const uint32_t v = pairs[p];
      const int r = 63 - (int)(v & 0xffu), q = 63 - (int)(v >> 8);
      L[r][q] -= L[r][c] * L[q][c];
    }
    for (int t = tid; t < w * cw; t += 256) {
      const int r = c + 1 + t / cw, q = t % cw;
      Li[r][q] -= L[r][c] * Li[c][q];
    }
    __syncthreads();
  }
  for (int t = tid; t < 64 * 64; t += 256) {
    const int r = t / 64, c = t % 64;
    const bool in = r < bs && c < bs;
    if (in) jb.A[(int64_t)(kcol + r) * jb.ld + kcol + c] = (c <= r) ? L[r][c] : 0.0;
    jb.inv[t] = in ? Li[r][c] : 0.0;
  }
  if (tid == 0 && bad && jb.info && *jb.info == 0) *jb.info = bad;
}

__global__ void k_zero_strict_upper(double* A, int64_t s) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= s * s) return;
  if (t % s > t / s) A[t] = 0.0;
}

__global__ void k_add_identity_and_mirror(double* H, int64_t ldh, int64_t s) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= s * s) return;
  const int64_t r = t / s, c = t % s;
  if (c > r) H[r * ldh + c] = H[c * ldh + r];
  else if (c == r) H[r * ldh + c] += 1.0;
}

}  // namespace

cudaError_t launch_gemm_f32_nn(const GemmDesc* descs_dev, int nbatch, int maxM, int maxN, float alpha, float beta,
                               cudaStream_t st, const uint8_t* bmask) {
  if (nbatch <= 0 || maxM <= 0 || maxN <= 0) return cudaSuccess;
  dim3 grid((unsigned)ceil_div(maxM, 64), (unsigned)ceil_div(maxN, 64), (unsigned)nbatch);
  k_gemm_f32_nn<<<grid, 256, 0, st>>>(descs_dev, GemmDesc{}, alpha, beta, bmask);
  return cudaGetLastError();
}

cudaError_t launch_gemm_f32_nn_one(const GemmDesc& g, float alpha, float beta, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  dim3 grid((unsigned)ceil_div(g.M, 64), (unsigned)ceil_div(g.N, 64), 1);
  k_gemm_f32_nn<<<grid, 256, 0, st>>>(nullptr, g, alpha, beta, nullptr);
  return cudaGetLastError();
}

cudaError_t launch_gemm_f64(const GemmDesc* descs_dev, int nbatch, int maxM, int maxN, int transA, int transB,
                            double alpha, double beta, int lower_only, cudaStream_t st, bool double_float) {
  if (nbatch <= 0 || maxM <= 0 || maxN <= 0) return cudaSuccess;
  dim3 grid((unsigned)ceil_div(maxM, 64), (unsigned)ceil_div(maxN, 64), (unsigned)nbatch);
  if (double_float)
    k_gemm_df<false, false><<<grid, 256, 0, st>>>(descs_dev, transA, transB, alpha, beta, lower_only);
  else
    k_gemm<double, 16><<<grid, 256, 0, st>>>(descs_dev, transA, transB, alpha, beta, lower_only);
  return cudaGetLastError();
}

// double-float GEMM with both operands given as float pairs
cudaError_t launch_gemm_df_pairs(const GemmDesc* descs_dev, int nbatch, int maxM, int maxN, int transA, int transB,
                                 double alpha, double beta, int lower_only, cudaStream_t st) {
  if (nbatch <= 0 || maxM <= 0 || maxN <= 0) return cudaSuccess;
  dim3 grid((unsigned)ceil_div(maxM, 64), (unsigned)ceil_div(maxN, 64), (unsigned)nbatch);
  k_gemm_df<true, true><<<grid, 256, 0, st>>>(descs_dev, transA, transB, alpha, beta, lower_only);
  return cudaGetLastError();
}

cudaError_t launch_to_pairs(const GemmDesc* descs_dev, int nbatch, int maxM, int maxN, cudaStream_t st) {
  if (nbatch <= 0 || maxM <= 0 || maxN <= 0) return cudaSuccess;
  dim3 grid((unsigned)ceil_div(maxM, 8), (unsigned)ceil_div(maxN, 32), (unsigned)nbatch);
  k_to_pairs<<<grid, dim3(32, 8), 0, st>>>(descs_dev);
  return cudaGetLastError();
}

cudaError_t launch_gram_f32_to_f64(const float* Z, int64_t ldz, int64_t n, int64_t s, double* H, int64_t ldh,
                                   cudaStream_t st) {
  if (n <= 0 || s <= 0) return cudaSuccess;
  dim3 grid((unsigned)ceil_div(s, GR_M), (unsigned)ceil_div(s, GR_N));
  k_gram_tile<<<grid, 256, 0, st>>>(Z, ldz, n, s, H, ldh);
  return cudaGetLastError();
}

cudaError_t launch_zero_strict_upper(double* A, int64_t s, int nbatch, cudaStream_t st) {
  for (int b = 0; b < nbatch; ++b) {
    k_zero_strict_upper<<<(unsigned)ceil_div(s * s, 256), 256, 0, st>>>(A + (size_t)b * s * s, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_add_identity_and_mirror(double* H, int64_t ldh, int64_t s, cudaStream_t st) {
  if (s <= 0) return cudaSuccess;
  k_add_identity_and_mirror<<<(unsigned)ceil_div(s * s, 256), 256, 0, st>>>(H, ldh, s);
  return cudaGetLastError();
}

cudaError_t launch_potrf_diag(const DiagJob* jobs_dev, int njobs, int kcol, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  k_potrf_diag<<<njobs, 256, 0, st>>>(jobs_dev, kcol);
  return cudaGetLastError();
}

// Blocked right-looking Cholesky (64-column panels) of every A_b in place, then
// optionally Q_b = A_b^-1 by forward and backward substitution against the
// identity, using the inverted 64 x 64 diagonal factors:
//   potrf step k:  L_kk = chol(A_kk);  A_ik <- A_ik L_kk^-T;  A_il -= A_ik A_lk^T
//   L Y = I:       Y_k = L_kk^-1 B_k;  B_i -= L_ik Y_k   (i > k)
//   L^T Q = Y:     Q_k = L_kk^-T Y_k;  Y_i -= L_ki^T Q_k (i < k)
// Descriptors live in `dev_scratch` (>= factor_scratch_bytes bytes).
// Q[r][c] = Q[c][r] for c > r (the upper triangle from the lower)
__global__ void k_mirror_lower(double* __restrict__ Q, int64_t ld, int64_t s) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= s * s) return;
  const int64_t r = t / s, c = t % s;
  if (c > r) Q[r * ld + c] = Q[c * ld + r];
}

cudaError_t launch_mirror_lower(double* Q, int64_t ld, int64_t s, cudaStream_t st) {
  if (s <= 1) return cudaSuccess;
  k_mirror_lower<<<(unsigned)ceil_div(s * s, 256), 256, 0, st>>>(Q, ld, s);
  return cudaGetLastError();
}

// descriptor phases of the blocked factorisation: 0 panel, 1 trailing update, 2-3 forward
// sweep, 4-5 backward sweep, 6-9 conversions to float pairs (double-float mode)
constexpr int FACTOR_PHASES = 10;

// RFF_FACTOR=df selects the double-float block updates below instead of the tensor-core ones
// of ozaki.cu (read once)
static bool use_double_float_updates() {
  static const bool df = [] {
    const char* e = getenv("RFF_FACTOR");
    return e && strcmp(e, "df") == 0;
  }();
  return df;
}

size_t factor_scratch_bytes(int njobs, int smax) {
  const int nb = (int)ceil_div(smax, 64);
  // per job: the diagonal inverses, and two 64 x (nb * 64) float-pair staging buffers
  const size_t df = (size_t)njobs * nb * 64 * 64 * sizeof(double) +
                    (size_t)njobs * 2 * 64 * nb * 64 * sizeof(float2) + (size_t)njobs * sizeof(DiagJob) * nb +
                    (size_t)njobs * nb * FACTOR_PHASES * sizeof(GemmDesc) + 1024;
  return std::max(df, oz_factor_scratch_bytes(njobs, smax));
}

cudaError_t factor_and_invert_f64(const std::vector<MatJob>& jobs, bool invert, void* dev_scratch, cudaStream_t st,
                                  bool double_float, int oz_bits) {
  const int nj = (int)jobs.size();
  if (nj == 0) return cudaSuccess;
  if (!use_double_float_updates()) return factor_and_invert_oz(jobs, invert, dev_scratch, st, oz_bits);
  int smax = 0;
  for (const auto& j : jobs) smax = std::max(smax, j.s);
  const int nb = (int)ceil_div(smax, 64);
  char* p = static_cast<char*>(dev_scratch);
  double* inv = reinterpret_cast<double*>(p);
  p += (size_t)nj * nb * 64 * 64 * sizeof(double);
  // float-pair copies of the operands that many CTAs of one double-float GEMM read: P2 holds
  // the L panel below the diagonal block (rest x 64, ld 64) or the L block row (64 x c0,
  // ld ldp); B2 the block row of Q (64 x ncol, ld ldp)
  const int64_t ldp = (int64_t)nb * 64;
  float2* pairs = reinterpret_cast<float2*>(p);
  p += (size_t)nj * 2 * 64 * ldp * sizeof(float2);
  DiagJob* djobs = reinterpret_cast<DiagJob*>(p);
  p += (size_t)nj * nb * sizeof(DiagJob);
  GemmDesc* gd = reinterpret_cast<GemmDesc*>(p);

  std::vector<DiagJob> hd((size_t)nj * nb);
  for (int k = 0; k < nb; ++k)
    for (int b = 0; b < nj; ++b)
      hd[(size_t)k * nj + b] = DiagJob{jobs[b].A, jobs[b].ld, jobs[b].s, inv + ((size_t)b * nb + k) * 4096,
                                       jobs[b].info};
  cudaError_t e = cudaMemcpyAsync(djobs, hd.data(), hd.size() * sizeof(DiagJob), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;

  // descriptor table: [phase][k][b]
  std::vector<GemmDesc> g((size_t)FACTOR_PHASES * nb * nj);
  auto at = [&](int ph, int k, int b) -> GemmDesc& { return g[((size_t)ph * nb + k) * nj + b]; };
  for (int k = 0; k < nb; ++k)
    for (int b = 0; b < nj; ++b) {
      const MatJob& J = jobs[b];
      const int64_t c0 = (int64_t)k * 64;
      const int bs = (int)std::max<int64_t>(0, std::min<int64_t>(64, J.s - c0));
      const int rest = (int)std::max<int64_t>(0, J.s - c0 - 64);
      double* Ikk = inv + ((size_t)b * nb + k) * 4096;
      float2* P2 = pairs + (size_t)b * 2 * 64 * ldp;
      float2* B2 = P2 + 64 * ldp;
      double* Lp = J.A + (c0 + 64) * J.ld + c0;   // L panel below the diagonal block
      GemmDesc z{};
      // panel: A_ik <- A_ik * inv^T (in place)
      GemmDesc pn = z;
      if (bs > 0 && rest > 0) pn = GemmDesc{J.A + (c0 + 64) * J.ld + c0, Ikk, nullptr, J.A + (c0 + 64) * J.ld + c0,
                                            rest, bs, bs, J.ld, 64, 0, J.ld};
      at(0, k, b) = pn;
      GemmDesc tr = z, cp = z;
      if (bs > 0 && rest > 0) {
        if (double_float) {
          cp = GemmDesc{Lp, nullptr, nullptr, P2, rest, bs, 0, J.ld, 0, 0, 64};
          tr = GemmDesc{P2, P2, Lp + 64, Lp + 64, rest, rest, bs, 64, 64, J.ld, J.ld};
        } else {
          tr = GemmDesc{Lp, Lp, Lp + 64, Lp + 64, rest, rest, bs, J.ld, J.ld, J.ld, J.ld};
        }
      }
      at(1, k, b) = tr;
      at(6, k, b) = cp;
      // Inverse Q = L^-T L^-1 from Q = I: the forward sweep (L Y = I) touches only the
      // columns up to the diagonal block of block row k (Y is lower triangular); the
      // backward sweep (L^T Q = Y) computes the block lower triangle of the symmetric Q,
      // which needs the same columns; the strict upper triangle is mirrored afterwards.
      // s^3/3 flops per sweep instead of s^3.
      GemmDesc fa = z, fb = z, ba = z, bb = z, cq = z, cl = z, cqb = z;
      const int ncol = (int)(c0 + bs);
      double* Qk = J.Q + c0 * J.ldq;   // block row k of Q
      if (invert && bs > 0) {
        fa = GemmDesc{Ikk, Qk, nullptr, Qk, bs, ncol, bs, 64, J.ldq, 0, J.ldq};
        ba = fa;
        if (double_float) {
          // the forward update reads the panel pairs of phase 6 and Q_k converted after fa
          cq = GemmDesc{Qk, nullptr, nullptr, B2, bs, ncol, 0, J.ldq, 0, 0, ldp};
          if (rest > 0) fb = GemmDesc{P2, B2, Qk + 64 * J.ldq, Qk + 64 * J.ldq, rest, ncol, bs, 64, ldp, J.ldq,
                                      J.ldq};
          if (c0 > 0) {
            cl = GemmDesc{J.A + c0 * J.ld, nullptr, nullptr, P2, bs, (int)c0, 0, J.ld, 0, 0, ldp};
            cqb = GemmDesc{Qk, nullptr, nullptr, B2, bs, (int)c0, 0, J.ldq, 0, 0, ldp};
            bb = GemmDesc{P2, B2, J.Q, J.Q, (int)c0, (int)c0, bs, ldp, ldp, J.ldq, J.ldq};
          }
        } else {
          if (rest > 0) fb = GemmDesc{Lp, Qk, Qk + 64 * J.ldq, Qk + 64 * J.ldq, rest, ncol, bs, J.ld, J.ldq, J.ldq,
                                      J.ldq};
          if (c0 > 0) bb = GemmDesc{J.A + c0 * J.ld, Qk, J.Q, J.Q, (int)c0, (int)c0, bs, J.ld, J.ldq, J.ldq, J.ldq};
        }
      }
      at(2, k, b) = fa;
      at(3, k, b) = fb;
      at(4, k, b) = ba;
      at(5, k, b) = bb;
      at(7, k, b) = cq;
      at(8, k, b) = cl;
      at(9, k, b) = cqb;
    }
  e = cudaMemcpyAsync(gd, g.data(), g.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  auto dev = [&](int ph, int k) { return gd + ((size_t)ph * nb + k) * nj; };

  // the GEMMs that many CTAs feed from one panel or block row (trailing update, forward and
  // backward updates) read float pairs converted once per step in double-float mode; the
  // 64-row products (panel solve, diagonal-block products) split their FP64 operands on load
  const bool df = double_float;
  auto upd = [&](int ph, int k, int M, int N, int tA, int tB, int lower) {
    return df ? launch_gemm_df_pairs(dev(ph, k), nj, M, N, tA, tB, -1.0, 1.0, lower, st)
              : launch_gemm_f64(dev(ph, k), nj, M, N, tA, tB, -1.0, 1.0, lower, st);
  };
  for (int k = 0; k < nb; ++k) {
    const int c0 = k * 64, rest = std::max(0, smax - c0 - 64);
    if ((e = launch_potrf_diag(djobs + (size_t)k * nj, nj, c0, st)) != cudaSuccess) return e;
    if (rest > 0) {
      if ((e = launch_gemm_f64(dev(0, k), nj, rest, 64, 0, 1, 1.0, 0.0, 0, st, df)) != cudaSuccess) return e;
      if (df && (e = launch_to_pairs(dev(6, k), nj, rest, 64, st)) != cudaSuccess) return e;
      if ((e = upd(1, k, rest, rest, 0, 1, 1)) != cudaSuccess) return e;
    }
  }
  if (!invert) return cudaSuccess;
  for (int k = 0; k < nb; ++k) {
    const int c0 = k * 64, rest = std::max(0, smax - c0 - 64), ncol = std::min(smax, c0 + 64);
    if ((e = launch_gemm_f64(dev(2, k), nj, 64, ncol, 0, 0, 1.0, 0.0, 0, st, df)) != cudaSuccess) return e;
    if (rest > 0) {
      if (df && ((e = launch_to_pairs(dev(6, k), nj, rest, 64, st)) != cudaSuccess ||
                 (e = launch_to_pairs(dev(7, k), nj, 64, ncol, st)) != cudaSuccess))
        return e;
      if ((e = upd(3, k, rest, ncol, 0, 0, 0)) != cudaSuccess) return e;
    }
  }
  for (int k = nb - 1; k >= 0; --k) {
    const int c0 = k * 64, ncol = std::min(smax, c0 + 64);
    if ((e = launch_gemm_f64(dev(4, k), nj, 64, ncol, 1, 0, 1.0, 0.0, 0, st, df)) != cudaSuccess) return e;
    if (c0 > 0) {
      if (df && ((e = launch_to_pairs(dev(8, k), nj, 64, c0, st)) != cudaSuccess ||
                 (e = launch_to_pairs(dev(9, k), nj, 64, c0, st)) != cudaSuccess))
        return e;
      if ((e = upd(5, k, c0, c0, 1, 0, 0)) != cudaSuccess) return e;
    }
  }
  for (const auto& J : jobs)
    if ((e = launch_mirror_lower(J.Q, J.ldq, J.s, st)) != cudaSuccess) return e;
  return cudaSuccess;
}

}  // namespace rff
