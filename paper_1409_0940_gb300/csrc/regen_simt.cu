// FP32 SIMT regeneration passes: the plain FP32 path (no tensor cores).
//
// Each CTA multiplies a fixed 64-row panel of one operand ("A") against a run of
// 64-row panels of the other ("B"), both holding rows of length K (the input
// dimension d, padded):
//     T   = A_panel . B_panel^T                       (X_i G_j or its transpose)
//     Z   = sqrt(2/D) cos(T + b)  masked to valid slots  (the transform T[X_i, j], Sec. 4;
//           the random Laplace map: Z = exp(-T) / sqrt(D))
//     acc += Z . M[B rows]                             (the chained product)
// and writes acc when a run ends.  With A = feature rows of G^T and B = data rows
// this is pass 1, R_ij = Z_ij^T V_ij (the Z_ij^T (Obar_ij + nu_i) term of eq. (gpWij));
// with A = data rows and B = feature rows it is pass 2, O'_ij = Z_ij W'_ij
// (eq. (gpOij)), and prediction when M is Wbar and the run spans all blocks.
#include "common.cuh"
#include "internal.h"

namespace rff {

namespace {

constexpr int BM = 64, BN = 64, BK = 32, NT = 256;
constexpr int APAD = BM + 4, BPAD = BN + 4, ZPAD = BN + 1;

struct SimtSmem {
  float As[BK][APAD];
  float Bs[BK][BPAD];
  float Zs[BM][ZPAD];
  // Ms (BN x m_pad) follows dynamically
};

// One 64 x 64 tile: T = A[a0:a0+64] . B[b0:b0+64]^T, then Z into smem.
// bias_on_a: the feature index is the A row (pass 1) or the B row (pass 2).
__device__ __forceinline__ void tile_z(SimtSmem& sm, const float* __restrict__ A, int64_t lda, int64_t a0,
                                       const float* __restrict__ B, int64_t ldb, int64_t b0, int K,
                                       const float* __restrict__ bias, bool bias_on_a, float scale,
                                       const int32_t* __restrict__ a_ok, const int32_t* __restrict__ b_ok,
                                       int map) {
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  float acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  const int lr = tid / 4, lk = (tid % 4) * 8;
  for (int k0 = 0; k0 < K; k0 += BK) {
    const float4* pa = reinterpret_cast<const float4*>(A + (a0 + lr) * lda + k0 + lk);
    const float4* pb = reinterpret_cast<const float4*>(B + (b0 + lr) * ldb + k0 + lk);
    const float4 a_0 = pa[0], a_1 = pa[1], b_0 = pb[0], b_1 = pb[1];
    __syncthreads();
    sm.As[lk + 0][lr] = a_0.x; sm.As[lk + 1][lr] = a_0.y; sm.As[lk + 2][lr] = a_0.z; sm.As[lk + 3][lr] = a_0.w;
    sm.As[lk + 4][lr] = a_1.x; sm.As[lk + 5][lr] = a_1.y; sm.As[lk + 6][lr] = a_1.z; sm.As[lk + 7][lr] = a_1.w;
    sm.Bs[lk + 0][lr] = b_0.x; sm.Bs[lk + 1][lr] = b_0.y; sm.Bs[lk + 2][lr] = b_0.z; sm.Bs[lk + 3][lr] = b_0.w;
    sm.Bs[lk + 4][lr] = b_1.x; sm.Bs[lk + 5][lr] = b_1.y; sm.Bs[lk + 6][lr] = b_1.z; sm.Bs[lk + 7][lr] = b_1.w;
    __syncthreads();
#pragma unroll 8
    for (int k = 0; k < BK; ++k) {
      const float4 av = *reinterpret_cast<const float4*>(&sm.As[k][ty * 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&sm.Bs[k][tx * 4]);
      const float a[4] = {av.x, av.y, av.z, av.w}, b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
  }
  // epilogue: cos with the feature phase (or exp(-T), the Laplace map), masked to valid rows/features
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t ar = a0 + ty * 4 + i;
    const bool aok = a_ok ? (a_ok[ar] >= 0) : true;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t br = b0 + tx * 4 + j;
      const bool ok = aok && (b_ok ? (b_ok[br] >= 0) : true);
      const float ph = bias_on_a ? bias[ar] : bias[br];
      sm.Zs[ty * 4 + i][tx * 4 + j] = !ok ? 0.f : map == 1 ? scale * expf(-acc[i][j]) : scale * cos_rr(acc[i][j] + ph);
    }
  }
}

// acc2[4][MQ] += Zs[ty*4+i][n] * Ms[n][tx + 16 q]
template <int MQ>
__device__ __forceinline__ void chain(const SimtSmem& sm, const float* __restrict__ Ms, int mpad,
                                      float (&acc2)[4][MQ]) {
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
#pragma unroll 4
  for (int n = 0; n < BN; ++n) {
    float z[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) z[i] = sm.Zs[ty * 4 + i][n];
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
      const float mv = Ms[n * mpad + tx + 16 * q];
#pragma unroll
      for (int i = 0; i < 4; ++i) acc2[i][q] = fmaf(z[i], mv, acc2[i][q]);
    }
  }
}

__device__ __forceinline__ void load_M(float* Ms, const float* __restrict__ M, int64_t b0, int mpad) {
  const int n4 = BN * mpad / 4;
  const float4* src = reinterpret_cast<const float4*>(M + b0 * mpad);
  float4* dst = reinterpret_cast<float4*>(Ms);
  for (int t = threadIdx.x; t < n4; t += NT) dst[t] = src[t];
}

template <int MQ>
__device__ __forceinline__ void store_acc(float (&acc2)[4][MQ], float* __restrict__ out, int64_t row0, int mpad) {
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
      out[(row0 + ty * 4 + i) * mpad + tx + 16 * q] = acc2[i][q];
      acc2[i][q] = 0.f;
    }
}

// Pass 2 / predict: one CTA per 64 data rows; runs over the feature slots of
// every column block.  per_block: write O'_ij at the end of each block j (to
// out + j * out_block_stride); else accumulate over all blocks and write once.
template <int MQ>
__global__ void __launch_bounds__(NT) k_pass2_simt(PassArgs p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SimtSmem& sm = *reinterpret_cast<SimtSmem*>(smem_raw);
  float* Ms = reinterpret_cast<float*>(smem_raw + sizeof(SimtSmem));
  const int64_t a0 = (int64_t)blockIdx.x * BM;
  // row block of this tile: the chain operand W'_ij depends on it
  int rb = 0;
  while (rb + 1 < p.R && p.row_slot[rb + 1] <= a0) ++rb;
  const uint8_t* act = p.bmask ? p.bmask + rb * p.C : nullptr;   // skip inactive blocks (per_block)
  const float* M = p.M + rb * p.m_block_stride;
  float acc2[4][MQ];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < MQ; ++q) acc2[i][q] = 0.f;
  for (int j = 0; j < p.C; ++j) {
    if (act && !act[j]) continue;
    const int64_t f0 = p.col_slot[j], f1 = f0 + p.col_size[j];
    for (int64_t b0 = f0; b0 < f1; b0 += BN) {
      tile_z(sm, p.X, p.ldx, a0, p.Gt, p.ldg, b0, p.K, p.bias, false, p.scale, p.row_ok, p.feat_ok, p.map);
      __syncthreads();
      load_M(Ms, M, b0, p.mpad);
      __syncthreads();
      chain<MQ>(sm, Ms, p.mpad, acc2);
      __syncthreads();
    }
    if (p.per_block) store_acc<MQ>(acc2, p.out + j * p.out_block_stride, a0, p.mpad);
  }
  if (!p.per_block) store_acc<MQ>(acc2, p.out, a0, p.mpad);
}

// Pass 1: one CTA per (64 feature slots, row block i, row split); runs over the
// data rows of its split.  Writes R-partials (features x m_pad).
template <int MQ>
__global__ void __launch_bounds__(NT) k_pass1_simt(PassArgs p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SimtSmem& sm = *reinterpret_cast<SimtSmem*>(smem_raw);
  float* Ms = reinterpret_cast<float*>(smem_raw + sizeof(SimtSmem));
  const int64_t a0 = (int64_t)blockIdx.x * BM;  // feature slot tile
  const int i = blockIdx.y, split = blockIdx.z;
  // column block of this feature tile, and whether it holds any valid feature
  int j = 0;
  while (j + 1 < p.C && p.col_slot[j + 1] <= a0) ++j;
  if (a0 - p.col_slot[j] >= p.col_size[j]) return;
  if (p.bmask && !p.bmask[i * p.C + j]) return;   // inactive block: its partials are not read
  const int64_t r0 = p.row_slot[i], nrt = ceil_div(p.row_size[i], BM);
  const int64_t t0 = split * nrt / p.nsplit, t1 = (split + 1) * nrt / p.nsplit;
  const float* M = p.M + j * p.m_block_stride;
  float acc2[4][MQ];
#pragma unroll
  for (int ii = 0; ii < 4; ++ii)
#pragma unroll
    for (int q = 0; q < MQ; ++q) acc2[ii][q] = 0.f;
  for (int64_t t = t0; t < t1; ++t) {
    const int64_t b0 = r0 + t * BN;
    tile_z(sm, p.Gt, p.ldg, a0, p.X, p.ldx, b0, p.K, p.bias, true, p.scale, p.feat_ok, p.row_ok, p.map);
    __syncthreads();
    load_M(Ms, M, b0, p.mpad);
    __syncthreads();
    chain<MQ>(sm, Ms, p.mpad, acc2);
    __syncthreads();
  }
  store_acc<MQ>(acc2, p.out + ((int64_t)split * p.R + i) * p.out_block_stride, a0, p.mpad);
}

// Materialise Z for rows [r0, r0 + nr) and feature slots [f0, f0 + nf) into
// out (nr x nf, leading dimension ldo); one CTA per 64 x 64 tile.
__global__ void __launch_bounds__(NT) k_write_z_simt(ZArgs p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SimtSmem& sm = *reinterpret_cast<SimtSmem*>(smem_raw);
  const int64_t a0 = p.r0 + (int64_t)blockIdx.x * BM, b0 = p.f0 + (int64_t)blockIdx.y * BN;
  tile_z(sm, p.X, p.ldx, a0, p.Gt, p.ldg, b0, p.K, p.bias, false, p.scale, p.row_ok, p.feat_ok, p.map);
  __syncthreads();
  for (int t = threadIdx.x; t < BM * BN; t += NT) {
    const int r = t / BN, c = t % BN;
    const int64_t gr = a0 - p.r0 + r, gc = b0 - p.f0 + c;
    if (gr < p.nr && gc < p.nf) p.out[gr * p.ldo + gc] = sm.Zs[r][c];
  }
}

template <int MQ>
cudaError_t launch_pass_mq(int which, const PassArgs& p, dim3 grid, cudaStream_t st) {
  const size_t smem = sizeof(SimtSmem) + (size_t)BN * p.mpad * sizeof(float);
  if (which == 1) {
    cudaFuncSetAttribute(k_pass1_simt<MQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_pass1_simt<MQ><<<grid, NT, smem, st>>>(p);
  } else {
    cudaFuncSetAttribute(k_pass2_simt<MQ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_pass2_simt<MQ><<<grid, NT, smem, st>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t launch_pass(int which, const PassArgs& p, dim3 grid, cudaStream_t st) {
  switch (p.mpad / 16) {
#define RFF_MQ(q) \
  case q:         \
    return launch_pass_mq<q>(which, p, grid, st);
    RFF_MQ(1) RFF_MQ(2) RFF_MQ(3) RFF_MQ(4) RFF_MQ(5) RFF_MQ(6) RFF_MQ(7) RFF_MQ(8)
    RFF_MQ(9) RFF_MQ(10) RFF_MQ(11) RFF_MQ(12) RFF_MQ(13) RFF_MQ(14) RFF_MQ(15) RFF_MQ(16)
#undef RFF_MQ
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_pass2_simt(const PassArgs& p, int64_t nrow_slots, cudaStream_t st) {
  if (nrow_slots % BM) return cudaErrorInvalidValue;
  return launch_pass(2, p, dim3((unsigned)(nrow_slots / BM)), st);
}

cudaError_t launch_pass1_simt(const PassArgs& p, int64_t nfeat_slots, cudaStream_t st) {
  if (nfeat_slots % BM) return cudaErrorInvalidValue;
  return launch_pass(1, p, dim3((unsigned)(nfeat_slots / BM), (unsigned)p.R, (unsigned)p.nsplit), st);
}

cudaError_t launch_write_z_simt(const ZArgs& p, cudaStream_t st) {
  if (p.nr <= 0 || p.nf <= 0) return cudaSuccess;
  const size_t smem = sizeof(SimtSmem);
  cudaFuncSetAttribute(k_write_z_simt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((unsigned)ceil_div(p.nr, BM), (unsigned)ceil_div(p.nf, BN));
  k_write_z_simt<<<grid, NT, smem, st>>>(p);
  return cudaGetLastError();
}

}  // namespace rff
