// FP32 SIMT regeneration passes: the plain FP32 path (no tensor cores).
//
// Each CTA multiplies a fixed 128-row panel of one operand ("A") against a run of
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
//
// Thread tile: 8 A rows (ty*4 + {0..3} and 64 + ty*4 + {0..3}) by 4 B rows (tx*4 + {0..3})
// for T, and the same 8 A rows by m_pad/16 output columns (tx + 16 q) for acc, so that every
// shared-memory read of a warp is a broadcast or a run of consecutive words.  The next K
// chunk of both panels is fetched into registers while the current one is multiplied.
#include "common.cuh"
#include "internal.h"

namespace rff {

namespace {

constexpr int BM = 128, BN = 64, BK = 32, NT = 256;
constexpr int APAD = BM + 4, BPAD = BN + 4;

struct SimtSmem {
  float As[BK][APAD];    // A panel, K-major
  float Bs[BK][BPAD];    // B panel, K-major
  float ZsT[BN][APAD];   // Z tile transposed: [B row][A row]
  // Ms (BN x m_pad) follows dynamically
};

struct PanelRegs {
  float4 a[4];   // A: 128 rows x 32 K = 1024 float4, four per thread
  float4 b[2];   // B: 64 rows x 32 K = 512 float4, two per thread
};

__device__ __forceinline__ void fetch_panels(PanelRegs& r, const float* __restrict__ A, int64_t lda, int64_t a0,
                                             const float* __restrict__ B, int64_t ldb, int64_t b0, int k0) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = tid + NT * q, row = e / 8, k4 = e % 8;
    r.a[q] = __ldg(reinterpret_cast<const float4*>(A + (a0 + row) * lda + k0 + 4 * k4));
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int e = tid + NT * q, row = e / 8, k4 = e % 8;
    r.b[q] = __ldg(reinterpret_cast<const float4*>(B + (b0 + row) * ldb + k0 + 4 * k4));
  }
}

__device__ __forceinline__ void stash_panels(SimtSmem& sm, const PanelRegs& r) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int e = tid + NT * q, row = e / 8, k = 4 * (e % 8);
    sm.As[k][row] = r.a[q].x;
    sm.As[k + 1][row] = r.a[q].y;
    sm.As[k + 2][row] = r.a[q].z;
    sm.As[k + 3][row] = r.a[q].w;
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int e = tid + NT * q, row = e / 8, k = 4 * (e % 8);
    sm.Bs[k][row] = r.b[q].x;
    sm.Bs[k + 1][row] = r.b[q].y;
    sm.Bs[k + 2][row] = r.b[q].z;
    sm.Bs[k + 3][row] = r.b[q].w;
  }
}

__device__ __forceinline__ int arow_of(int ty, int i) { return i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4); }

// One 128 x 64 tile: T = A[a0:a0+128] . B[b0:b0+64]^T, then Z^T into shared memory.
// bias_on_a: the feature index is the A row (pass 1) or the B row (pass 2).
// Ends with a barrier: ZsT is complete, As/Bs free.
__device__ __forceinline__ void tile_z(SimtSmem& sm, const float* __restrict__ A, int64_t lda, int64_t a0,
                                       const float* __restrict__ B, int64_t ldb, int64_t b0, int K,
                                       const float* __restrict__ bias, bool bias_on_a, float scale,
                                       const int32_t* __restrict__ a_ok, const int32_t* __restrict__ b_ok,
                                       int map) {
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  PanelRegs r;
  fetch_panels(r, A, lda, a0, B, ldb, b0, 0);
  for (int k0 = 0; k0 < K; k0 += BK) {
    __syncthreads();   // the previous chunk (or the previous tile's chain) is done with shared memory
    stash_panels(sm, r);
    __syncthreads();
    if (k0 + BK < K) fetch_panels(r, A, lda, a0, B, ldb, b0, k0 + BK);
#pragma unroll 8
    for (int k = 0; k < BK; ++k) {
      const float4 a_lo = *reinterpret_cast<const float4*>(&sm.As[k][ty * 4]);
      const float4 a_hi = *reinterpret_cast<const float4*>(&sm.As[k][64 + ty * 4]);
      const float4 bv = *reinterpret_cast<const float4*>(&sm.Bs[k][tx * 4]);
      const float a[8] = {a_lo.x, a_lo.y, a_lo.z, a_lo.w, a_hi.x, a_hi.y, a_hi.z, a_hi.w};
      const float b[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
  }
  // epilogue: cos with the feature phase (or exp(-T), the Laplace map), masked to valid rows/features
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int ar = arow_of(ty, i);
    const bool aok = a_ok ? (a_ok[a0 + ar] >= 0) : true;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int br = tx * 4 + j;
      const bool ok = aok && (b_ok ? (b_ok[b0 + br] >= 0) : true);
      const float ph = bias_on_a ? bias[a0 + ar] : bias[b0 + br];
      sm.ZsT[br][ar] = !ok ? 0.f : map == 1 ? scale * expf(-acc[i][j]) : scale * cos_rr(acc[i][j] + ph);
    }
  }
  __syncthreads();
}

// acc2[i][q] += Z[arow_of(ty, i)][n] * Ms[n][tx + 16 q] over the 64 B rows n
template <int MQ>
__device__ __forceinline__ void chain(const SimtSmem& sm, const float* __restrict__ Ms, int mpad,
                                      float (&acc2)[8][MQ]) {
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
#pragma unroll 2
  for (int n = 0; n < BN; ++n) {
    const float4 z_lo = *reinterpret_cast<const float4*>(&sm.ZsT[n][ty * 4]);
    const float4 z_hi = *reinterpret_cast<const float4*>(&sm.ZsT[n][64 + ty * 4]);
    const float z[8] = {z_lo.x, z_lo.y, z_lo.z, z_lo.w, z_hi.x, z_hi.y, z_hi.z, z_hi.w};
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
      const float mv = Ms[n * mpad + tx + 16 * q];
#pragma unroll
      for (int i = 0; i < 8; ++i) acc2[i][q] = fmaf(z[i], mv, acc2[i][q]);
    }
  }
}

// Ms = the 64 rows b0.. of M (64 x m_pad); callers separate it from chain() by barriers
__device__ __forceinline__ void load_M(float* Ms, const float* __restrict__ M, int64_t b0, int mpad) {
  const int n4 = BN * mpad / 4;
  const float4* src = reinterpret_cast<const float4*>(M + b0 * mpad);
  float4* dst = reinterpret_cast<float4*>(Ms);
  for (int t = threadIdx.x; t < n4; t += NT) dst[t] = src[t];
}

template <int MQ>
__device__ __forceinline__ void store_acc(float (&acc2)[8][MQ], float* __restrict__ out, int64_t row0, int mpad) {
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int q = 0; q < MQ; ++q) {
      out[(row0 + arow_of(ty, i)) * mpad + tx + 16 * q] = acc2[i][q];
      acc2[i][q] = 0.f;
    }
}

// Pass 2 / predict: one CTA per 128 data rows; runs over the feature slots of
// every column block.  per_block: write O'_ij at the end of each block j (to
// out + j * out_block_stride); else accumulate over all blocks and write once.
// For m_pad <= 64 each 64-feature tile's FP32 sum is folded into a float-float
// accumulator (TwoSum): a 4096-feature block then carries the error of one 64-term
// sum, not of a 4096-term one (the outer form's W' = c + Z^T P (V - Z c) takes the
// rounding of Z c with gain ~1 relative to |Z c|, which exceeds |W'|).
template <int MQ>
__global__ void __launch_bounds__(NT, 1) k_pass2_simt(PassArgs p) {
  constexpr bool COMP = MQ <= 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SimtSmem& sm = *reinterpret_cast<SimtSmem*>(smem_raw);
  float* Ms = reinterpret_cast<float*>(smem_raw + sizeof(SimtSmem));
  const int64_t a0 = (int64_t)blockIdx.x * BM;
  // row block of this tile: the chain operand W'_ij depends on it
  int rb = 0;
  while (rb + 1 < p.R && p.row_slot[rb + 1] <= a0) ++rb;
  const uint8_t* act = p.bmask ? p.bmask + rb * p.C : nullptr;   // skip inactive blocks (per_block)
  const float* M = p.M + rb * p.m_block_stride;
  if (!RFF_SPAN(a0, BM, p.x_rows)) return;
  float acc2[8][MQ];
  float shi[COMP ? 8 : 1][COMP ? MQ : 1], slo[COMP ? 8 : 1][COMP ? MQ : 1];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int q = 0; q < MQ; ++q) acc2[i][q] = 0.f;
  if (COMP) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int q = 0; q < MQ; ++q) shi[COMP ? i : 0][COMP ? q : 0] = slo[COMP ? i : 0][COMP ? q : 0] = 0.f;
  }
  for (int j = 0; j < p.C; ++j) {
    if (act && !act[j]) continue;
    const int64_t f0 = p.col_slot[j], f1 = f0 + p.col_size[j];
    for (int64_t b0 = f0; b0 < f1; b0 += BN) {
      if (!RFF_SPAN(b0, BN, p.g_rows) || !RFF_SPAN(rb * p.m_block_stride + b0 * p.mpad, BN * p.mpad, p.m_elems))
        return;
      tile_z(sm, p.X, p.ldx, a0, p.Gt, p.ldg, b0, p.K, p.bias, false, p.scale, p.row_ok, p.feat_ok, p.map);
      load_M(Ms, M, b0, p.mpad);
      __syncthreads();
      chain<MQ>(sm, Ms, p.mpad, acc2);
      if (COMP) {
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int q = 0; q < MQ; ++q) {
            float& h = shi[COMP ? i : 0][COMP ? q : 0];
            float& l = slo[COMP ? i : 0][COMP ? q : 0];
            two_sum_into(h, l, acc2[i][q]);
            acc2[i][q] = 0.f;
          }
      }
    }
    if (COMP) {   // the block's sum back into acc2 for the store (or the next block)
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int q = 0; q < MQ; ++q) {
          float& h = shi[COMP ? i : 0][COMP ? q : 0];
          float& l = slo[COMP ? i : 0][COMP ? q : 0];
          if (p.per_block) {
            acc2[i][q] = h + l;
            h = l = 0.f;
          }
        }
    }
    if (p.per_block && RFF_SPAN(j * p.out_block_stride + a0 * p.mpad, BM * p.mpad, p.out_elems))
      store_acc<MQ>(acc2, p.out + j * p.out_block_stride, a0, p.mpad);
  }
  if (COMP && !p.per_block) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int q = 0; q < MQ; ++q) acc2[i][q] = shi[COMP ? i : 0][COMP ? q : 0] + slo[COMP ? i : 0][COMP ? q : 0];
  }
  if (!p.per_block && RFF_SPAN(a0 * p.mpad, BM * p.mpad, p.out_elems)) store_acc<MQ>(acc2, p.out, a0, p.mpad);
}

// Pass 1: one CTA per (128 feature slots, row block i, row split); runs over the
// data rows of its split in 64-row steps.  Writes R-partials (features x m_pad).
template <int MQ>
__global__ void __launch_bounds__(NT, 1) k_pass1_simt(PassArgs p) {
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
  const int64_t r0 = p.row_slot[i], nsteps = ceil_div(p.row_size[i], BN);
  const int64_t t0 = split * nsteps / p.nsplit, t1 = (split + 1) * nsteps / p.nsplit;
  const float* M = p.M + j * p.m_block_stride;
  if (!RFF_SPAN(a0, BM, p.g_rows)) return;
  float acc2[8][MQ];
#pragma unroll
  for (int ii = 0; ii < 8; ++ii)
#pragma unroll
    for (int q = 0; q < MQ; ++q) acc2[ii][q] = 0.f;
  for (int64_t t = t0; t < t1; ++t) {
    const int64_t b0 = r0 + t * BN;
    if (!RFF_SPAN(b0, BN, p.x_rows) || !RFF_SPAN(j * p.m_block_stride + b0 * p.mpad, BN * p.mpad, p.m_elems))
      return;
    tile_z(sm, p.Gt, p.ldg, a0, p.X, p.ldx, b0, p.K, p.bias, true, p.scale, p.feat_ok, p.row_ok, p.map);
    load_M(Ms, M, b0, p.mpad);
    __syncthreads();
    chain<MQ>(sm, Ms, p.mpad, acc2);
  }
  const int64_t o = ((int64_t)split * p.R + i) * p.out_block_stride;
  if (RFF_SPAN(o + a0 * p.mpad, BM * p.mpad, p.out_elems)) store_acc<MQ>(acc2, p.out + o, a0, p.mpad);
}

// Materialise Z for rows [r0, r0 + nr) and feature slots [f0, f0 + nf) into
// out (nr x nf, leading dimension ldo); one CTA per 128 x 64 tile.
__global__ void __launch_bounds__(NT, 1) k_write_z_simt(ZArgs p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SimtSmem& sm = *reinterpret_cast<SimtSmem*>(smem_raw);
  const int64_t a0 = p.r0 + (int64_t)blockIdx.x * BM, b0 = p.f0 + (int64_t)blockIdx.y * BN;
  tile_z(sm, p.X, p.ldx, a0, p.Gt, p.ldg, b0, p.K, p.bias, false, p.scale, p.row_ok, p.feat_ok, p.map);
  for (int t = threadIdx.x; t < BM * BN; t += NT) {
    const int r = t / BN, c = t % BN;
    const int64_t gr = a0 - p.r0 + r, gc = b0 - p.f0 + c;
    if (gr < p.nr && gc < p.nf) p.out[gr * p.ldo + gc] = sm.ZsT[c][r];
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
  if (p.K % BK) return cudaErrorInvalidValue;
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
  if (p.K % BK) return cudaErrorInvalidValue;
  const size_t smem = sizeof(SimtSmem);
  cudaFuncSetAttribute(k_write_z_simt, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((unsigned)ceil_div(p.nr, BM), (unsigned)ceil_div(p.nf, BN));
  k_write_z_simt<<<grid, NT, smem, st>>>(p);
  return cudaGetLastError();
}

RFF_CHECK_UNIT(regen_simt)

}  // namespace rff
