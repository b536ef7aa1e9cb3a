// TensorSketch features of the polynomial kernel k(x, y) = (<x, y> / sigma^2 + c)^q (Sec. 4
// lists TensorSketch among the solver's maps; Pham and Pagh, KDD 2013).
//
// With x' = (x / sigma, sqrt(c)) (d + 1 entries), column block j (S = s_j features) carries its
// own sketch TS_j(x) = CS_1(x') * ... * CS_q(x'): q CountSketches of length S combined by
// circular convolution, CS_p(x')[t] = sum over i with h_p(i) = t of g_p(i) x'_i.  A map that
// must produce its whole transformed vector is assembled from independent per-block maps
// (Sec. 4), so Z[:, block j] = sqrt(S / D) TS_j(X).
//
// Stream layout: for block j, degree p (0-based) and augmented entry i, Philox counter
// (j, p (d + 1) + i, 7, 0): h = (w0 S) >> 32, g = -1 if the top bit of w1 is set, else +1.
//
// One CTA per (group of rows, block j): the block's hashes and signs, and the bucket lists of
// the first CountSketch (the entries of every bucket in increasing i), are built in shared
// memory once; then, row by row, the first sketch is gathered bucket by bucket and each further
// degree is one circular convolution with a sparse CountSketch, computed in pull form
//   next[t] = sum over i (increasing) of g_p(i) x'_i acc[(t - h_p(i)) mod S],
// so that every output is one FP32 chain in a fixed order: the result does not depend on the
// launch geometry, and no atomics touch the values.  The running sketch is kept twice in a row
// (acc[t] = acc[t + S]), so acc[(t - h) mod S] = acc[t - h + S] needs no wrap test: for each
// entry i a thread forms one address and reads its outputs' operands at fixed offsets from it,
// one shared-memory load and one FMA per multiply-add.
#include "common.cuh"
#include "internal.h"

namespace rff {

namespace {

constexpr int TS_NT = 256;

struct TsSmem {
  int32_t* hsh;    // q x (d+1)
  float* sgn;      // q x (d+1)
  float* xs;       // d+1
  int32_t* bptr;   // S+1: bucket starts of the first CountSketch
  int32_t* bitem;  // d+1: its entries, bucket by bucket, increasing i
  float* acc;      // 2 S: the running sketch, twice
  float* nxt;      // 2 S
};

__device__ __forceinline__ TsSmem ts_carve(unsigned char* raw, int q, int d1, int S) {
  TsSmem m;
  m.hsh = reinterpret_cast<int32_t*>(raw);
  m.sgn = reinterpret_cast<float*>(m.hsh + q * d1);
  m.xs = m.sgn + q * d1;
  m.bptr = reinterpret_cast<int32_t*>(m.xs + d1);
  m.bitem = m.bptr + (S + 1);
  m.acc = reinterpret_cast<float*>(m.bitem + d1);
  m.nxt = m.acc + 2 * S;
  return m;
}

template <int KT>
__global__ void __launch_bounds__(TS_NT) k_tensorsketch(TsArgs a) {
  extern __shared__ __align__(16) unsigned char ts_raw[];
  const int j = a.j0 + (int)blockIdx.y;
  const int S = (int)a.col_size[j], d1 = a.d + 1, q = a.q;
  const int64_t fcol = a.col_slot[j] - a.f_base;          // out column of the block's feature 0
  const int SP = a.pad ? (int)round_up(S, SLOT) : S;       // columns written (padding as zeros)
  const float scale = (float)sqrt((double)S / (double)a.D);
  TsSmem m = ts_carve(ts_raw, q, d1, S);
  const int tid = threadIdx.x;
  for (int e = tid; e < q * d1; e += TS_NT) {
    const U4 w = philox4x32_10(U4{(uint32_t)j, (uint32_t)e, 7u, 0u}, a.k0, a.k1);
    m.hsh[e] = (int32_t)(((uint64_t)w.x * (uint64_t)S) >> 32);
    m.sgn[e] = (w.y >> 31) ? -1.f : 1.f;
  }
  __syncthreads();
  // bucket lists of the first sketch: thread t counts bucket t, a scan gives the starts, and
  // thread t then lists its bucket's entries in increasing i
  for (int t = tid; t < S; t += TS_NT) {
    int c = 0;
    for (int i = 0; i < d1; ++i) c += m.hsh[i] == t;
    m.bptr[t + 1] = c;
  }
  __syncthreads();
  if (tid == 0) {
    m.bptr[0] = 0;
    for (int t = 0; t < S; ++t) m.bptr[t + 1] += m.bptr[t];
  }
  __syncthreads();
  for (int t = tid; t < S; t += TS_NT) {
    int o = m.bptr[t];
    for (int i = 0; i < d1; ++i)
      if (m.hsh[i] == t) m.bitem[o++] = i;
  }
  __syncthreads();
  float zmax = 0.f;
  for (int64_t r = blockIdx.x; r < a.nr; r += gridDim.x) {
    const int64_t slot = a.r0 + r;
    const bool ok = a.row_ok ? a.row_ok[slot] >= 0 : true;   // the same for the whole CTA
    if (ok) {
      for (int i = tid; i < d1; i += TS_NT)
        m.xs[i] = (i < a.d) ? a.X[slot * a.ldx + i] * a.inv_sigma : a.sqrt_c;
      __syncthreads();
      for (int t = tid; t < S; t += TS_NT) {
        float v = 0.f;
        for (int k = m.bptr[t]; k < m.bptr[t + 1]; ++k) v = fmaf(m.sgn[m.bitem[k]], m.xs[m.bitem[k]], v);
        m.acc[t] = v;
        m.acc[t + S] = v;
      }
      __syncthreads();
      for (int p = 1; p < q; ++p) {
        float acc[KT];
#pragma unroll
        for (int k = 0; k < KT; ++k) acc[k] = 0.f;
        for (int i = 0; i < d1; ++i) {
          const float w = m.sgn[p * d1 + i] * m.xs[i];
          if (w == 0.f) continue;   // the same for every thread (sparse rows skip their zeros)
          const float* src = m.acc + (S - m.hsh[p * d1 + i]) + tid;   // acc[t - h + S] for t = tid
#pragma unroll
          for (int k = 0; k < KT; ++k)
            if (tid + TS_NT * k < S) acc[k] = fmaf(w, src[TS_NT * k], acc[k]);
        }
#pragma unroll
        for (int k = 0; k < KT; ++k) {
          const int t = tid + TS_NT * k;
          if (t < S) {
            m.nxt[t] = acc[k];
            m.nxt[t + S] = acc[k];
          }
        }
        __syncthreads();
        float* sw = m.acc;
        m.acc = m.nxt;
        m.nxt = sw;
      }
    }
    if (a.out) {
      float* orow = a.out + r * a.ldo + fcol;
      for (int t = tid; t < SP; t += TS_NT) {
        const float v = (ok && t < S) ? scale * m.acc[t] : 0.f;
        if (RFF_IN(r * a.ldo + fcol + t, a.out_elems)) orow[t] = v;
      }
    }
    if (ok)
      for (int t = tid; t < S; t += TS_NT) zmax = fmaxf(zmax, fabsf(scale * m.acc[t]));
    __syncthreads();   // acc and xs are rewritten by the next row
  }
  if (a.amax) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) zmax = fmaxf(zmax, __shfl_xor_sync(0xffffffffu, zmax, o));
    if ((tid & 31) == 0 && zmax > 0.f) atomicMax(a.amax, __float_as_uint(zmax));
  }
}

}  // namespace

size_t tensorsketch_smem_bytes(int q, int64_t d, int64_t S) {
  const int64_t d1 = d + 1;
  return (size_t)(q * d1 * 8 + d1 * 4 + (S + 1) * 4 + d1 * 4 + 4 * S * 4);
}

cudaError_t launch_tensorsketch(const TsArgs& a, int nblocks, int64_t smax, cudaStream_t st) {
  if (a.nr <= 0 || nblocks <= 0) return cudaSuccess;
  if (a.q < 1 || a.q > TS_MAX_DEGREE || smax < 1 || smax > TS_MAX_BLOCK) return cudaErrorInvalidValue;
  const size_t smem = tensorsketch_smem_bytes(a.q, a.d, smax);
  if (smem > TS_MAX_SMEM) return cudaErrorInvalidValue;
  int dev = 0, nsm = 148;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  cudaGetLastError();
  // about four CTAs per SM in all, each over a strided set of rows of one block
  const int64_t gx = std::max<int64_t>(1, std::min<int64_t>(a.nr, ceil_div(4 * (int64_t)nsm, nblocks)));
  const dim3 grid((unsigned)gx, (unsigned)nblocks);
  const int kt = (int)ceil_div(smax, TS_NT);
#define RFF_TS(K)                                                                                      \
  if (kt <= K) {                                                                                       \
    cudaError_t e = cudaFuncSetAttribute(k_tensorsketch<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                         (int)TS_MAX_SMEM);                                            \
    if (e != cudaSuccess) return e;                                                                    \
    k_tensorsketch<K><<<grid, TS_NT, smem, st>>>(a);                                                   \
    return cudaGetLastError();                                                                         \
  }
  RFF_TS(1) RFF_TS(2) RFF_TS(4) RFF_TS(8) RFF_TS(16) RFF_TS(32)
#undef RFF_TS
  return cudaErrorInvalidValue;
}

RFF_CHECK_UNIT(sketch)

}  // namespace rff
