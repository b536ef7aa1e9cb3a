// Split-BF16 streaming GEMM on tensor cores, driven by a job table.
//
// Every job multiplies one 128-row tile of operand A (rows a_row.., K from a_k0)
// by the m_pad-row operand B (rows b_row.., K from b_k0) over nk chunks of 32:
//
//   acc (TMEM, 128 x m_pad fp32) = sum over the split products A_s . B_t^T
//
// with A = A1 + A2 (+ A3) and B = B1 + B2 (+ B3) split into 16-bit terms.  Three
// BF16 terms each (NA = NB = 3) take the six products whose exponents sum to at
// most 2^-16 (11, 12, 21, 13, 22, 31): the accuracy of an FP32 product.  Two
// terms each (scaled FP16 hi/lo, 22 significant bits) take 11, 12, 21.  The
// accumulator times out_scale (and the inverse FP16 scale of B, from the device
// maximum b_amax) is written row-major to out + job.out (ld m_pad); amax, when
// given, collects max |result| for the FP16 split of the result that follows.
//
// Users: the cached projection of eq. (gpWij) (A = Q_ij split three ways, B = the
// right-hand side), and the two chained products of the cached-Z precision
// (pass 1: A = Z^T, B = V^T; pass 2: A = Z, B = W'^T; eq. (gpWij), (gpOij)).
//
// A TMA ring of 32-element K chunks (64-byte swizzle), or 64-element ones (128-byte
// swizzle), feeds the tiles of each chunk.  Warp 0 issues the copies, one thread of warp 1
// the MMAs, warps 2..9 write the result.  Waits are bounded as in the regeneration kernel: on a timeout
// the CTA records an error code, waits (bounded) for its copies and products in
// flight, frees TMEM and returns.
#include <algorithm>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "tc.h"
#include "tcgen05.cuh"

namespace rff {

namespace {

using namespace tc5;

constexpr int QKC = 32;                      // K elements of a job's chunk count (SgJob::nk)
constexpr int QMAXS = 8;
constexpr int QEPI = 8;                      // writing warps: two per TMEM lane quarter, half the columns each
constexpr int QNT = 64 + 32 * QEPI;
constexpr int ERR_Q = 8;

struct QArgs {
  CUtensorMap tA[3], tB[3];
  int mpad, ns;
  uint32_t stage_bytes, tmem_cols;
  uint32_t acc_b;            // column of the second accumulator (the small products), 0 = one accumulator
  uint32_t nbuf;             // accumulator sets in TMEM (2: the next job's products overlap the epilogue)
  uint32_t buf_cols;         // TMEM columns of one set
  int njobs;
  const SgJob* jobs;
  float* out;
  int64_t out_elems;
  float out_scale;
  const unsigned* b_amax;
  unsigned* amax;
  const uint8_t* bmask;      // active blocks of a stochastic iteration, or null
  int accumulate;            // 1: out += result (amax of the sum)
  int* err;
  long long timeout_cycles;
};

struct QShared {
  uint64_t full[QMAXS], empty[QMAXS];
  uint64_t acc_full[2], acc_empty[2], mma_done;
  uint32_t tmem;
  int abort_flag;
};

__device__ __forceinline__ bool qwait(uint32_t bar, uint32_t parity, QShared& sh, const QArgs& a) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try(bar, parity)) return true;
    if (*(volatile int*)&sh.abort_flag) return false;
    if (clock64() - t0 > a.timeout_cycles) {
      *(volatile int*)&sh.abort_flag = 1;
      atomicOr(a.err, ERR_Q);
      return false;
    }
  }
}

// split-product order (A term, B term): exponents summing to at most 2^-16
__host__ __device__ constexpr int prod_a(int p) { return p == 2 || p == 4 ? 1 : p == 5 ? 2 : 0; }
__host__ __device__ constexpr int prod_b(int p) { return p == 1 || p == 4 ? 1 : p == 3 ? 2 : 0; }

// A job is skipped by every role alike when it has no K chunks or its block is inactive.
__device__ __forceinline__ bool q_skip(const SgJob& j, const QArgs& a) {
  return j.nk <= 0 || (a.bmask && !a.bmask[j.blk]);
}

// Each CTA takes the jobs blockIdx.x, blockIdx.x + gridDim.x, ... (one job per CTA when the
// grid covers the table).  The copies run ahead through the ring across jobs; a job's products
// go to accumulator set (its count) mod nbuf, which the writing warps free after reading it.
// KC: K elements per ring stage, 32 (64-byte rows, 64-byte swizzle) or 64 (128-byte rows and
// swizzle: fewer shared-memory wavefronts per product, half as many stages); a job's nk counts
// chunks of 32, so with KC = 64 an odd count reads 32 more K columns, which the caller keeps
// zero in A (or beyond the tensor, where the copy fills zeros).
template <int NA, int NB, int F16, int KC>
__global__ void __launch_bounds__(QNT) k_split_gemm(const __grid_constant__ QArgs a) {
  constexpr int NPROD = (NA == 3 && NB == 3) ? 6 : 3;
  constexpr uint32_t ATILE = 128 * KC * 2;                  // one 128-row A term
  constexpr uint32_t SBO = 8 * KC * 2, LAYOUT = KC == 64 ? 2 : 4;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  QShared& sh = *reinterpret_cast<QShared*>(base + a.ns * a.stage_bytes);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t bar_full = smem_u32(&sh.full[0]), bar_empty = smem_u32(&sh.empty[0]);
  const uint32_t bar_accf = smem_u32(&sh.acc_full[0]), bar_acce = smem_u32(&sh.acc_empty[0]);
  const uint32_t bar_done = smem_u32(&sh.mma_done);
  const uint32_t mb = (uint32_t)a.mpad * (KC * 2);   // one B term: m_pad rows
  if (threadIdx.x == 0) {
    sh.abort_flag = 0;
    for (int i = 0; i < a.ns; ++i) {
      mbar_init(bar_full + 8 * i, 1);
      mbar_init(bar_empty + 8 * i, 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(bar_accf + 8 * i, 1);
      mbar_init(bar_acce + 8 * i, QEPI);   // one arrival per writing warp
    }
    mbar_init(bar_done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&sh.tmem)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sh.tmem;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t issued = 0;   // ring stages filled, over all of this CTA's jobs
      bool ok = true;
      for (int jx = blockIdx.x; ok && jx < a.njobs; jx += gridDim.x) {
        const SgJob job = a.jobs[jx];
        if (q_skip(job, a)) continue;
        const int nkc = (job.nk * QKC + KC - 1) / KC;   // stages of KC elements
        for (int kc = 0; kc < nkc; ++kc) {
          const int st = issued % a.ns;
          const uint32_t use = issued / a.ns;
          if (use > 0 && !qwait(bar_empty + 8 * st, (use - 1) & 1, sh, a)) {
            ok = false;
            break;
          }
          const uint32_t fb = bar_full + 8 * st;
          mbar_expect_tx(fb, a.stage_bytes);
          const uint32_t dst = smem_u32(base + st * a.stage_bytes);
#pragma unroll
          for (int s = 0; s < NA; ++s) tma_load_2d(dst + s * ATILE, &a.tA[s], job.a_k0 + kc * KC, job.a_row, fb);
#pragma unroll
          for (int s = 0; s < NB; ++s)
            tma_load_2d(dst + NA * ATILE + s * mb, &a.tB[s], job.b_k0 + kc * KC, job.b_row, fb);
          ++issued;
        }
      }
      // copies in flight finish before the CTA may exit (bounded)
      for (uint32_t u = issued > (uint32_t)a.ns ? issued - a.ns : 0; u < issued; ++u) {
        const int st = u % a.ns;
        const long long t0 = clock64();
        while (!mbar_try(bar_full + 8 * st, (u / a.ns) & 1) && clock64() - t0 < a.timeout_cycles) {
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = F16 ? idesc_f16(128, a.mpad) : idesc_bf16(128, a.mpad);
      bool ok = true;
      uint32_t used = 0, done_jobs = 0;   // ring stages consumed, jobs multiplied
      for (int jx = blockIdx.x; ok && jx < a.njobs; jx += gridDim.x) {
        const SgJob job = a.jobs[jx];
        if (q_skip(job, a)) continue;
        const uint32_t buf = done_jobs % a.nbuf, round = done_jobs / a.nbuf;
        if (round > 0 && !qwait(bar_acce + 8 * buf, (round - 1) & 1, sh, a)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t acc = tmem + buf * a.buf_cols;
        const int nkc = (job.nk * QKC + KC - 1) / KC;   // stages of KC elements
        for (int kc = 0; kc < nkc; ++kc, ++used) {
          const int st = used % a.ns;
          if (!qwait(bar_full + 8 * st, (used / a.ns) & 1, sh, a)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t sa = smem_u32(base + st * a.stage_bytes);
          const uint32_t sb = sa + NA * ATILE;
#pragma unroll
          for (int kk = 0; kk < KC / 16; ++kk) {
#pragma unroll
            for (int p = 0; p < NPROD; ++p) {
              const uint64_t da = smem_desc(sa + prod_a(p) * ATILE + kk * 32, SBO, LAYOUT);
              const uint64_t db = smem_desc(sb + prod_b(p) * mb + kk * 32, SBO, LAYOUT);
              if (a.acc_b) {
                // hi.hi alone in the first accumulator, the smaller products in the second
                const uint32_t d = p == 0 ? acc : acc + a.acc_b;
                mma_bf16(d, da, db, idesc, (kc > 0 || kk > 0 || p > 1) ? 1u : 0u);
              } else {
                mma_bf16(acc, da, db, idesc, (kc > 0 || kk > 0 || p > 0) ? 1u : 0u);
              }
            }
          }
          mma_commit(bar_empty + 8 * st);
        }
        if (!ok) break;
        mma_commit(bar_accf + 8 * buf);
        ++done_jobs;
      }
      mma_commit(bar_done);
      qwait(bar_done, 0, sh, a);
    }
  } else {
    // epilogue: lanes = rows of the A tile; warps 2..5 take the first m_pad/2 columns, warps
    // 6..9 the rest, 8 per TMEM read
    const int quarter = warp & 3;
    const int c_begin = ((warp - 2) >> 2) * (a.mpad / 2), c_end = c_begin + a.mpad / 2;
    const int row = quarter * 32 + lane;
    uint32_t done_jobs = 0;
    float mx = 0.f;
    for (int jx = blockIdx.x; jx < a.njobs; jx += gridDim.x) {
      const SgJob job = a.jobs[jx];
      if (q_skip(job, a)) continue;
      const uint32_t buf = done_jobs % a.nbuf, round = done_jobs / a.nbuf;
      int ok = 0;
      if (lane == 0) ok = qwait(bar_accf + 8 * buf, round & 1, sh, a) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) break;
      fence_after();
      const uint32_t taddr = tmem + buf * a.buf_cols + ((uint32_t)(quarter * 32) << 16);
      float* orow_p = a.out + job.out + (int64_t)row * a.mpad;
      const float sc = a.out_scale * (a.b_amax ? f16_inv_scale(__uint_as_float(*a.b_amax)) : 1.f);
      for (int c = c_begin; c < c_end; c += 8) {
        uint32_t r8[8], s8[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        tmem_ld8(taddr + c, r8);
        if (a.acc_b) tmem_ld8(taddr + a.acc_b + c, s8);
        tmem_wait_ld();
        float x[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) x[t] = sc * (__uint_as_float(r8[t]) + __uint_as_float(s8[t]));
        float4* dst = reinterpret_cast<float4*>(orow_p + c);
        const bool in = RFF_SPAN(job.out + (int64_t)row * a.mpad + c, 8, a.out_elems);
        if (a.accumulate && in) {
          const float4 p0 = dst[0], p1 = dst[1];
          x[0] += p0.x; x[1] += p0.y; x[2] += p0.z; x[3] += p0.w;
          x[4] += p1.x; x[5] += p1.y; x[6] += p1.z; x[7] += p1.w;
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) mx = fmaxf(mx, fabsf(x[t]));
        if (in) {
          dst[0] = make_float4(x[0], x[1], x[2], x[3]);
          dst[1] = make_float4(x[4], x[5], x[6], x[7]);
        }
      }
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(bar_acce + 8 * buf);   // the set is free for the job after next
      ++done_jobs;
    }
    if (a.amax) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
      if (lane == 0 && mx > 0.f) atomicMax(a.amax, __float_as_uint(mx));
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols) : "memory");
  }
}

// ---- the right-hand side, split three ways and transposed: rT_t[i][c][slot]
__global__ void k_rhs_split3T(const float* __restrict__ Wbar, const float* __restrict__ muij,
                              const float* __restrict__ Rpart, int nsplit, int R, int64_t fslots, int mpad,
                              const int32_t* __restrict__ feat_ok, const float* __restrict__ What,
                              __nv_bfloat16* __restrict__ r1, __nv_bfloat16* __restrict__ r2,
                              __nv_bfloat16* __restrict__ r3) {
  __shared__ float tile[32][33];
  const int i = blockIdx.z;
  const int64_t p0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;   // 256 threads
  const int64_t nfe = fslots * mpad;
  for (int rr = ty; rr < 32; rr += 8) {
    const int64_t p = p0 + rr;
    const int c = c0 + tx;
    float v = 0.f;
    if (p < fslots && c < mpad && feat_ok[p] >= 0) {
      const int64_t e = p * mpad + c, t = (int64_t)i * nfe + e;
      v = Wbar[e] - muij[t];
      if (What) v -= What[t];
      for (int sp = 0; sp < nsplit; ++sp)
        if (RFF_IN((int64_t)sp * R * nfe + t, (int64_t)nsplit * R * nfe)) v += Rpart[(int64_t)sp * R * nfe + t];
    }
    tile[rr][tx] = v;
  }
  __syncthreads();
  for (int cc = ty; cc < 32; cc += 8) {
    const int c = c0 + cc;
    const int64_t p = p0 + tx;
    if (c < mpad && p < fslots) {
      const float x = tile[tx][cc];
      const __nv_bfloat16 h = __float2bfloat16_rn(x);
      const float rem = x - __bfloat162float(h);
      const __nv_bfloat16 m = __float2bfloat16_rn(rem);
      const __nv_bfloat16 l = __float2bfloat16_rn(rem - __bfloat162float(m));
      const int64_t o = ((int64_t)i * mpad + c) * fslots + p;
      if (!RFF_IN(o, (int64_t)R * mpad * fslots)) continue;
      r1[o] = h;
      r2[o] = m;
      r3[o] = l;
    }
  }
}

// ---- one block's Q (s x s, float64) into the three split arrays at row qrow
__global__ void k_split3_q(const double* __restrict__ Q, int s, int64_t ldq, int64_t qrow,
                           __nv_bfloat16* __restrict__ q1, __nv_bfloat16* __restrict__ q2,
                           __nv_bfloat16* __restrict__ q3) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)s * s) return;
  const int64_t r = t / s, c = t % s;
  const double x = Q[t];
  const uint64_t b = (uint64_t)__double_as_longlong(x);
  const int E = (int)((b >> 52) & 0x7ff);
  __nv_bfloat16 h, m, l;
  if (E >= 1023 - 64 && E <= 1023 + 64) {   // 2^-64 <= |x| < 2^65: every power below is a normal FP32
    // x = t + rs: t its leading 24 bits as an FP32 number and rs the remaining 29 (both exact,
    // built by integer instructions: this part's FP64 pipe runs at 1/64 of the FP32 rate);
    // then h = bf16(t), and m, l the BF16 terms of (t - h) + rs, whose FP32 rounding lies
    // below 2^-32 |x|
    const uint32_t sgn = (uint32_t)(b >> 32) & 0x80000000u;
    const float t32 = __uint_as_float(sgn | ((uint32_t)(E - 1023 + 127) << 23) | (uint32_t)((b >> 29) & 0x7fffffu));
    const float r32 = __uint2float_rn((uint32_t)(b & 0x1fffffffu)) * __uint_as_float((uint32_t)(E - 1075 + 127) << 23);
    h = __float2bfloat16_rn(t32);
    const float rem = __fadd_rn(__fsub_rn(t32, __bfloat162float(h)), sgn ? -r32 : r32);
    m = __float2bfloat16_rn(rem);
    l = __float2bfloat16_rn(__fsub_rn(rem, __bfloat162float(m)));
  } else {   // zero, tiny, huge or not finite: the FP64 route
    h = __double2bfloat16(x);
    const double rem = x - (double)__bfloat162float(h);
    m = __double2bfloat16(rem);
    l = __double2bfloat16(rem - (double)__bfloat162float(m));
  }
  const int64_t o = (qrow + r) * ldq + c;
  q1[o] = h;
  q2[o] = m;
  q3[o] = l;
}

int qsm_count() {
  static int n = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
      v = 0;
    return v > 0 ? v : 1;
  }();
  return n;
}

template <int NA, int NB, int F16, int KC>
cudaError_t set_smem_attr() {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(k_split_gemm<NA, NB, F16, KC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                1024 + 216 * 1024 + 256);
  });
  return attr;
}

}  // namespace

cudaError_t launch_split3_q(const double* Q, int s, int64_t ldq, int64_t qrow, __nv_bfloat16* q1,
                            __nv_bfloat16* q2, __nv_bfloat16* q3, cudaStream_t st) {
  const int64_t n = (int64_t)s * s;
  if (n <= 0) return cudaSuccess;
  k_split3_q<<<(unsigned)ceil_div(n, 256), 256, 0, st>>>(Q, s, ldq, qrow, q1, q2, q3);
  return cudaGetLastError();
}

cudaError_t launch_rhs_split3T(const float* Wbar, const float* muij, const float* Rpart, int nsplit, int R,
                               int64_t fslots, int mpad, const int32_t* feat_ok, __nv_bfloat16* r1,
                               __nv_bfloat16* r2, __nv_bfloat16* r3, cudaStream_t st, const float* What) {
  dim3 grid((unsigned)ceil_div(fslots, 32), (unsigned)ceil_div(mpad, 32), (unsigned)R);
  k_rhs_split3T<<<grid, 256, 0, st>>>(Wbar, muij, Rpart, nsplit, R, fslots, mpad, feat_ok, What, r1, r2, r3);
  return cudaGetLastError();
}

cudaError_t split_gemm(const SgView& v) {
  if (v.njobs <= 0) return cudaSuccess;
  if (v.mpad > 256 || v.mpad < 16 || v.mpad % 16) return cudaErrorInvalidValue;
  if (!((v.na == 3 && v.nb == 3 && !v.f16) || (v.na == 2 && v.nb == 2 && v.f16))) return cudaErrorInvalidValue;
  QArgs a;
  memset(&a, 0, sizeof(a));
  cudaError_t e;
  const size_t budget = std::min<size_t>(v.smem_budget ? v.smem_budget : 216 * 1024, 216 * 1024);
  // 64-element stages only where two of them fit (m_pad = 256 with three terms does not)
  const int kc = (v.kc == 64 && 2 * (size_t)(v.na * 128 + v.nb * v.mpad) * 64 * 2 <= budget) ? 64 : 32;
  for (int s = 0; s < v.na; ++s)
    if ((e = tc_make_map_bf16(&a.tA[s], v.A[s], v.a_cols, v.a_rows, v.a_cols, 128, kc)) != cudaSuccess) return e;
  for (int s = 0; s < v.nb; ++s)
    if ((e = tc_make_map_bf16(&a.tB[s], v.B[s], v.b_cols, v.b_rows, v.b_cols, v.mpad, kc)) != cudaSuccess)
      return e;
  a.mpad = v.mpad;
  a.stage_bytes = (uint32_t)(v.na * 128 + v.nb * v.mpad) * kc * 2;
  a.ns = (int)std::min<size_t>(QMAXS, budget / a.stage_bytes);
  if (a.ns < 2) a.ns = 2;
  a.tmem_cols = v.mpad <= 32 ? 32 : v.mpad <= 64 ? 64 : v.mpad <= 128 ? 128 : 256;
  if (v.two_acc) {
    // the tensor cores' FP32 accumulator rounds toward zero at every accumulation: the
    // dominant hi.hi products get an accumulator of their own (K/16 accumulations instead of
    // NPROD K/16), the small products share the second, and the two are added in FP32
    a.acc_b = a.tmem_cols;
    a.tmem_cols *= 2;
  }
  a.jobs = v.jobs;
  a.njobs = v.njobs;
  a.out = v.out;
  a.out_elems = v.out_elems;
  a.out_scale = v.out_scale;
  a.b_amax = v.b_amax;
  a.amax = v.amax;
  a.bmask = v.bmask;
  a.accumulate = v.accumulate;
  a.err = tc_error_ptr();
  if (!a.err) return cudaErrorMemoryAllocation;
  a.timeout_cycles = 4000000000LL;   // about two seconds at the boost clock
  const size_t smem = 1024 + (size_t)a.ns * a.stage_bytes + 256;
  // the four instances: BF16 three-term or FP16 two-term operands, 32- or 64-element stages
  auto kern = [&]() -> const void* {
    if (v.na == 3) return kc == 64 ? (const void*)k_split_gemm<3, 3, 0, 64> : (const void*)k_split_gemm<3, 3, 0, 32>;
    return kc == 64 ? (const void*)k_split_gemm<2, 2, 1, 64> : (const void*)k_split_gemm<2, 2, 1, 32>;
  };
  if (v.na == 3)
    e = kc == 64 ? set_smem_attr<3, 3, 0, 64>() : set_smem_attr<3, 3, 0, 32>();
  else
    e = kc == 64 ? set_smem_attr<2, 2, 1, 64>() : set_smem_attr<2, 2, 1, 32>();
  if (e != cudaSuccess) return e;
  // one job per CTA, or (persistent) at most as many CTAs as fit on the device at once, each
  // taking every grid-th job; two accumulator sets when the tensor memory of the CTAs that
  // share an SM holds them
  a.buf_cols = a.tmem_cols;
  a.nbuf = 1;
  int64_t grid = v.njobs;
  if (v.persistent) {
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern(), QNT, smem);
    if (e != cudaSuccess) return e;
    per_sm = std::max(per_sm, 1);
    grid = std::min<int64_t>(v.njobs, (int64_t)qsm_count() * per_sm);
    if (2u * a.tmem_cols * (uint32_t)per_sm <= 512u) {
      a.nbuf = 2;
      a.tmem_cols *= 2;
    }
  }
  if (v.na == 3) {
    if (kc == 64) k_split_gemm<3, 3, 0, 64><<<(unsigned)grid, QNT, smem, v.st>>>(a);
    else k_split_gemm<3, 3, 0, 32><<<(unsigned)grid, QNT, smem, v.st>>>(a);
  } else {
    if (kc == 64) k_split_gemm<2, 2, 1, 64><<<(unsigned)grid, QNT, smem, v.st>>>(a);
    else k_split_gemm<2, 2, 1, 32><<<(unsigned)grid, QNT, smem, v.st>>>(a);
  }
  return cudaGetLastError();
}

RFF_CHECK_UNIT(qgemm)

}  // namespace rff
