// Blocked Cholesky factorisation and inverse of eq. (cache) with the block updates on the
// tensor cores, by error-free slicing of the FP64 operands (Ozaki, Ogita, Oishi and Rump,
// "Error-free transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).
//
// Every update of the factorisation is D = beta C + alpha A B^T with K <= 64, A (M x K) and
// B (N x K) given by rows.  Each row of an operand is scaled by a power of two 2^e (e: the
// smallest with every |x| < 2^e in the row) and cut into S = 6 slices of 8 bits,
//   x = 2^e sum_s a_s 2^(-8(s+1)) + r,   a_s integers, |a_s| <= 255,  0 <= |r| < 2^(e-48),
// (the 48 leading bits of the row's fixed-point form, sign and magnitude), each a_s exact in
// FP16.  The product of slices s and t summed over K = 64 is an integer of at most
// 64 * 255^2 = 4,161,600; one TMEM accumulator per c = 0..5 takes the 21 pairs with s + t = c.
// For c <= 3 (at most 4 pairs) every partial sum stays within 4 * 4,161,600 < 2^24: the
// tensor cores' FP32 accumulator holds it exactly, whatever the order or the rounding of its
// additions.  The accumulators of c = 4, 5 (weights 2^-32, 2^-40) may pass 2^24 and lose at
// most one unit per product instruction (K = 16 each, 44 in all), below 2^-49 of
// max|A_r| max|B_c| K; the dropped pairs (s + t >= 6) and the slicing remainders weigh about
// 2^-45 of it together.  The epilogue adds the six integers with their weights 2^(-8c) in
// double-float (TwoSum), scales the pair by 2^(e_A + e_B - 16) through the exponent field and
// adds it to C in FP64: two FP64 additions per element, the only work done on this part's
// FP64 pipe (1/64 of the FP32 rate).  Six slices of 8 bits take 84 product instructions per
// 128 x 32 tile where seven of 7 bits (the same accuracy) would take 112: at N = 32 the tensor
// cores' instruction issue, not their arithmetic, bounds the kernel.
//
// S = 6 (48 bits) serves the public Cholesky factorisation.  The solver's set-up stores the
// inverse to 24 bits (FP32, or three BF16 pieces) and takes S = 5: 40 bits, 15 pairs (60
// product instructions per tile), the accumulator of c = 4 the only one that may round; the
// inverse then stays within about cond(H) 2^-40 of its FP64 value.
//
// The 64 x 64 diagonal blocks are factored and inverted in FP64 (k_potrf_diag); the
// structure of the factorisation and of the inverse (forward sweep L Y = I, backward sweep
// L^T Q = Y over the block lower triangle, mirrored at the end) is that of the double-float
// driver in dense.cu.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tc.h"
#include "tcgen05.cuh"

namespace rff {

namespace {

using namespace tc5;

constexpr int OZ_SMAX = 6;                 // slices per operand row (S), at most
constexpr int OZ_BITS = 8;                 // bits per slice
constexpr int OZ_K = 64;                   // K of every update
constexpr int OZ_BM = 128, OZ_BN = 32;     // output tile (rows of A, columns of B)
constexpr int OZ_ITEM_COLS = 512;          // columns of one work item (16 tiles)
constexpr int OZ_ITEMS_PER_CTA = 2;        // work items a CTA takes in turn (at least one CTA per SM)
constexpr uint32_t OZ_ATILE = OZ_BM * OZ_K * 2;                // 16 KB: one slice of a 128-row block
constexpr uint32_t OZ_BTILE = OZ_BN * OZ_K * 2;                // 4 KB: one slice of a 32-column tile
// TMEM columns of one accumulator set, and the shared-memory tiles (144 KB at S = 6)
__host__ __device__ constexpr uint32_t oz_acols(int S) { return (uint32_t)S * OZ_BN; }
__host__ __device__ constexpr uint32_t oz_tiles(int S) { return (uint32_t)S * OZ_ATILE + 2u * S * OZ_BTILE; }
constexpr int OZ_BAD = 1 << 20;            // exponent recorded for a row holding an Inf or a NaN
constexpr int ERR_OZ = 16;
constexpr int OZ_EPI_WARPS = 16;          // four per TMEM lane quarter, 8 columns each
constexpr int OZ_THREADS = 32 * (2 + OZ_EPI_WARPS);   // warp 0 copies, warp 1 multiplies, the rest write D

struct OzSliceJob {
  const double* src;
  int64_t ld;
  int rows, kdim;
  int trans;          // 0: x[r][k] = src[r ld + k];  1: x[r][k] = src[k ld + r]
  __half* dst;        // S x rpad x 64: slice s of row r at (s rpad + r) 64
  int32_t* exps;      // rpad
};

struct OzJob {
  const double* C;
  double* D;
  int64_t ldc, ldd;
  int M, N;
  int a_row, b_row;   // tensor-map row of slice 0 of this job's A / B (slice s: + s rpad)
  const int32_t* ea;
  const int32_t* eb;
};

// one work item: rows m0 .. m0+127 of job `job` against the 32-column tiles n0 .. n1 of B
struct OzItem {
  int32_t job, m0, n0, n1;
};

struct OzArgs {
  CUtensorMap tA, tB;
  const OzJob* jobs;
  const OzItem* items;
  int nitems;
  int rpad;
  int neg;            // alpha = -1 (else +1)
  int beta;           // 1: D = C + alpha A B^T;  0: D = alpha A B^T
  int lower;          // write only the 64 x 64 tiles on or below the diagonal
  int* err;
  long long timeout_cycles;
};

struct OzShared {
  uint64_t a_full, a_empty, b_full[2], b_empty[2], acc_full[2], acc_empty[2], done;
  uint32_t tmem;
  int abort_flag;
};

// the fbits-bit fixed-point magnitude of x (bits b, biased exponent e) in units of
// 2^(e_row - fbits), e_row = emax - 1022 the row's exponent: floor(|x| 2^(fbits - e_row))
__device__ __forceinline__ uint64_t oz_fixed(uint64_t b, int e, int emax, int fbits) {
  if (e == 0 || e == 0x7ff || emax == 0x7ff) return 0;   // zero or subnormal; Inf/NaN rows are flagged
  const uint64_t m = (b & ((1ull << 52) - 1)) | (1ull << 52);
  const int sh = (53 - fbits) + emax - e;
  return sh >= 64 ? 0ull : m >> sh;
}

__device__ __forceinline__ __half oz_digit(uint64_t F, int sh, uint64_t b) {
  int v = (int)((F >> sh) & ((1u << OZ_BITS) - 1u));
  if (b >> 63) v = -v;
  return __int2half_rn(v);
}

template <int S>
__global__ void __launch_bounds__(256) k_oz_slice(const OzSliceJob* __restrict__ jobs, int rpad) {
  const OzSliceJob J = jobs[blockIdx.z];
  const int r0 = blockIdx.x * 32;
  if (!J.dst || r0 >= rpad) return;   // an empty job: this matrix ends before the step
  __shared__ double t[32][65];
  for (int idx = threadIdx.x; idx < 32 * 64; idx += 256) {
    int r, k;
    if (J.trans) {
      k = idx / 32;
      r = idx % 32;
    } else {
      r = idx / 64;
      k = idx % 64;
    }
    double x = 0.0;
    if (r0 + r < J.rows && k < J.kdim)
      x = J.trans ? J.src[(int64_t)k * J.ld + r0 + r] : J.src[(int64_t)(r0 + r) * J.ld + k];
    t[r][k] = x;
  }
  __syncthreads();
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
#pragma unroll 1
  for (int rr = 0; rr < 4; ++rr) {
    const int r = warp * 4 + rr;
    const uint64_t b0 = (uint64_t)__double_as_longlong(t[r][lane]);
    const uint64_t b1 = (uint64_t)__double_as_longlong(t[r][lane + 32]);
    const int e0 = (int)((b0 >> 52) & 0x7ff), e1 = (int)((b1 >> 52) & 0x7ff);
    const int emax = (int)__reduce_max_sync(0xffffffffu, (unsigned)max(e0, e1));
    const uint64_t F0 = oz_fixed(b0, e0, emax, S * OZ_BITS), F1 = oz_fixed(b1, e1, emax, S * OZ_BITS);
    const int64_t row = r0 + r;
#pragma unroll
    for (int s = 0; s < S; ++s) {
      const int sh = OZ_BITS * (S - 1 - s);
      const int64_t o = ((int64_t)s * rpad + row) * 64;
      if (RFF_SPAN(o, 64, (int64_t)S * rpad * 64)) {
        J.dst[o + lane] = oz_digit(F0, sh, b0);
        J.dst[o + lane + 32] = oz_digit(F1, sh, b1);
      }
    }
    if (lane == 0 && RFF_IN(row, rpad)) J.exps[row] = emax == 0x7ff ? OZ_BAD : (emax == 0 ? 0 : emax - 1022);
  }
}

__device__ __forceinline__ bool oz_wait(uint32_t bar, uint32_t parity, OzShared& sh, const OzArgs& a) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  while (true) {
    if (mbar_try_sleep(bar, parity, 20000)) return true;
    if (*(volatile int*)&sh.abort_flag) return false;
    if (clock64() - t0 > a.timeout_cycles) {
      *(volatile int*)&sh.abort_flag = 1;
      atomicOr(a.err, ERR_OZ);
      return false;
    }
  }
}

// sum over c of g[c] 2^(-8c) as a double-float (hi, lo), |lo| <= ulp(hi) / 2.  Every term is
// an FP32 number.  Those of c >= 4 (below 2^-8 in units of the leading integer's weight) are
// summed in plain FP32 (one rounding each, below 2^-32 of those units); the four leading ones
// are added by TwoSum, whose rounding errors are recovered in lo.  Against the bound
// max|A_r| max|B_c| K (about 2^22 units) the pair is accurate to about 2^-46.
template <int S>
__device__ __forceinline__ void oz_combine(const uint32_t (&g)[S][4], int j, float& hi, float& lo) {
  static_assert(S >= 5, "the four leading weights are summed by TwoSum");
  hi = 0.f;
#pragma unroll
  for (int c = S - 1; c >= 4; --c) hi = __fmaf_rn(__uint_as_float(g[c][j]), __int_as_float((127 - 8 * c) << 23), hi);
  lo = 0.f;
#pragma unroll
  for (int c = 3; c >= 0; --c) {
    const float w = c == 0 ? 1.f : c == 1 ? 0x1p-8f : c == 2 ? 0x1p-16f : 0x1p-24f;
    const float tv = __fmul_rn(__uint_as_float(g[c][j]), w);
    const float s = __fadd_rn(tv, hi);
    const float bb = __fsub_rn(s, tv);
    const float err = __fadd_rn(__fsub_rn(tv, __fsub_rn(s, bb)), __fsub_rn(hi, bb));
    hi = s;
    lo = __fadd_rn(lo, err);
  }
  const float s = __fadd_rn(hi, lo);
  lo = __fsub_rn(lo, __fsub_rn(s, hi));
  hi = s;
}

// Each CTA (one per SM at a time: the slices fill shared memory) takes a few work items in turn.  Per item warp 0 copies the six A
// slices of the row block once and the six B slices of each 32-column tile into a double
// buffer (TMA, 128-byte swizzle); one thread of warp 1 issues the 21 x 4 products of a tile
// into one of two TMEM accumulator sets (six 128 x 32 accumulators each); warps 2..17 read a
// finished set, update their 32 rows x 8 columns of D and free it, while the next tile's
// copies and products run.  Every wait is bounded: on a timeout the CTA records an error
// code, stops issuing, lets its copies and products in flight finish (bounded), frees TMEM and
// returns.
template <int S>
__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_rows(const __grid_constant__ OzArgs a) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  OzShared& sh = *reinterpret_cast<OzShared*>(base + oz_tiles(S));
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const uint32_t sa = smem_u32(base), sb = sa + S * OZ_ATILE;
  const uint32_t bar_a_full = smem_u32(&sh.a_full), bar_a_empty = smem_u32(&sh.a_empty);
  const uint32_t bar_b_full = smem_u32(&sh.b_full[0]), bar_b_empty = smem_u32(&sh.b_empty[0]);
  const uint32_t bar_acc_full = smem_u32(&sh.acc_full[0]), bar_acc_empty = smem_u32(&sh.acc_empty[0]);
  const uint32_t bar_done = smem_u32(&sh.done);
  if (threadIdx.x == 0) {
    sh.abort_flag = 0;
    mbar_init(bar_a_full, 1);
    mbar_init(bar_a_empty, 1);
    mbar_init(bar_done, 1);
    for (int i = 0; i < 2; ++i) {
      mbar_init(bar_b_full + 8 * i, 1);
      mbar_init(bar_b_empty + 8 * i, 1);
      mbar_init(bar_acc_full + 8 * i, 1);
      mbar_init(bar_acc_empty + 8 * i, OZ_EPI_WARPS);   // one arrival per writing warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc<1>(smem_u32(&sh.tmem), 512);
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = sh.tmem;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t it = 0, ni = 0;   // B tiles and A blocks whose copies were issued
      bool ok = true;
      for (int i = blockIdx.x; ok && i < a.nitems; i += gridDim.x) {
        const OzItem w = a.items[i];
        const OzJob J = a.jobs[w.job];
        if (ni > 0 && !oz_wait(bar_a_empty, (ni - 1) & 1, sh, a)) {
          ok = false;
          break;
        }
        ++ni;
        mbar_expect_tx(bar_a_full, S * OZ_ATILE);
#pragma unroll 1
        for (int s = 0; s < S; ++s)
          tma_load_2d(sa + s * OZ_ATILE, &a.tA, 0, J.a_row + s * a.rpad + w.m0, bar_a_full);
        for (int n0 = w.n0; n0 < w.n1; n0 += OZ_BN, ++it) {
          const uint32_t st = it & 1;
          if (it >= 2 && !oz_wait(bar_b_empty + 8 * st, ((it >> 1) - 1) & 1, sh, a)) {
            ok = false;
            break;
          }
          mbar_expect_tx(bar_b_full + 8 * st, S * OZ_BTILE);
#pragma unroll 1
          for (int s = 0; s < S; ++s)
            tma_load_2d(sb + (st * S + s) * OZ_BTILE, &a.tB, 0, J.b_row + s * a.rpad + n0, bar_b_full + 8 * st);
        }
      }
      if (!ok) {   // copies still in flight land before the CTA may exit (bounded)
        const long long t0 = clock64();
        if (ni > 0)
          while (!mbar_try(bar_a_full, (ni - 1) & 1) && clock64() - t0 < a.timeout_cycles) {
          }
        for (uint32_t u = it > 2 ? it - 2 : 0; u < it; ++u)
          while (!mbar_try(bar_b_full + 8 * (u & 1), (u >> 1) & 1) && clock64() - t0 < a.timeout_cycles) {
          }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = idesc_f16(OZ_BM, OZ_BN);
      uint32_t it = 0, ni = 0;
      bool ok = true;
      for (int i = blockIdx.x; ok && i < a.nitems; i += gridDim.x, ++ni) {
        const OzItem w = a.items[i];
        if (!oz_wait(bar_a_full, ni & 1, sh, a)) {
          ok = false;
          break;
        }
        for (int n0 = w.n0; n0 < w.n1; n0 += OZ_BN, ++it) {
          const uint32_t st = it & 1;
          if (!oz_wait(bar_b_full + 8 * st, (it >> 1) & 1, sh, a) ||
              (it >= 2 && !oz_wait(bar_acc_empty + 8 * st, ((it >> 1) - 1) & 1, sh, a))) {
            ok = false;
            break;
          }
          fence_after();
          // 84 products, fully unrolled: a product is only ~16 tensor cycles at N = 32, so the
          // issuing thread adds compile-time offsets to two base descriptors (the start address
          // field is the byte address / 16: offsets inside shared memory never carry out of it)
          const uint32_t acc = tmem + st * oz_acols(S);
          const uint64_t da0 = sw128_desc(sa), db0 = sw128_desc(sb + st * S * OZ_BTILE);
#pragma unroll
          for (int s = 0; s < S; ++s)
#pragma unroll
            for (int t = 0; t + s < S; ++t)
#pragma unroll
              for (int kk = 0; kk < OZ_K / 16; ++kk)
                mma_bf16(acc + (uint32_t)((s + t) * OZ_BN), da0 + (uint64_t)((s * OZ_ATILE + kk * 32) >> 4),
                         db0 + (uint64_t)((t * OZ_BTILE + kk * 32) >> 4), idesc, (s > 0 || kk > 0) ? 1u : 0u);
          mma_commit(bar_b_empty + 8 * st);
          mma_commit(bar_acc_full + 8 * st);
        }
        if (ok) mma_commit(bar_a_empty);
      }
      mma_commit(bar_done);   // the products in flight finish before TMEM is freed (bounded)
      const long long t0 = clock64();
      while (!mbar_try(bar_done, 0) && clock64() - t0 < a.timeout_cycles) {
      }
    }
  } else {
    // Software-pipelined over the CTA's tiles: the column exponents and the C values of the next
    // tile are loaded into registers before the current one is waited for and combined.
    const int quarter = warp & 3, col8 = (warp - 2) >> 2;
    const uint32_t lane_base = (uint32_t)(quarter * 32) << 16;
    int i = blockIdx.x;
    if (i < a.nitems) {
      int n0 = a.items[i].n0;
      double cv[8], cvn[8];
      int eb[8], ebn[8];
      uint32_t wmask, wmaskn = 0;
      // loads of tile (item ii, column n) into (c, e, m)
      auto fetch = [&](int ii, int n, double (&c)[8], int (&e)[8], uint32_t& m) {
        const OzItem w = a.items[ii];
        const OzJob& J = a.jobs[w.job];
        const int r = w.m0 + quarter * 32 + lane;
        const int c0 = n + col8 * 8;
        const int M = J.M, N = J.N;
        m = 0;
        if (r < M) {
          const int cend = min(N, c0 + 8);
          const int clim = a.lower ? min(cend, ((r >> 6) + 1) << 6) : cend;
          if (clim > c0) m = (1u << min(clim - c0, 8)) - 1u;
        }
        const int4* ebp = reinterpret_cast<const int4*>(J.eb + c0);   // 32-byte aligned: c0 % 8 == 0
        const int4 e0 = ebp[0], e1 = ebp[1];
        e[0] = e0.x; e[1] = e0.y; e[2] = e0.z; e[3] = e0.w;
        e[4] = e1.x; e[5] = e1.y; e[6] = e1.z; e[7] = e1.w;
        const double* crow = J.C + (int64_t)r * J.ldc + c0;
        if (a.beta && m == 0xffu && (reinterpret_cast<uintptr_t>(crow) & 15) == 0) {
#pragma unroll
          for (int j = 0; j < 8; j += 2) {
            const double2 v2 = *reinterpret_cast<const double2*>(crow + j);
            c[j] = v2.x;
            c[j + 1] = v2.y;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 8; ++j) c[j] = (a.beta && (m >> j & 1u)) ? crow[j] : 0.0;
        }
      };
      fetch(i, n0, cv, eb, wmask);
      for (uint32_t it = 0;; ++it) {
        // the tile after this one: the next columns of this item, else the CTA's next item
        int ni = i, nn0 = n0 + OZ_BN;
        if (nn0 >= a.items[i].n1) {
          ni = i + gridDim.x;
          nn0 = ni < a.nitems ? a.items[ni].n0 : 0;
        }
        if (ni < a.nitems) fetch(ni, nn0, cvn, ebn, wmaskn);
        const uint32_t st = it & 1;
        int got = 0;
        if (lane == 0) got = oz_wait(bar_acc_full + 8 * st, (it >> 1) & 1, sh, a) ? 1 : 0;
        got = __shfl_sync(0xffffffffu, got, 0);
        if (!got) break;
        fence_after();
        const OzItem w = a.items[i];
        const OzJob& J = a.jobs[w.job];
        const int r = w.m0 + quarter * 32 + lane;
        const int ea = r < J.M ? J.ea[r] : 0;
        double* drow = J.D + (int64_t)r * J.ldd + n0 + col8 * 8;
        const bool vec = wmask == 0xffu && (reinterpret_cast<uintptr_t>(drow) & 15) == 0;
#pragma unroll
        for (int q = 0; q < 8; q += 4) {   // two rounds of four columns
          uint32_t g[S][4];
#pragma unroll
          for (int c = 0; c < S; ++c)
            tmem_ld4(tmem + lane_base + st * oz_acols(S) + (uint32_t)(c * OZ_BN + col8 * 8 + q), g[c]);
          tmem_wait_ld();
          double v[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float hi, lo;
            oz_combine<S>(g, j, hi, lo);
            if (a.neg) {
              hi = -hi;
              lo = -lo;
            }
            const int k = ea + eb[q + j] - 2 * OZ_BITS;
            v[j] = cv[q + j] + (f32_to_f64_scaled(hi, k) + f32_to_f64_scaled(lo, k));
            if (ea >= OZ_BAD || eb[q + j] >= OZ_BAD) v[j] = __longlong_as_double(0x7ff8000000000000ll);
          }
          if (vec) {
            *reinterpret_cast<double2*>(drow + q) = make_double2(v[0], v[1]);
            *reinterpret_cast<double2*>(drow + q + 2) = make_double2(v[2], v[3]);
          } else {
#pragma unroll
            for (int j = 0; j < 4; ++j)
              if (wmask >> (q + j) & 1u) drow[q + j] = v[j];
          }
        }
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(bar_acc_empty + 8 * st);   // the set is free for the tile after next
        if (ni >= a.nitems) break;
        i = ni;
        n0 = nn0;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          cv[j] = cvn[j];
          eb[j] = ebn[j];
        }
        wmask = wmaskn;
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1) tmem_dealloc<1>(tmem, 512);
}

constexpr size_t oz_smem_bytes(int S) { return 1024 + oz_tiles(S) + 64; }

template <int S>
cudaError_t oz_rows_attr() {
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    attr = cudaFuncSetAttribute(k_oz_rows<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)oz_smem_bytes(S));
  });
  return attr;
}

// the update phases of one step k, in the order they run
enum { OZ_PANEL, OZ_TRAIL, OZ_FA, OZ_FB, OZ_BA, OZ_BB, OZ_NPHASE };

// the shape of phase ph at step k of a matrix of order s: M x N, and whether only the block
// lower triangle is written
struct OzShape {
  int M, N, lower;
};
OzShape oz_shape(int ph, int k, int s) {
  const int c0 = k * 64;
  const int bs = std::max(0, std::min(64, s - c0)), rest = std::max(0, s - c0 - 64), ncol = c0 + bs;
  if (bs == 0) return OzShape{0, 0, 0};
  switch (ph) {
    case OZ_PANEL: return OzShape{rest, rest > 0 ? bs : 0, 0};
    case OZ_TRAIL: return OzShape{rest, rest, 1};
    case OZ_FA: return OzShape{bs, ncol, 0};
    case OZ_FB: return OzShape{rest, rest > 0 ? ncol : 0, 0};
    case OZ_BA: return OzShape{bs, ncol, 0};
    default: return OzShape{c0, c0, 1};
  }
}

int sm_count() {
  static int n = [] {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess)
      v = 0;
    return v > 0 ? v : 1;
  }();
  return n;
}

// work items of one product: per 128-row block, its columns (those on or left of the block
// diagonal when lower) in pieces of `cols`
template <typename F>
void oz_items(const OzShape& sh, int cols, F&& emit) {
  for (int m0 = 0; m0 < sh.M; m0 += OZ_BM) {
    const int nlim = sh.lower ? std::min(sh.N, (m0 / 64 + 2) * 64) : sh.N;
    const int nend = (int)round_up(nlim, OZ_BN);
    for (int n0 = 0; n0 < nend; n0 += cols) emit(m0, n0, std::min(n0 + cols, nend));
  }
}

// columns of one work item: OZ_ITEM_COLS, narrower (down to one 32-column tile) where the nj
// matrices of a batch would give fewer items than there are SMs -- the small products of a
// step (the panel, the diagonal block rows of both sweeps), which otherwise leave most SMs idle
int oz_item_cols(const OzShape& sh, int nj) {
  auto count = [&](int cols) {
    int64_t n = 0;
    oz_items(sh, cols, [&](int, int, int) { ++n; });
    return n * nj;
  };
  int w = OZ_ITEM_COLS;
  while (w > OZ_BN && count(w) < sm_count()) w /= 2;
  return w;
}

int64_t oz_items_per_job(int smax, bool invert, int nj) {
  const int nb = (int)ceil_div(smax, 64);
  int64_t n = 0;
  for (int k = 0; k < nb; ++k)
    for (int ph = 0; ph < OZ_NPHASE; ++ph) {
      if (!invert && ph >= OZ_FA) break;
      const OzShape sh = oz_shape(ph, k, smax);
      oz_items(sh, oz_item_cols(sh, nj), [&](int, int, int) { ++n; });
    }
  return n;
}

struct OzLayout {
  int nj, nb, rpad;
  size_t inv, djobs, sa, sb, ea, eb, sjobs, gjobs, items, total;
};

OzLayout oz_layout(int nj, int smax) {
  OzLayout L{};
  L.nj = nj;
  L.nb = (int)ceil_div(smax, 64);
  L.rpad = (int)round_up(smax, OZ_BM);
  size_t p = 0;
  auto take = [&](size_t bytes) {
    const size_t at = p;
    p = round_up((int64_t)(p + bytes), 1024);
    return at;
  };
  L.inv = take((size_t)nj * L.nb * 4096 * sizeof(double));
  L.djobs = take((size_t)nj * L.nb * sizeof(DiagJob));
  L.sa = take((size_t)nj * OZ_SMAX * L.rpad * 64 * 2);
  L.sb = take((size_t)nj * OZ_SMAX * L.rpad * 64 * 2);
  L.ea = take((size_t)nj * L.rpad * 4);
  L.eb = take((size_t)nj * L.rpad * 4);
  L.sjobs = take((size_t)OZ_NPHASE * L.nb * 2 * nj * sizeof(OzSliceJob));
  L.gjobs = take((size_t)OZ_NPHASE * L.nb * nj * sizeof(OzJob));
  // every job's items are at most those of a matrix of order smax
  L.items = take((size_t)nj * oz_items_per_job(smax, true, nj) * sizeof(OzItem));
  L.total = p + 1024;   // the caller's pointer is aligned up to 1 KB first
  return L;
}

template <int S>
cudaError_t factor_and_invert_sliced(const std::vector<MatJob>& jobs, bool invert, void* dev_scratch, cudaStream_t st) {
  const int nj = (int)jobs.size();
  if (nj == 0) return cudaSuccess;
  int smax = 0;
  for (const auto& j : jobs) smax = std::max(smax, j.s);
  if (smax <= 0) return cudaSuccess;
  const OzLayout L = oz_layout(nj, smax);
  const int nb = L.nb, rpad = L.rpad;
  char* p = reinterpret_cast<char*>(round_up((int64_t)reinterpret_cast<uintptr_t>(dev_scratch), 1024));
  double* inv = reinterpret_cast<double*>(p + L.inv);
  DiagJob* djobs = reinterpret_cast<DiagJob*>(p + L.djobs);
  __half* sa = reinterpret_cast<__half*>(p + L.sa);
  __half* sb = reinterpret_cast<__half*>(p + L.sb);
  int32_t* ea = reinterpret_cast<int32_t*>(p + L.ea);
  int32_t* eb = reinterpret_cast<int32_t*>(p + L.eb);
  OzSliceJob* sjobs = reinterpret_cast<OzSliceJob*>(p + L.sjobs);
  OzJob* gjobs = reinterpret_cast<OzJob*>(p + L.gjobs);
  OzItem* ditems = reinterpret_cast<OzItem*>(p + L.items);
  cudaError_t e;
  if ((e = oz_rows_attr<S>()) != cudaSuccess) return e;

  std::vector<DiagJob> hd((size_t)nj * nb);
  for (int k = 0; k < nb; ++k)
    for (int b = 0; b < nj; ++b)
      hd[(size_t)k * nj + b] = DiagJob{jobs[b].A, jobs[b].ld, jobs[b].s, inv + ((size_t)b * nb + k) * 4096,
                                       jobs[b].info};
  if ((e = cudaMemcpyAsync(djobs, hd.data(), hd.size() * sizeof(DiagJob), cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return e;

  // tables: slice jobs [phase][k][operand][b], products [phase][k][b], work items per (phase, k)
  std::vector<OzSliceJob> hs((size_t)OZ_NPHASE * nb * 2 * nj);
  std::vector<OzJob> hg((size_t)OZ_NPHASE * nb * nj);
  std::vector<OzItem> hi;
  std::vector<int64_t> item_at((size_t)OZ_NPHASE * nb + 1, 0);
  auto sj = [&](int ph, int k, int op, int b) -> OzSliceJob& { return hs[(((size_t)ph * nb + k) * 2 + op) * nj + b]; };
  auto gj = [&](int ph, int k, int b) -> OzJob& { return hg[((size_t)ph * nb + k) * nj + b]; };
  for (int k = 0; k < nb; ++k)
    for (int b = 0; b < nj; ++b) {
      const MatJob& J = jobs[b];
      const int64_t c0 = (int64_t)k * 64;
      const int bs = (int)std::max<int64_t>(0, std::min<int64_t>(64, J.s - c0));
      if (bs == 0) continue;   // this matrix ends before block k: its jobs stay empty
      const int rest = (int)std::max<int64_t>(0, J.s - c0 - 64);
      const int ncol = (int)(c0 + bs);
      const double* Ikk = inv + ((size_t)b * nb + k) * 4096;
      double* Lp = J.A + (c0 + 64) * J.ld + c0;   // L panel below the diagonal block
      double* Qk = J.Q ? J.Q + c0 * J.ldq : nullptr;
      __half* da = sa + (size_t)b * S * rpad * 64;
      __half* db = sb + (size_t)b * S * rpad * 64;
      int32_t* xa = ea + (size_t)b * rpad;
      int32_t* xb = eb + (size_t)b * rpad;
      const int arow = b * S * rpad;
      auto slice = [&](int ph, const double* srcA, int64_t ldA, int rowsA, int transA, const double* srcB,
                       int64_t ldB, int rowsB, int transB) {
        sj(ph, k, 0, b) = OzSliceJob{srcA, ldA, rowsA, bs, transA, da, xa};
        sj(ph, k, 1, b) = OzSliceJob{srcB, ldB, rowsB, bs, transB, db, xb};
      };
      auto prod = [&](int ph, const double* C, double* D, int64_t ld) {
        const OzShape sh = oz_shape(ph, k, J.s);
        gj(ph, k, b) = OzJob{C, D, ld, ld, sh.M, sh.N, arow, arow, xa, xb};
      };
      // panel A_ik <- A_ik L_kk^-T (D = A_ik Ikk^T), then trailing A_il -= L_ik L_lk^T
      if (rest > 0) {
        slice(OZ_PANEL, Lp, J.ld, rest, 0, Ikk, 64, bs, 0);
        prod(OZ_PANEL, nullptr, Lp, J.ld);
        slice(OZ_TRAIL, Lp, J.ld, rest, 0, Lp, J.ld, rest, 0);
        prod(OZ_TRAIL, Lp + 64, Lp + 64, J.ld);
      }
      if (!invert || !Qk) continue;
      // forward sweep: Y_k = Ikk Y_k (columns 0..ncol), Y_i -= L_ik Y_k below
      slice(OZ_FA, Ikk, 64, bs, 0, Qk, J.ldq, ncol, 1);
      prod(OZ_FA, nullptr, Qk, J.ldq);
      if (rest > 0) {
        slice(OZ_FB, Lp, J.ld, rest, 0, Qk, J.ldq, ncol, 1);
        prod(OZ_FB, Qk + 64 * J.ldq, Qk + 64 * J.ldq, J.ldq);
      }
      // backward sweep: Q_k = Ikk^T Q_k, then Q_i -= L_ki^T Q_k above (block lower triangle)
      slice(OZ_BA, Ikk, 64, bs, 1, Qk, J.ldq, ncol, 1);
      prod(OZ_BA, nullptr, Qk, J.ldq);
      if (c0 > 0) {
        slice(OZ_BB, J.A + c0 * J.ld, J.ld, (int)c0, 1, Qk, J.ldq, (int)c0, 1);
        prod(OZ_BB, J.Q, J.Q, J.ldq);
      }
    }
  for (int ph = 0; ph < OZ_NPHASE; ++ph)
    for (int k = 0; k < nb; ++k) {
      item_at[(size_t)ph * nb + k] = (int64_t)hi.size();
      const int cols = oz_item_cols(oz_shape(ph, k, smax), nj);   // the same width for every matrix
      for (int b = 0; b < nj; ++b) {
        const OzJob& g = gj(ph, k, b);
        if (g.M <= 0 || g.N <= 0) continue;
        oz_items(OzShape{g.M, g.N, ph == OZ_TRAIL || ph == OZ_BB}, cols, [&](int m0, int n0, int n1) {
          hi.push_back(OzItem{b, m0, n0, n1});
        });
      }
    }
  item_at[(size_t)OZ_NPHASE * nb] = (int64_t)hi.size();
  if ((size_t)hi.size() * sizeof(OzItem) > L.total - L.items) return cudaErrorInvalidValue;
  if ((e = cudaMemcpyAsync(sjobs, hs.data(), hs.size() * sizeof(OzSliceJob), cudaMemcpyHostToDevice, st)) !=
          cudaSuccess ||
      (e = cudaMemcpyAsync(gjobs, hg.data(), hg.size() * sizeof(OzJob), cudaMemcpyHostToDevice, st)) !=
          cudaSuccess ||
      (!hi.empty() &&
       (e = cudaMemcpyAsync(ditems, hi.data(), hi.size() * sizeof(OzItem), cudaMemcpyHostToDevice, st)) !=
           cudaSuccess))
    return e;
  // the host tables are read by the copies: pageable memory is staged before the calls return

  OzArgs a;
  memset(&a, 0, sizeof(a));
  const int64_t map_rows = (int64_t)nj * S * rpad;
  if ((e = tc_make_map_bf16(&a.tA, sa, 64, map_rows, 64, OZ_BM, 64)) != cudaSuccess) return e;
  if ((e = tc_make_map_bf16(&a.tB, sb, 64, map_rows, 64, OZ_BN, 64)) != cudaSuccess) return e;
  a.rpad = rpad;
  a.err = tc_error_ptr();
  if (!a.err) return cudaErrorMemoryAllocation;
  a.timeout_cycles = 4000000000LL;   // about two seconds at the boost clock
  const int nsm = sm_count();

  // slices of both operands of phase ph (rows up to rowsA / rowsB, zero to the tile edge), then
  // the product over its work items
  auto run = [&](int ph, int k, int rowsA, int rowsB, int neg, int beta, int lower) -> cudaError_t {
    const int64_t i0 = item_at[(size_t)ph * nb + k], i1 = item_at[(size_t)ph * nb + k + 1];
    if (i1 <= i0) return cudaSuccess;
    const int rows = (int)round_up(std::max(rowsA, rowsB), OZ_BM);
    dim3 sg((unsigned)(std::min(rows, rpad) / 32), 1, (unsigned)(2 * nj));
    k_oz_slice<S><<<sg, 256, 0, st>>>(sjobs + ((size_t)ph * nb + k) * 2 * nj, rpad);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    a.jobs = gjobs + ((size_t)ph * nb + k) * nj;
    a.items = ditems + i0;
    a.nitems = (int)(i1 - i0);
    a.neg = neg;
    a.beta = beta;
    a.lower = lower;
    // at most OZ_ITEMS_PER_CTA items per CTA: a CTA fills its SM's shared memory, so other
    // kernels (a server's scoring on a high-priority stream) start only when one finishes
    const int64_t ni = i1 - i0;
    const int64_t grid = std::min<int64_t>(ni, std::max<int64_t>(nsm, ceil_div(ni, OZ_ITEMS_PER_CTA)));
    k_oz_rows<S><<<(unsigned)grid, OZ_THREADS, oz_smem_bytes(S), st>>>(a);
    return cudaGetLastError();
  };
  for (int k = 0; k < nb; ++k) {
    const int c0 = k * 64, rest = std::max(0, smax - c0 - 64);
    if ((e = launch_potrf_diag(djobs + (size_t)k * nj, nj, c0, st)) != cudaSuccess) return e;
    if ((e = run(OZ_PANEL, k, rest, 64, 0, 0, 0)) != cudaSuccess) return e;
    if ((e = run(OZ_TRAIL, k, rest, rest, 1, 1, 1)) != cudaSuccess) return e;
  }
  if (!invert) return cudaSuccess;
  for (int k = 0; k < nb; ++k) {
    const int c0 = k * 64, rest = std::max(0, smax - c0 - 64), ncol = std::min(smax, c0 + 64);
    if ((e = run(OZ_FA, k, 64, ncol, 0, 0, 0)) != cudaSuccess) return e;
    if ((e = run(OZ_FB, k, rest, ncol, 1, 1, 0)) != cudaSuccess) return e;
  }
  for (int k = nb - 1; k >= 0; --k) {
    const int c0 = k * 64, ncol = std::min(smax, c0 + 64);
    if ((e = run(OZ_BA, k, 64, ncol, 0, 0, 0)) != cudaSuccess) return e;
    if ((e = run(OZ_BB, k, c0, c0, 1, 1, 1)) != cudaSuccess) return e;
  }
  for (const auto& J : jobs)
    if (J.Q && (e = launch_mirror_lower(J.Q, J.ldq, J.s, st)) != cudaSuccess) return e;
  return cudaSuccess;
}

}  // namespace

size_t oz_factor_scratch_bytes(int njobs, int smax) { return oz_layout(njobs, smax).total; }

cudaError_t factor_and_invert_oz(const std::vector<MatJob>& jobs, bool invert, void* dev_scratch, cudaStream_t st,
                                 int bits) {
  switch (bits) {
    case 48: return factor_and_invert_sliced<6>(jobs, invert, dev_scratch, st);
    case 40: return factor_and_invert_sliced<5>(jobs, invert, dev_scratch, st);
    default: return cudaErrorInvalidValue;
  }
}

RFF_CHECK_UNIT(ozaki)

}  // namespace rff
