// Bandwidth-bound kernels of the iteration: proximal operators (Sec. 2.3; the
// O and W updates of Sec. 3), the row-local exchange that follows the graph
// projection (eq. (obar_ij), (obar) in the reorganised form of Sec. 3), the
// averaging and dual updates, layout changes and deterministic reductions.
#include "common.cuh"
#include "internal.h"

#include <algorithm>
#include <mutex>

namespace rff {

namespace {

constexpr int LOSS_SQUARED = 0, LOSS_HINGE = 1, LOSS_LOGISTIC = 2, LOSS_MULTINOMIAL = 3, LOSS_L1 = 4,
              LOSS_CRAMMER_SINGER = 5;
// losses whose prox couples the outputs of a row (a warp per row); the others act per entry
__host__ __device__ constexpr bool row_loss(int loss) {
  return loss == LOSS_MULTINOMIAL || loss == LOSS_CRAMMER_SINGER;
}

// dst[p][c] = src[map[p]][c] for c < w, zero elsewhere (map[p] < 0: zero row)
__global__ void k_scatter_rows(const float* __restrict__ src, int64_t lds, int64_t w,
                               const int32_t* __restrict__ map, int64_t nrows, float* __restrict__ dst, int64_t ld) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nrows * ld) return;
  const int64_t p = t / ld, c = t % ld;
  const int32_t g = map ? map[p] : (int32_t)p;
  dst[t] = (g >= 0 && c < w) ? src[(int64_t)g * lds + c] : 0.f;
}

__global__ void k_csr_check(const int64_t* __restrict__ indptr, const int32_t* __restrict__ indices, int64_t n,
                            int64_t d, int64_t nnz, int* __restrict__ flag) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r >= n) return;
  const int64_t a = indptr[r], b = indptr[r + 1];
  bool bad = a < 0 || b < a || b > nnz || (r == 0 && a != 0) || (r == n - 1 && b != nnz);
  if (!bad)
    for (int64_t e = a; e < b; ++e)
      if (indices[e] < 0 || indices[e] >= d) { bad = true; break; }
  if (bad) atomicOr(flag, 1);
}

// one thread per slot row: its entries in order, so repeated columns add up deterministically
__global__ void k_scatter_csr(const int64_t* __restrict__ indptr, const int32_t* __restrict__ indices,
                              const float* __restrict__ values, const int32_t* __restrict__ map, int64_t nrows,
                              float* __restrict__ dst, int64_t ld) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= nrows) return;
  const int32_t r = map[p];
  if (r < 0) return;
  for (int64_t e = indptr[r]; e < indptr[r + 1]; ++e)
    if (RFF_IN(indices[e], ld)) dst[p * ld + indices[e]] += values[e];
}

__global__ void k_set_column(float* __restrict__ X, int64_t ld, int64_t rows, int64_t col, float v) {
  const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (r < rows) X[r * ld + col] = v;
}

__global__ void k_split_f16(const float* __restrict__ src, int64_t n, float scale, __half* __restrict__ hi,
                            __half* __restrict__ lo) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  split_f16(src[t], scale, hi[t], lo[t]);
}

__global__ void k_split(const float* __restrict__ src, int64_t n, __nv_bfloat16* __restrict__ hi,
                        __nv_bfloat16* __restrict__ lo) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  split_bf16(src[t], hi[t], lo[t]);
}

// ---- scalar proxes: argmin_o 1/2 (o - v)^2 + t V(y, o)
__device__ __forceinline__ float prox_squared(float v, float y, float t) { return (v + 2.f * t * y) / (1.f + 2.f * t); }

__device__ __forceinline__ float prox_hinge(float v, float y, float t) {
  const float u = y * v;
  return u > 1.f ? v : (u < 1.f - t ? v + t * y : y);
}

// logistic, y = +-1: in p = y o, a = y v solve f(p) = p - a - t / (1 + e^p) = 0,
// f increasing, root in [a, a + t]: Newton steps kept inside the bracket, which
// is tightened by the sign of f at every step.
__device__ __forceinline__ float prox_logistic(float v, float y, float t, int iters) {
  const float a = y * v;
  float lo = a, hi = a + t, p = a + 0.5f * t;
  for (int it = 0; it < iters; ++it) {
    const float sm = 1.f / (1.f + __expf(p));   // sigma(-p)
    const float f = p - a - t * sm;
    if (f < 0.f) lo = p; else hi = p;
    const float fp = 1.f + t * sm * (1.f - sm);
    if (f == 0.f) break;
    float q = p - f / fp;
    if (!(q >= lo && q <= hi)) q = 0.5f * (lo + hi);
    p = q;
  }
  return y * p;
}

// l1 loss |y - o|: v - y soft-thresholded by t, about y
__device__ __forceinline__ float prox_l1(float v, float y, float t) {
  const float d = v - y;
  return y + copysignf(fmaxf(fabsf(d) - t, 0.f), d);
}

__device__ __forceinline__ float prox_scalar(int loss, float v, float y, float t, int iters) {
  if (loss == LOSS_SQUARED) return prox_squared(v, y, t);
  if (loss == LOSS_HINGE) return prox_hinge(v, y, t);
  if (loss == LOSS_L1) return prox_l1(v, y, t);
  return prox_logistic(v, y, t, iters);
}

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ float warp_max(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fmaxf(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// Multinomial logistic prox of one row, one warp, lanes over the m outputs (up
// to 8 per lane), c = argmax_k y_k (first maximum).  The optimality condition
// o = v - t (softmax(o) - e_c) is solved through s = log sum_k exp(o_k): with
// w = v + t e_c, each p_k = exp(o_k - s) satisfies log p_k + t p_k = w_k - s,
// a scalar equation solved by Newton from a Lambert-W estimate, and s is the
// root of F(s) = sum_k p_k(s) - 1, which is convex and decreasing; Newton on s
// from s0 = max_k w_k - t (where F >= 0) therefore rises monotonically to the
// root.  Finally o = w - t p.  Only the first solve for each log p_k starts from the
// estimate (four Newton steps); after each step ds of s it restarts from the first-order
// update q - ds / (1 + t p) and takes two Newton steps.
constexpr int MAXPL = 8;

__device__ __forceinline__ float solve_logp(float a, float t, float logt) {
  // q = log p with q + t e^q = a; start from W(t e^a) ~ log1p(z) or L - log L
  const float L = logt + a;
  const float W0 = (L < 1.f) ? log1pf(expf(L)) : L - logf(L);
  float q = logf(fmaxf(W0, 1e-37f)) - logt;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float e = expf(q);
    q -= (q + t * e - a) / (1.f + t * e);
  }
  return q;
}

// class index of a row, the first maximum of y over the m outputs (a warp, lanes over outputs)
__device__ __forceinline__ int row_class(const float (&y)[MAXPL], int m) {
  const int lane = threadIdx.x & 31;
  float best = -INFINITY;
  int bidx = 1 << 30;
#pragma unroll
  for (int q = 0; q < MAXPL; ++q) {
    const int k = lane + 32 * q;
    if (k < m && (y[q] > best)) { best = y[q]; bidx = k; }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, off);
    const int oi = __shfl_xor_sync(0xffffffffu, bidx, off);
    if (ob > best || (ob == best && oi < bidx)) { best = ob; bidx = oi; }
  }
  return bidx;
}

__device__ void prox_multinomial_row(const float (&v)[MAXPL], const float (&y)[MAXPL], int m, float t, int iters,
                                     float (&o)[MAXPL]) {
  const int lane = threadIdx.x & 31;
  if (!(t > 1e-30f)) {
#pragma unroll
    for (int q = 0; q < MAXPL; ++q) o[q] = v[q];
    return;
  }
  const int bidx = row_class(y, m);
  float w[MAXPL];
  float wmax = -INFINITY;
#pragma unroll
  for (int q = 0; q < MAXPL; ++q) {
    const int k = lane + 32 * q;
    w[q] = v[q] + (k == bidx ? t : 0.f);
    if (k < m) wmax = fmaxf(wmax, w[q]);
  }
  wmax = warp_max(wmax);
  const float logt = logf(t);
  float s = wmax - t;
  float lq[MAXPL], pv[MAXPL];   // log p_k and p_k at the current s
#pragma unroll
  for (int q = 0; q < MAXPL; ++q) {
    lq[q] = 0.f;
    pv[q] = 0.f;
    if (lane + 32 * q < m) {
      lq[q] = solve_logp(w[q] - s, t, logt);
      pv[q] = expf(lq[q]);
    }
  }
  for (int it = 0; it < iters; ++it) {
    float F = 0.f, dF = 0.f;
    float rinv[MAXPL];
#pragma unroll
    for (int q = 0; q < MAXPL; ++q) {
      rinv[q] = 1.f / (1.f + t * pv[q]);
      if (lane + 32 * q < m) {
        F += pv[q];
        dF += pv[q] * rinv[q];
      }
    }
    F = warp_sum(F) - 1.f;
    dF = warp_sum(dF);
    const float ds = F / dF;
    s += ds;
#pragma unroll
    for (int q = 0; q < MAXPL; ++q) {
      if (lane + 32 * q < m) {
        const float a = w[q] - s;
        float x = lq[q] - ds * rinv[q];
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          const float e = expf(x);
          x -= (x + t * e - a) / (1.f + t * e);
        }
        lq[q] = x;
        pv[q] = expf(x);
      }
    }
  }
#pragma unroll
  for (int q = 0; q < MAXPL; ++q) {
    const int k = lane + 32 * q;
    o[q] = (k < m) ? w[q] - t * pv[q] : 0.f;
  }
}

// Crammer-Singer multiclass hinge prox of one row (a warp, lanes over the m outputs),
// V(y, o) = max_k (Delta_k + o_k - o_c), Delta_k = 1 - [k = c], c = argmax_k y_k (first).
// The dual of the prox is a projection onto the probability simplex; scaled by t it reads:
// with w_k = v_k + Delta_k + t [k = c], the prox is o_k = min(w_k, tau) - Delta_k where tau
// solves sum_k max(w_k - tau, 0) = t.  tau by Michelot's finite method (1986): from the set of
// all outputs, tau = (sum of w over the set - t) / its size, and the entries at or below tau
// leave the set, until none leaves.  The set shrinks at every round but the last (at most m
// rounds) and keeps its largest entry, which lies above tau for t > 0.  The sums run over
// w_k - max_k w_k: the entries of the final set lie within t of the maximum (tau >= max w - t),
// so tau is formed from values of the size of t rather than of |w|.  The warp sums are
// butterflies, so every lane holds the same tau and takes the same exit.
__device__ void prox_crammer_singer_row(const float (&v)[MAXPL], const float (&y)[MAXPL], int m, float t,
                                        float (&o)[MAXPL]) {
  const int lane = threadIdx.x & 31;
  if (!(t > 0.f)) {
#pragma unroll
    for (int q = 0; q < MAXPL; ++q) o[q] = v[q];
    return;
  }
  const int c = row_class(y, m);
  float w[MAXPL];
  bool in[MAXPL];
  float wmax = -INFINITY;
#pragma unroll
  for (int q = 0; q < MAXPL; ++q) {
    const int k = lane + 32 * q;
    in[q] = k < m;
    w[q] = v[q] + (k == c ? t : 1.f);
    if (in[q]) wmax = fmaxf(wmax, w[q]);
  }
  wmax = warp_max(wmax);
  float sum = 0.f;
#pragma unroll
  for (int q = 0; q < MAXPL; ++q) {
    w[q] -= wmax;   // shifted: tau below is relative to the maximum
    if (in[q]) sum += w[q];
  }
  int cnt = m;
  float tau = (warp_sum(sum) - t) / (float)cnt;
  for (int round = 0; round < m; ++round) {
    float s2 = 0.f;
    int c2 = 0;
#pragma unroll
    for (int q = 0; q < MAXPL; ++q)
      if (in[q] && w[q] > tau) { s2 += w[q]; ++c2; }
    s2 = warp_sum(s2);
    c2 = __reduce_add_sync(0xffffffffu, c2);
    if (c2 == cnt || c2 == 0) break;
#pragma unroll
    for (int q = 0; q < MAXPL; ++q) in[q] = in[q] && w[q] > tau;
    cnt = c2;
    tau = (s2 - t) / (float)cnt;
  }
#pragma unroll
  for (int q = 0; q < MAXPL; ++q) {
    const int k = lane + 32 * q;
    o[q] = (k < m) ? (fminf(w[q], tau) + wmax) - (k == c ? 0.f : 1.f) : 0.f;
  }
}

__device__ __forceinline__ void prox_row(int loss, const float (&v)[MAXPL], const float (&y)[MAXPL], int m, float t,
                                         int iters, float (&o)[MAXPL]) {
  if (loss == LOSS_MULTINOMIAL) prox_multinomial_row(v, y, m, t, iters, o);
  else prox_crammer_singer_row(v, y, m, t, o);
}

__global__ void k_prox_loss(int loss, const float* __restrict__ V, const float* __restrict__ Y, int64_t n, int m,
                            int64_t ld, float t, int iters, float* __restrict__ out) {
  if (row_loss(loss)) {
    const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
    if (row >= n) return;
    const int lane = threadIdx.x & 31;
    float v[MAXPL], y[MAXPL], o[MAXPL];
#pragma unroll
    for (int q = 0; q < MAXPL; ++q) {
      const int k = lane + 32 * q;
      v[q] = (k < m) ? V[row * ld + k] : 0.f;
      y[q] = (k < m) ? Y[row * ld + k] : 0.f;
    }
    prox_row(loss, v, y, m, t, iters, o);
#pragma unroll
    for (int q = 0; q < MAXPL; ++q) {
      const int k = lane + 32 * q;
      if (k < m) out[row * ld + k] = o[q];
    }
    return;
  }
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n * (int64_t)m) return;
  const int64_t r = e / m, c = e % m;
  out[r * ld + c] = prox_scalar(loss, V[r * ld + c], Y[r * ld + c], t, iters);
}

// prox of tau r at (V - mu): l2 |w|^2 -> (v - mu)/(1 + 2 tau); l1 -> soft threshold.
// With tau_col, column c (= e mod ncol) uses tau * tau_col[c] (one lambda per output column).
__global__ void k_prox_reg(int reg, const float* __restrict__ V, const float* __restrict__ mu, int64_t n, float tau,
                           const float* __restrict__ tau_col, int ncol, float* __restrict__ out) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= n) return;
  const float t = tau_col ? tau * tau_col[e % ncol] : tau;
  const float x = V[e] - (mu ? mu[e] : 0.f);
  out[e] = (reg == 0) ? x / (1.f + 2.f * t) : copysignf(fmaxf(fabsf(x) - t, 0.f), x);
}

// Row-local exchange after pass 2 (one CTA per 32 row slots, 8 warps):
//   S = sum_j O'_ij;  Delta = O - S;  Obar = S/(C+1) + C/(C+1) O;  nu += O - Obar
//   U_i = Delta/(C+1) + nu                 (Obar_ij + nu_i = O'_ij + U_i: the projections'
//                                           operand, one for every column block)
//   O <- prox_{t V}(Obar - nu)             (the loss step of the next iteration)
// Phase 1 (a warp per row, lanes over outputs) updates Obar, nu and O and keeps
// Delta/(C+1) + nu of the tile in shared memory; phase 2 writes U_i, either row-major in
// FP32 (the SIMT path's and the outer form's operand) or transposed and split into a scaled
// FP16 hi/lo pair (U^T[c][slot], the tensor-core operand) through a shared-memory
// transpose, so that both the reads and the writes are coalesced.  The scale of that split
// comes before any U exists: U = nu + 2 (O - S)/(C+1) with S = sum_j O'_j, so
// |U| <= B = max|nu| + 2/(C+1) (max|O| + C max|O'|) over this kernel's inputs (widened by
// 2^-10 for the rounding of the bound itself); every CTA computes the same B.  Padding rows
// and columns are written as zeros.
constexpr int EX_ROWS = 32;

template <int LOSS>
__global__ void __launch_bounds__(256, row_loss(LOSS) ? 3 : 4) k_exchange(RowEpiArgs a) {
  extern __shared__ float ex_smem[];
  const int mp = a.mpad;
  float* tile = ex_smem;   // U of the 32 rows, [32][mpad + 1] (zero where not live)
  const bool split = a.VThi != nullptr;
  float vscale = 1.f;
  if (split) {
    const float opm = __uint_as_float(a.amax[AMAX_OP]), om = __uint_as_float(a.amax[AMAX_O]),
                num = __uint_as_float(a.amax[AMAX_NU]);
    const float c1 = (float)(a.C + 1);
    // U = nu^new + Delta/(C+1) = nu + 2 (O - S)/(C+1): |U| <= max|nu| + 2 (max|O| + C max|O'|)/(C+1)
    const float bound = (num + 2.f * (om + (float)a.C * opm) / c1) * (1.f + 0x1p-10f);
    vscale = f16_scale(bound);
    if (blockIdx.x == 0 && threadIdx.x == 0 && bound > 0.f) atomicMax(&a.amax[AMAX_V], __float_as_uint(bound));
  }
  float omax = 0.f, numax = 0.f;
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int64_t p0 = (int64_t)blockIdx.x * EX_ROWS;
  if (!RFF_SPAN(p0, EX_ROWS, a.nslots)) return;
  const int64_t jstride = a.nslots * mp;
  const float inv_c1 = 1.f / (float)(a.C + 1);
  const float cfrac = (float)a.C * inv_c1;
  // elementwise losses: the tile's 32 x m_pad elements as 16-byte items, two items per thread
  // with all their loads (O, nu, Y and the C blocks of O') issued before any use, so that
  // enough bytes are in flight to keep HBM busy; the arithmetic per element and its order are
  // those of the row form below
  if constexpr (!row_loss(LOSS)) {
    const int n4 = EX_ROWS * mp / 4;
    const int64_t tb = p0 * mp;
    constexpr int NB = 2;
#pragma unroll 1
    for (int i0 = threadIdx.x; i0 < n4; i0 += NB * 256) {
      float4 Ov[NB], nuv[NB], yv[NB], Sv[NB];
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int e4 = i0 + u * 256;
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        Ov[u] = nuv[u] = yv[u] = Sv[u] = z;
        if (e4 < n4) {
          Ov[u] = *reinterpret_cast<const float4*>(a.O + tb + 4 * e4);
          nuv[u] = *reinterpret_cast<const float4*>(a.nu + tb + 4 * e4);
          yv[u] = __ldg(reinterpret_cast<const float4*>(a.Y + tb + 4 * e4));
        }
      }
#pragma unroll 4
      for (int j = 0; j < a.C; ++j) {
        const float* opj = a.Op + j * jstride + tb;
#pragma unroll
        for (int u = 0; u < NB; ++u) {
          const int e4 = i0 + u * 256;
          if (e4 < n4) {
            const float4 v = __ldg(reinterpret_cast<const float4*>(opj + 4 * e4));
            Sv[u].x += v.x;
            Sv[u].y += v.y;
            Sv[u].z += v.z;
            Sv[u].w += v.w;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int e4 = i0 + u * 256;
        if (e4 >= n4) continue;
        const int r = (4 * e4) / mp, k0 = (4 * e4) % mp;
        const bool ok = a.row_ok[p0 + r] >= 0;
        float S[4] = {Sv[u].x, Sv[u].y, Sv[u].z, Sv[u].w}, O[4] = {Ov[u].x, Ov[u].y, Ov[u].z, Ov[u].w};
        float nu[4] = {nuv[u].x, nuv[u].y, nuv[u].z, nuv[u].w}, y[4] = {yv[u].x, yv[u].y, yv[u].z, yv[u].w};
        float ob[4], tm[4], on[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const bool live = ok && k0 + c < a.m;
          const float Delta = O[c] - S[c];
          const float Obar = S[c] * inv_c1 + cfrac * O[c];
          const float nun = nu[c] + (O[c] - Obar);
          ob[c] = live ? Obar : 0.f;
          nu[c] = live ? nun : 0.f;
          if (live) numax = fmaxf(numax, fabsf(nun));
          tm[c] = live ? Delta * inv_c1 + nun : 0.f;
          on[c] = live ? prox_scalar(LOSS, Obar - nun, y[c], a.t_loss, a.newton) : 0.f;
          if (live) omax = fmaxf(omax, fabsf(on[c]));
        }
        *reinterpret_cast<float4*>(a.Obar + tb + 4 * e4) = make_float4(ob[0], ob[1], ob[2], ob[3]);
        *reinterpret_cast<float4*>(a.nu + tb + 4 * e4) = make_float4(nu[0], nu[1], nu[2], nu[3]);
        *reinterpret_cast<float4*>(a.O + tb + 4 * e4) = make_float4(on[0], on[1], on[2], on[3]);
#pragma unroll
        for (int c = 0; c < 4; ++c) tile[r * (mp + 1) + k0 + c] = tm[c];
      }
    }
  }
  for (int r = warp; row_loss(LOSS) && r < EX_ROWS; r += 8) {
    const int64_t p = p0 + r;
    const bool ok = a.row_ok[p] >= 0;
    const int64_t base = p * mp;
    float w_in[MAXPL], y[MAXPL], Ov[MAXPL], nuv[MAXPL], Sv[MAXPL];
    // all of the row's loads first (independent, so they are in flight together)
#pragma unroll
    for (int q = 0; q < MAXPL; ++q) {
      const int k = lane + 32 * q;
      const bool in = k < mp;
      Ov[q] = in ? a.O[base + k] : 0.f;
      nuv[q] = in ? a.nu[base + k] : 0.f;
      y[q] = in ? a.Y[base + k] : 0.f;
      Sv[q] = 0.f;
    }
    for (int j = 0; j < a.C; ++j) {
      const float* opj = a.Op + j * jstride + base;
#pragma unroll
      for (int q = 0; q < MAXPL; ++q) {
        const int k = lane + 32 * q;
        if (k < mp) Sv[q] += opj[k];
      }
    }
#pragma unroll
    for (int q = 0; q < MAXPL; ++q) {
      const int k = lane + 32 * q;
      w_in[q] = 0.f;
      if (k >= mp) continue;
      const float S = Sv[q];
      const float O = Ov[q];
      float nu = nuv[q];
      const float Delta = O - S;
      const float Obar = S * inv_c1 + cfrac * O;
      nu += O - Obar;
      const bool live = ok && k < a.m;
      a.Obar[base + k] = live ? Obar : 0.f;
      a.nu[base + k] = live ? nu : 0.f;
      if (live) numax = fmaxf(numax, fabsf(nu));
      tile[r * (mp + 1) + k] = live ? Delta * inv_c1 + nu : 0.f;
      if (live) w_in[q] = Obar - nu;
      else y[q] = 0.f;
    }
    float o[MAXPL];
    if (row_loss(LOSS)) {
      prox_row(LOSS, w_in, y, a.m, a.t_loss, a.newton, o);
    } else {
#pragma unroll
      for (int q = 0; q < MAXPL; ++q) o[q] = prox_scalar(LOSS, w_in[q], y[q], a.t_loss, a.newton);
    }
#pragma unroll
    for (int q = 0; q < MAXPL; ++q) {
      const int k = lane + 32 * q;
      const bool live = ok && k < a.m;
      if (k < mp) a.O[base + k] = live ? o[q] : 0.f;
      if (live) omax = fmaxf(omax, fabsf(o[q]));
    }
  }
  if (split) {
    // max |O|, |nu| of the outputs: the bound of the next exchange
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) {
      omax = fmaxf(omax, __shfl_xor_sync(0xffffffffu, omax, sh));
      numax = fmaxf(numax, __shfl_xor_sync(0xffffffffu, numax, sh));
    }
    if (lane == 0) {
      if (omax > 0.f) atomicMax(&a.amax[AMAX_O_NEXT], __float_as_uint(omax));
      if (numax > 0.f) atomicMax(&a.amax[AMAX_NU_NEXT], __float_as_uint(numax));
    }
  }
  __syncthreads();
  // phase 2: U_i, once (block 0 of the V buffers): row-major FP32, or transposed and split
  // into the scaled FP16 pair from the shared-memory tile
  if (!split) {
    float* v = a.V32 + p0 * mp;
    for (int e = threadIdx.x; e < EX_ROWS * mp; e += 256) v[e] = tile[(e / mp) * (mp + 1) + e % mp];
    return;
  }
  // lanes over the 32 rows, warps over columns: U^T[c][p0 + lane]
  for (int c = warp; c < mp; c += 8) {
    __half hi, lo;
    split_f16(tile[lane * (mp + 1) + c], vscale, hi, lo);
    const int64_t o = (int64_t)c * a.nslots + p0 + lane;
    a.VThi[o] = hi;
    a.VTlo[o] = lo;
  }
}

// rhs = Wbar - mu'_ij + sum of the R partials (padding feature slots zero when feat_ok is given)
__global__ void k_rhs(const float* __restrict__ Wbar, const float* __restrict__ muij, const float* __restrict__ Rpart,
                      int nsplit, int R, int64_t nfe, const int32_t* __restrict__ feat_ok, int mpad,
                      const float* __restrict__ What, float* __restrict__ rhs) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)R * nfe) return;
  const int64_t e = t % nfe;
  if (feat_ok && feat_ok[e / mpad] < 0) {
    rhs[t] = 0.f;
    return;
  }
  float acc = Wbar[e] - muij[t];
  if (What) acc -= What[t];
  for (int s = 0; s < nsplit; ++s) acc += Rpart[(int64_t)s * R * nfe + t];
  rhs[t] = acc;
}

// W'_ij (+)= rhs_ij - Z_ij^T O'_ij from the R partials of the second pass-1 product (outer
// form of the projection; accumulate: the incremental projection adds the increment to
// W'_ij); padding feature slots zero
__global__ void k_sub_partials(const float* __restrict__ rhs, const float* __restrict__ Rpart, int nsplit, int R,
                               int64_t nfe, const int32_t* __restrict__ feat_ok, int mpad, float* __restrict__ What,
                               const uint8_t* __restrict__ bmask, const int64_t* __restrict__ col_slot, int C,
                               int accumulate) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)R * nfe) return;
  const int64_t e = t % nfe;
  if (bmask) {   // an inactive block keeps its W'_ij
    const int64_t slot = e / mpad;
    int j = 0;
    while (j + 1 < C && col_slot[j + 1] <= slot) ++j;
    if (!bmask[(t / nfe) * C + j]) return;
  }
  if (feat_ok[e / mpad] < 0) {
    What[t] = 0.f;
    return;
  }
  float acc = 0.f;
  for (int s = 0; s < nsplit; ++s) acc += Rpart[(int64_t)s * R * nfe + t];
  What[t] = (accumulate ? What[t] : 0.f) + (rhs[t] - acc);
}

// outer form: e_ij = O'_ij + U_i - u_ij, written over u (every block j of the same rows)
__global__ void k_outer_residual(float* __restrict__ u, const float* __restrict__ Op, const float* __restrict__ U,
                                 int64_t nrow_elems, int C) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nrow_elems * C) return;
  u[t] = (Op[t] + U[t % nrow_elems]) - u[t];
}

// outer form: O'_ij += U_i + y_ij, blocks of inactive (i, j) untouched
__global__ void k_outer_update(float* __restrict__ Op, const float* __restrict__ U, const float* __restrict__ y,
                               int64_t nslots, int mpad, int R, int C, const int64_t* __restrict__ row_slot,
                               const uint8_t* __restrict__ bmask) {
  const int64_t nre = nslots * mpad;
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= nre * C) return;
  const int64_t e = t % nre;
  if (bmask) {
    const int64_t slot = e / mpad;
    int i = 0;
    while (i + 1 < R && row_slot[i + 1] <= slot) ++i;
    if (!bmask[i * C + (int)(t / nre)]) return;
  }
  Op[t] += U[e] + y[t];
}

// dst[c][r] = src[r][c] (src rows x cols, dst ld dld)
__global__ void k_transpose_f32(const float* __restrict__ src, int64_t rows, int64_t cols, float* __restrict__ dst,
                                int64_t dld) {
  __shared__ float tile[32][33];
  const int64_t r0 = (int64_t)blockIdx.x * 32, c0 = (int64_t)blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  for (int rr = ty; rr < 32; rr += 8) {
    const int64_t r = r0 + rr, c = c0 + tx;
    tile[rr][tx] = (r < rows && c < cols) ? src[r * cols + c] : 0.f;
  }
  __syncthreads();
  for (int cc = ty; cc < 32; cc += 8) {
    const int64_t c = c0 + cc, r = r0 + tx;
    if (c < cols && r < rows) dst[c * dld + r] = tile[tx][cc];
  }
}

// Double-float arithmetic on the FP32 pipes (this part's FP64 pipe runs at 1/64 of the FP32
// rate): Knuth's TwoSum and Dekker's Fast2Sum, every operation rounded on its own.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
  return FF{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ FF ff_fast(float a, float b) {   // |a| >= |b| or a == 0
  const float s = __fadd_rn(a, b);
  return FF{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ FF ff_add_f(FF x, float y) {
  const FF t = ff_two_sum(x.hi, y);
  return ff_fast(t.hi, __fadd_rn(t.lo, x.lo));
}
// x / c for a small positive integer c (exact in FP32): the remainder x.hi - q c is exact
// through the FMA
__device__ __forceinline__ FF ff_div_int(FF x, float c) {
  const float q1 = __fdiv_rn(x.hi, c);
  const float r = __fadd_rn(__fmaf_rn(-q1, c, x.hi), x.lo);
  return ff_fast(q1, __fdiv_rn(r, c));
}
// RN32(y + x - m) for a pair m: (y + x) as a pair, minus m, rounded once at the end
__device__ __forceinline__ float ff_round_sum(float y, float x, FF m) {
  FF t = ff_two_sum(y, x);
  t = ff_add_f(t, -m.hi);
  t = ff_add_f(t, -m.lo);
  return __fadd_rn(t.hi, t.lo);
}

// Wbar = (W + sum_i W'_ij)/(R+1), mu += W - Wbar, mu'_ij += W'_ij - Wbar.  The average and
// the dual updates are formed in double-float arithmetic from the FP32 operands (about 2^-47
// relative), and each result is rounded to FP32 once: the duals add up W - Wbar over the
// iterations, and an FP32 average would hand them its rounding every time (an error that
// grows with the iteration count).
__global__ void k_avg_dual(const float* __restrict__ W, const float* __restrict__ What, int R, int64_t nfe,
                           float* __restrict__ Wbar, float* __restrict__ mu, float* __restrict__ muij) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= nfe) return;
  const float w = W[e];
  FF s{w, 0.f};
  for (int i = 0; i < R; ++i) s = ff_add_f(s, What[(int64_t)i * nfe + e]);
  const FF wb = ff_div_int(s, (float)(R + 1));
  Wbar[e] = __fadd_rn(wb.hi, wb.lo);
  mu[e] = ff_round_sum(mu[e], w, wb);
  for (int i = 0; i < R; ++i) {
    const int64_t t = (int64_t)i * nfe + e;
    muij[t] = ff_round_sum(muij[t], What[t], wb);
  }
}

// src [b][rows][cols] float32 -> hi/lo [b][cols][dst_ld] BF16, 32 x 32 smem tiles
// The transposed FP16 split of a row-major FP32 matrix, scaled by a power of two:
// amax (device, max |src| as float bits) selects it (f16_scale), else scale.
__global__ void k_transpose_split_f16(const float* __restrict__ src, int64_t rows, int cols, int64_t sbs,
                                      __half* __restrict__ hi, __half* __restrict__ lo, int64_t dld, int64_t dbs,
                                      float scale, const unsigned* __restrict__ amax) {
  __shared__ float tile[32][33];
  const float sc = amax ? f16_scale(__uint_as_float(*amax)) : scale;
  const int b = blockIdx.z;
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 256 threads: 8 rows per pass
  for (int rr = ty; rr < 32; rr += 8) {
    const int64_t r = r0 + rr;
    const int c = c0 + tx;
    tile[rr][tx] = (r < rows && c < cols) ? src[b * sbs + r * cols + c] : 0.f;
  }
  __syncthreads();
  for (int cc = ty; cc < 32; cc += 8) {
    const int c = c0 + cc;
    const int64_t r = r0 + tx;
    if (c < cols && r < rows) {
      __half h, l;
      split_f16(tile[tx][cc], sc, h, l);
      hi[b * dbs + (int64_t)c * dld + r] = h;
      lo[b * dbs + (int64_t)c * dld + r] = l;
    }
  }
}

__global__ void k_transpose_split(const float* __restrict__ src, int64_t rows, int cols, int64_t sbs,
                                  __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int64_t dld,
                                  int64_t dbs) {
  __shared__ float tile[32][33];
  const int b = blockIdx.z;
  const int64_t r0 = (int64_t)blockIdx.x * 32;
  const int c0 = blockIdx.y * 32;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 256 threads: 8 rows per pass
  for (int rr = ty; rr < 32; rr += 8) {
    const int64_t r = r0 + rr;
    const int c = c0 + tx;
    tile[rr][tx] = (r < rows && c < cols) ? src[b * sbs + r * cols + c] : 0.f;
  }
  __syncthreads();
  for (int cc = ty; cc < 32; cc += 8) {
    const int c = c0 + cc;
    const int64_t r = r0 + tx;
    if (c < cols && r < rows) {
      __nv_bfloat16 h, l;
      split_bf16(tile[tx][cc], h, l);
      hi[b * dbs + (int64_t)c * dld + r] = h;
      lo[b * dbs + (int64_t)c * dld + r] = l;
    }
  }
}

template <int NT>
__device__ __forceinline__ double block_sum(double x) {
  __shared__ double red[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x / 32] = x;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < NT / 32; ++w) s += red[w];
  return s;
}

__global__ void __launch_bounds__(256) k_sqdiff(const float* __restrict__ a, const float* __restrict__ b, int64_t n,
                                                double* __restrict__ partials) {
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double d = (double)a[e] - (b ? (double)b[e] : 0.0);
    acc += d * d;
  }
  const double s = block_sum<256>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_loss_sum(int loss, const float* __restrict__ Y, const float* __restrict__ S,
                                                  const int32_t* __restrict__ row_ok, int64_t nslots, int m, int mpad,
                                                  double* __restrict__ partials) {
  double acc = 0.0;
  for (int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; p < nslots;
       p += (int64_t)gridDim.x * blockDim.x) {
    if (row_ok[p] < 0) continue;
    const float* y = Y + p * mpad;
    const float* o = S + p * mpad;
    if (loss == LOSS_MULTINOMIAL) {
      double mx = -1e300, yb = -1e300;
      int c = 0;
      for (int k = 0; k < m; ++k) {
        mx = fmax(mx, (double)o[k]);
        if (y[k] > yb) { yb = y[k]; c = k; }
      }
      double se = 0.0;
      for (int k = 0; k < m; ++k) se += exp((double)o[k] - mx);
      acc += mx + log(se) - (double)o[c];
    } else if (loss == LOSS_CRAMMER_SINGER) {
      double yb = -1e300;
      int c = 0;
      for (int k = 0; k < m; ++k)
        if (y[k] > yb) { yb = y[k]; c = k; }
      double mx = 0.0;   // the k = c term
      for (int k = 0; k < m; ++k)
        if (k != c) mx = fmax(mx, 1.0 + (double)o[k] - (double)o[c]);
      acc += mx;
    } else {
      for (int k = 0; k < m; ++k) {
        const double yy = y[k], oo = o[k];
        if (loss == LOSS_SQUARED) acc += (yy - oo) * (yy - oo);
        else if (loss == LOSS_HINGE) acc += fmax(0.0, 1.0 - yy * oo);
        else if (loss == LOSS_L1) acc += fabs(yy - oo);
        else acc += (-yy * oo > 0 ? -yy * oo + log1p(exp(yy * oo)) : log1p(exp(-yy * oo)));
      }
    }
  }
  const double s = block_sum<256>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// sum_e w_c r(W_e), c = e mod ncol (w null: all weights 1)
__global__ void __launch_bounds__(256) k_reg_sum(int reg, const float* __restrict__ W, int64_t n,
                                                 const float* __restrict__ w, int ncol,
                                                 double* __restrict__ partials) {
  double acc = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    acc += (w ? (double)w[e % ncol] : 1.0) * (reg == 0 ? (double)W[e] * W[e] : fabs((double)W[e]));
  const double s = block_sum<256>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

__global__ void k_f64_to_f32(const double* __restrict__ s, float* __restrict__ d, int64_t n) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < n) d[e] = (float)s[e];
}

// flag |= 1 for a NaN/Inf entry; with pm1, flag |= 2 for an entry outside {-1, +1}
// flag |= 1 for NaN/Inf, 2 for a value other than +-1 (pm1); maxbits = max |x| of the
// finite values as float bits (unsigned order equals float order for x >= 0)
__global__ void k_finite(const float* __restrict__ x, int64_t n, int pm1, int* __restrict__ flag,
                         unsigned* __restrict__ maxbits) {
  int f = 0;
  float mx = 0.f;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const float v = x[e];
    if (!isfinite(v)) f |= 1;
    else mx = fmaxf(mx, fabsf(v));
    if (pm1 == 1 && v != 1.f && v != -1.f) f |= 2;
    if (pm1 == 2 && v < 0.f) f |= 4;
  }
  if (f) atomicOr(flag, f);
  if (maxbits) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.f) atomicMax(maxbits, __float_as_uint(mx));
  }
}

__global__ void k_set_diag(double* __restrict__ A, int64_t ld, int64_t s, double v) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < s) A[t * ld + t] = v;
}

inline unsigned nblk(int64_t n, int bs = 256) { return (unsigned)ceil_div(n, bs); }

}  // namespace

cudaError_t launch_gather_rows(const float* src, int64_t lds, int64_t w, const int32_t* map, int64_t nrows,
                               float* dst, int64_t ld, cudaStream_t st) {
  if (nrows * ld <= 0) return cudaSuccess;
  k_scatter_rows<<<nblk(nrows * ld), 256, 0, st>>>(src, lds, w, map, nrows, dst, ld);
  return cudaGetLastError();
}

cudaError_t launch_set_column(float* X, int64_t ld, int64_t rows, int64_t col, float v, cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  k_set_column<<<nblk(rows), 256, 0, st>>>(X, ld, rows, col, v);
  return cudaGetLastError();
}

cudaError_t launch_split_f16(const float* src, int64_t n, float scale, __half* hi, __half* lo, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_split_f16<<<nblk(n), 256, 0, st>>>(src, n, scale, hi, lo);
  return cudaGetLastError();
}

cudaError_t launch_split_bf16(const float* src, int64_t n, __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_split<<<nblk(n), 256, 0, st>>>(src, n, hi, lo);
  return cudaGetLastError();
}

cudaError_t launch_csr_check(const int64_t* indptr, const int32_t* indices, int64_t n, int64_t d, int64_t nnz,
                             int* flag, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_csr_check<<<nblk(n), 256, 0, st>>>(indptr, indices, n, d, nnz, flag);
  return cudaGetLastError();
}

cudaError_t launch_scatter_csr(const int64_t* indptr, const int32_t* indices, const float* values,
                               const int32_t* map, int64_t nrows, float* dst, int64_t ld, cudaStream_t st) {
  if (nrows <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(dst, 0, (size_t)nrows * ld * sizeof(float), st);
  if (e != cudaSuccess) return e;
  k_scatter_csr<<<nblk(nrows), 256, 0, st>>>(indptr, indices, values, map, nrows, dst, ld);
  return cudaGetLastError();
}

cudaError_t launch_prox_loss(int loss, const float* V, const float* Y, int64_t n, int m, int64_t ld, float t,
                             int newton, float* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (m > 32 * MAXPL) return cudaErrorInvalidValue;
  const int64_t threads = row_loss(loss) ? n * 32 : n * m;
  k_prox_loss<<<nblk(threads), 256, 0, st>>>(loss, V, Y, n, m, ld, t, newton, out);
  return cudaGetLastError();
}

cudaError_t launch_prox_reg(int reg, const float* V, const float* mu, int64_t n, float tau, float* out,
                            cudaStream_t st, const float* tau_col, int ncol) {
  if (n <= 0) return cudaSuccess;
  k_prox_reg<<<nblk(n), 256, 0, st>>>(reg, V, mu, n, tau, tau_col, ncol > 0 ? ncol : 1, out);
  return cudaGetLastError();
}

cudaError_t launch_row_epilogue(const RowEpiArgs& a, cudaStream_t st) {
  if (a.nslots <= 0) return cudaSuccess;
  if (a.mpad > 32 * MAXPL || a.nslots % EX_ROWS) return cudaErrorInvalidValue;
  const bool split = a.VThi && a.VTlo && a.amax;
  if (!a.V32 && !split) return cudaErrorInvalidValue;
  const size_t smem = (size_t)EX_ROWS * (a.mpad + 1) * sizeof(float);
  const unsigned grid = (unsigned)(a.nslots / EX_ROWS);
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    const int mx = EX_ROWS * (32 * MAXPL + 1) * (int)sizeof(float);
    attr = cudaFuncSetAttribute(k_exchange<LOSS_SQUARED>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_exchange<LOSS_HINGE>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_exchange<LOSS_LOGISTIC>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_exchange<LOSS_MULTINOMIAL>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_exchange<LOSS_L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    if (attr == cudaSuccess)
      attr = cudaFuncSetAttribute(k_exchange<LOSS_CRAMMER_SINGER>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
  });
  if (attr != cudaSuccess) return attr;
  switch (a.loss) {
    case LOSS_SQUARED: k_exchange<LOSS_SQUARED><<<grid, 256, smem, st>>>(a); break;
    case LOSS_HINGE: k_exchange<LOSS_HINGE><<<grid, 256, smem, st>>>(a); break;
    case LOSS_LOGISTIC: k_exchange<LOSS_LOGISTIC><<<grid, 256, smem, st>>>(a); break;
    case LOSS_MULTINOMIAL: k_exchange<LOSS_MULTINOMIAL><<<grid, 256, smem, st>>>(a); break;
    case LOSS_L1: k_exchange<LOSS_L1><<<grid, 256, smem, st>>>(a); break;
    case LOSS_CRAMMER_SINGER: k_exchange<LOSS_CRAMMER_SINGER><<<grid, 256, smem, st>>>(a); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_rhs(const float* Wbar, const float* muij, const float* Rpart, int nsplit, int R, int64_t nfe,
                       float* rhs, cudaStream_t st, const int32_t* feat_ok, int mpad, const float* What) {
  k_rhs<<<nblk((int64_t)R * nfe), 256, 0, st>>>(Wbar, muij, Rpart, nsplit, R, nfe, feat_ok, mpad > 0 ? mpad : 1,
                                                What, rhs);
  return cudaGetLastError();
}

cudaError_t launch_sub_partials(const float* rhs, const float* Rpart, int nsplit, int R, int64_t nfe,
                                const int32_t* feat_ok, int mpad, float* What, cudaStream_t st, const uint8_t* bmask,
                                const int64_t* col_slot, int C, int accumulate) {
  k_sub_partials<<<nblk((int64_t)R * nfe), 256, 0, st>>>(rhs, Rpart, nsplit, R, nfe, feat_ok, mpad, What, bmask,
                                                          col_slot, C, accumulate);
  return cudaGetLastError();
}

cudaError_t launch_outer_residual(float* u, const float* Op, const float* U, int64_t nslots, int mpad, int C,
                                  cudaStream_t st) {
  const int64_t n = nslots * mpad * C;
  if (n <= 0) return cudaSuccess;
  k_outer_residual<<<nblk(n), 256, 0, st>>>(u, Op, U, nslots * mpad, C);
  return cudaGetLastError();
}

cudaError_t launch_outer_update(float* Op, const float* U, const float* y, int64_t nslots, int mpad, int R, int C,
                                const int64_t* d_row_slot, const uint8_t* bmask, cudaStream_t st) {
  const int64_t n = nslots * mpad * C;
  if (n <= 0) return cudaSuccess;
  k_outer_update<<<nblk(n), 256, 0, st>>>(Op, U, y, nslots, mpad, R, C, d_row_slot, bmask);
  return cudaGetLastError();
}

cudaError_t launch_transpose_f32(const float* src, int64_t rows, int64_t cols, float* dst, int64_t dld,
                                 cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  dim3 grid((unsigned)ceil_div(rows, 32), (unsigned)ceil_div(cols, 32));
  k_transpose_f32<<<grid, 256, 0, st>>>(src, rows, cols, dst, dld);
  return cudaGetLastError();
}

cudaError_t launch_avg_dual(const float* W, const float* What, int R, int64_t nfe, float* Wbar, float* mu,
                            float* muij, cudaStream_t st) {
  k_avg_dual<<<nblk(nfe), 256, 0, st>>>(W, What, R, nfe, Wbar, mu, muij);
  return cudaGetLastError();
}

cudaError_t launch_transpose_split_f16(const float* src, int64_t rows, int cols, int nbatch, int64_t src_batch_stride,
                                       __half* hi, __half* lo, int64_t dst_ld, int64_t dst_batch_stride, float scale,
                                       const unsigned* amax, cudaStream_t st) {
  if (rows <= 0 || cols <= 0 || nbatch <= 0) return cudaSuccess;
  dim3 grid((unsigned)ceil_div(rows, 32), (unsigned)ceil_div(cols, 32), (unsigned)nbatch);
  k_transpose_split_f16<<<grid, 256, 0, st>>>(src, rows, cols, src_batch_stride, hi, lo, dst_ld, dst_batch_stride,
                                              scale, amax);
  return cudaGetLastError();
}

cudaError_t launch_transpose_split(const float* src, int64_t rows, int cols, int nbatch, int64_t src_batch_stride,
                                   __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t dst_ld, int64_t dst_batch_stride,
                                   cudaStream_t st) {
  if (rows <= 0 || cols <= 0 || nbatch <= 0) return cudaSuccess;
  dim3 grid((unsigned)ceil_div(rows, 32), (unsigned)ceil_div(cols, 32), (unsigned)nbatch);
  k_transpose_split<<<grid, 256, 0, st>>>(src, rows, cols, src_batch_stride, hi, lo, dst_ld, dst_batch_stride);
  return cudaGetLastError();
}

cudaError_t launch_sqdiff_partials(const float* a, const float* b, int64_t n, double* partials, int nblocks,
                                   cudaStream_t st) {
  k_sqdiff<<<nblocks, 256, 0, st>>>(a, b, n, partials);
  return cudaGetLastError();
}

cudaError_t launch_loss_partials(int loss, const float* Y, const float* S, const int32_t* row_ok, int64_t nslots,
                                 int m, int mpad, double* partials, int nblocks, cudaStream_t st) {
  k_loss_sum<<<nblocks, 256, 0, st>>>(loss, Y, S, row_ok, nslots, m, mpad, partials);
  return cudaGetLastError();
}

cudaError_t launch_reg_partials(int reg, const float* W, int64_t n, double* partials, int nblocks, cudaStream_t st,
                                const float* w, int ncol) {
  k_reg_sum<<<nblocks, 256, 0, st>>>(reg, W, n, w, ncol > 0 ? ncol : 1, partials);
  return cudaGetLastError();
}

cudaError_t launch_convert_f64_f32(const double* src, float* dst, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_f64_to_f32<<<nblk(n), 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_finite_check(const float* x, int64_t n, int pm1, int* flag, cudaStream_t st, unsigned* maxbits) {
  if (n <= 0) return cudaSuccess;
  k_finite<<<(unsigned)std::min<int64_t>(ceil_div(n, 256), 4096), 256, 0, st>>>(x, n, pm1, flag, maxbits);
  return cudaGetLastError();
}

// Four consecutive columns per thread: the pieces' float4 loads are all issued before the
// sums (which keep the pieces' order), and H is updated by two double2 read-modify-writes
// where the address is 16-byte aligned (H itself may start on an 8-byte boundary).
constexpr int GRAM_PIECES_MAX = 16;

__global__ void k_gram_reduce(const float* __restrict__ P, int nchunk, int ntiles, const int2* __restrict__ tiles,
                              int64_t s, double* __restrict__ H, int64_t ldh) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= (int64_t)ntiles * 128 * 64) return;
  const int tile = (int)(t / (128 * 64)), e = (int)(t % (128 * 64)) * 4;
  const int64_t row = tiles[tile].x + e / 256, col = tiles[tile].y + e % 256;
  if (row >= s || col > row) return;
  float4 p[GRAM_PIECES_MAX];
#pragma unroll
  for (int c = 0; c < GRAM_PIECES_MAX; ++c)
    if (c < nchunk) p[c] = *reinterpret_cast<const float4*>(P + ((int64_t)c * ntiles + tile) * (128 * 256) + e);
  // the pieces' sum as a float pair (TwoSum: exact but for the pair's own rounding, ~2^-48),
  // turned into FP64 by integer instructions: two FP64 additions per element, not 2 nchunk
  float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int c = 0; c < GRAM_PIECES_MAX; ++c)
    if (c < nchunk) {
      two_sum_into(hi[0], lo[0], p[c].x);
      two_sum_into(hi[1], lo[1], p[c].y);
      two_sum_into(hi[2], lo[2], p[c].z);
      two_sum_into(hi[3], lo[3], p[c].w);
    }
  double v[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) v[q] = f32_to_f64_scaled(hi[q], 0) + f32_to_f64_scaled(lo[q], 0);
  double* h = H + row * ldh + col;
  if (col + 3 <= row && (reinterpret_cast<uintptr_t>(h) & 15) == 0) {
    double2* h2 = reinterpret_cast<double2*>(h);
    double2 a = h2[0], b = h2[1];
    a.x += v[0];
    a.y += v[1];
    b.x += v[2];
    b.y += v[3];
    h2[0] = a;
    h2[1] = b;
  } else {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (col + q <= row) h[q] += v[q];
  }
}

cudaError_t launch_gram_reduce(const float* P, int nchunk, int ntiles, const int2* tiles, int64_t s, double* H,
                               int64_t ldh, cudaStream_t st) {
  if (ntiles <= 0 || nchunk <= 0) return cudaSuccess;
  if (nchunk > GRAM_PIECES_MAX) return cudaErrorInvalidValue;
  k_gram_reduce<<<nblk((int64_t)ntiles * 128 * 64), 256, 0, st>>>(P, nchunk, ntiles, tiles, s, H, ldh);
  return cudaGetLastError();
}

// one warp per row: lane-strided maximum, then a butterfly keeping the lowest index on ties
__global__ void k_argmax_rows(const float* __restrict__ S, int64_t q, int m, int64_t ld, int32_t* __restrict__ labels) {
  const int64_t row = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) / 32;
  const int lane = threadIdx.x & 31;
  if (row >= q) return;
  const float* s = S + row * ld;
  if (m == 1) {
    if (lane == 0) labels[row] = s[0] >= 0.f ? 1 : -1;
    return;
  }
  float best = -INFINITY;
  int bi = 1 << 30;
  for (int k = lane; k < m; k += 32)
    if (s[k] > best) { best = s[k]; bi = k; }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float ob = __shfl_xor_sync(0xffffffffu, best, o);
    const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
    if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
  }
  if (lane == 0) labels[row] = bi;
}

cudaError_t launch_argmax_rows(const float* scores, int64_t q, int m, int64_t ld, int32_t* labels, cudaStream_t st) {
  if (q <= 0) return cudaSuccess;
  k_argmax_rows<<<nblk(q * 32), 256, 0, st>>>(scores, q, m, ld, labels);
  return cudaGetLastError();
}

cudaError_t launch_set_diag(double* A, int64_t ld, int64_t s, double v, cudaStream_t st) {
  if (s <= 0) return cudaSuccess;
  k_set_diag<<<nblk(s), 256, 0, st>>>(A, ld, s, v);
  return cudaGetLastError();
}

RFF_CHECK_UNIT(elementwise)

}  // namespace rff
