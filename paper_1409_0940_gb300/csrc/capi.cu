// The C ABI of include/rff_admm.h: handle, device memory, set-up (Philox draw,
// Gram matrices, FP64 Cholesky, cached inverses) and the iteration schedule of
// block-splitting ADMM (Sec. 3, update equations around eq. (gp), in the
// reorganised form: O'_ij kept per block, Z_ij regenerated twice per iteration).
#include "../../include/rff_admm.h"
#include "common.cuh"
#include "internal.h"
#include "tc.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

using namespace rff;

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

constexpr int64_t TS_SCORE_ROWS = 2048;   // TensorSketch scoring: rows sketched per product

// A named host range for profilers (NVTX; nothing happens unless a tool is attached): the
// set-up stages, the iterations and scoring show up by name on a timeline.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace

struct rff_admm_s {
  rff_admm_params p{};
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::string err;

  // ---- geometry
  bool has_data = false, factored = false;
  int64_t bias_col = -1;  // split path: column of X (ones) and G (b) that folds b into X.G
  size_t mem_limit = 0;   // device bytes this handle may use (0: whatever is free)
  int64_t n = 0, d = 0, dld = 0, m = 0, mpad = 0, D = 0, nslots = 0, fslots = 0;
  int R = 1, C = 1, nsplit = 1, nsplit_max = 1, iters_done = 0;
  int tc_kc = 0;  // ring K chunk of the tensor-core passes, chosen by the autotuner
  int tc_zt = 0;  // 1: Z tile of the tensor-core passes in TMEM (autotuned)
  int tc_cg = 1;  // 2: the tensor-core passes run as CTA pairs (autotuned)
  float t_loss = 0.f, t_reg = 0.f;
  std::vector<int64_t> row_start, row_size, row_slot, col_start, col_size, col_slot, foff;

  // ---- device memory (owned)
  std::vector<DevBuf> bufs;
  int32_t *row_of_slot = nullptr, *feat_of_slot = nullptr, *slot_of_feat = nullptr;
  int64_t *d_row_slot = nullptr, *d_row_size = nullptr, *d_col_slot = nullptr, *d_col_size = nullptr;
  int64_t* d_zero = nullptr;  // {0}: row block table of a query batch
  float *X32 = nullptr, *Gt32 = nullptr, *bias = nullptr, *Y = nullptr;
  // split path: X * xscale and G * gscale as FP16 hi/lo pairs (powers of two, |.| <= 2^8)
  __half *Xhi = nullptr, *Xlo = nullptr, *Ghi = nullptr, *Glo = nullptr;
  float xscale = 1.f, gscale = 1.f;
  float *O = nullptr, *Obar = nullptr, *nu = nullptr, *Op = nullptr;
  float* V32 = nullptr;       // V_ij = Obar_ij + nu_i, C x slots x mpad (FP32 path)
  // split path: the chained operands V^T, W'^T, Wbar^T as FP16 hi/lo pairs, each scaled by
  // f16_scale of a maximum or bound; the maxima (float bits) live in amax (AMAX_* words)
  unsigned* amax = nullptr;
  __half *VThi = nullptr, *VTlo = nullptr, *WThi = nullptr, *WTlo = nullptr, *WbThi = nullptr,
                *WbTlo = nullptr;
  float *W = nullptr, *Wbar = nullptr, *mu = nullptr, *What = nullptr, *muij = nullptr, *rhs = nullptr,
        *Rpart = nullptr;
  float* Q32 = nullptr;       // cached (I + Z_ij^T Z_ij)^-1 per block (float32 path), or the
                              // (I + Z_ij Z_ij^T)^-1 of the outer form (both paths)
  // outer form of the graph projection (eq. (graphU) via the identity of Sec. 3 with
  // (I + Z Z^T)^-1, chosen when every block has fewer rows than features): u = Z rhs
  bool outer = false;
  float* U32 = nullptr;       // C x slots x mpad
  // split path: the cached inverses split three ways into BF16, blocks stacked by rows
  // (block b from row qrow[b], rows padded to 128, ldq columns), and the right-hand
  // side of the projection split the same way, transposed to [R][mpad][fslots]
  __nv_bfloat16 *Q1 = nullptr, *Q2 = nullptr, *Q3 = nullptr, *rT1 = nullptr, *rT2 = nullptr, *rT3 = nullptr;
  int64_t ldq = 0, q_rows = 0;
  std::vector<int64_t> qrow;
  SgJob* qjobs = nullptr;     // projection GEMM jobs (one per 128-row tile of every Q_ij)
  int nqjobs = 0;
  // cached-Z precision: Z (n_slots x D_slots) and Z^T as hi/lo pairs, and the jobs of
  // the two streamed passes
  __half *Zhi = nullptr, *Zlo = nullptr, *ZThi = nullptr, *ZTlo = nullptr;   // FP16 split of zscale Z
  float zscale = 1.f;
  float ts_zmax = 0.f;           // TensorSketch: max |z| over the training rows (the split's scale)
  float* ts_buf = nullptr;       // TensorSketch scoring: TS_SCORE_ROWS rows of features
  SgJob *p1jobs = nullptr, *p2jobs = nullptr;
  int np1 = 0, np2 = 0, nsplit_cz = 1;
  // stochastic block subsets: a block is active in an iteration when its Philox word is
  // below bthr (= floor(p 2^24); 2^24: every block, the deterministic method)
  double bfrac = 1.0;
  uint32_t bthr = 1u << 24;
  uint8_t* bmask = nullptr;   // R x C, this iteration's active blocks (device)
  int64_t* bctr = nullptr;    // the iteration number the next mask is drawn for (device)
  int64_t bctr_host = 0;
  bool stochastic() const { return bthr < (1u << 24); }
  // the feature parameters' device copies (G or V or W, and their FP16 split) were given back:
  // they are regenerated from Philox when next needed
  bool features_released = false;
  const uint8_t* act() const { return stochastic() ? bmask : nullptr; }
  std::vector<double> lam_col;  // lambda of each output column (empty: params.lambda for all)
  float* lam_dev = nullptr;     // lambda_c / lambda per column (m_pad), or null
  GemmDesc* gdesc = nullptr;  // R*C
  double* partials = nullptr;
  int* flag = nullptr;
  float *nu_old = nullptr, *Obar_old = nullptr, *mu_old = nullptr, *Wbar_old = nullptr, *muij_old = nullptr;
  // grow-only scratch for queries and staging
  DevBuf scratch;
  // profiling: phase events per iteration, accumulated at the end of a solve call
  bool profiling = false;
  rff_admm_profile prof{};
  std::vector<cudaEvent_t> ev;
  int64_t launches = 0;
  int pending_profiled = 0;   // profiled iterations enqueued since the last accumulation
  // one iteration captured as a CUDA graph (after an eager first iteration)
  cudaGraphExec_t gexec = nullptr;
  void drop_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
  }

  // Device memory is stream-ordered (cudaMallocAsync / cudaFreeAsync on the handle's
  // stream): allocating or releasing it never waits for other handles' work on the
  // device, which matters when solves and scoring requests share a GPU.
  ~rff_admm_s() {
    drop_graph();
    for (auto e : ev) cudaEventDestroy(e);
    free_all();
    if (scratch.p) cudaFreeAsync(scratch.p, st);
    cudaStreamSynchronize(st);
    if (own_stream && st) cudaStreamDestroy(st);
  }
  void free_all() {
    for (auto& b : bufs)
      if (b.p) cudaFreeAsync(b.p, st);
    bufs.clear();
  }
  rff_status fail(rff_status s, const std::string& msg) {
    err = msg;
    return s;
  }
  rff_status cuda_fail(cudaError_t e, const char* what) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    return RFF_ECUDA;
  }
  // the split path: tensor-core kernels and BF16 operand copies (cached-Z uses them too)
  bool split_path() const { return p.prec == RFF_PREC_SPLIT_BF16 || p.prec == RFF_PREC_CACHED_Z; }
  // scoring forms X.G on the tensor cores (split path; random Fourier or Fastfood map)
  bool tc_scores() const {
    return split_path() && p.feature_map != RFF_MAP_LAPLACE && p.feature_map != RFF_MAP_TENSORSKETCH;
  }
  bool tensorsketch() const { return p.feature_map == RFF_MAP_TENSORSKETCH; }
  // the feature map's scale: max |z| (sqrt(2/D) for cos, 1/sqrt(D) for exp(-T) with T >= 0)
  float zmap_scale() const {
    if (p.feature_map == RFF_MAP_TENSORSKETCH) return ts_zmax > 0.f ? ts_zmax : 1.f;   // measured, no a-priori bound
    return (float)(p.feature_map == RFF_MAP_LAPLACE ? 1.0 / std::sqrt((double)D) : std::sqrt(2.0 / (double)D));
  }
  bool cached_z() const { return p.prec == RFF_PREC_CACHED_Z; }
  // Gram form: the projection is taken incrementally (phase_project), and pass 1 reads one
  // operand U_i for every column block
  bool incremental() const { return !outer; }
  int64_t rpart_elems() const { return (int64_t)std::max(nsplit_max, nsplit_cz) * R * fslots * mpad; }
};

namespace rff {
TcView tc_view(const rff_admm_s& s);
}

#define CK(call)                                        \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return h->cuda_fail(e_, #call); \
  } while (0)

namespace {

// Largest power of two s with maxabs * s <= 2^8 (1 when maxabs is 0): the scale of the
// FP16 split of the X.G operands.
float pow2_scale(double maxabs) {
  if (!(maxabs > 0) || !std::isfinite(maxabs)) return 1.f;
  int e = (int)std::floor(std::log2(256.0 / maxabs));
  e = std::max(-100, std::min(100, e));
  return std::ldexp(1.0f, e);
}

// G ~ N(0, sigma^-2) from Box-Muller with u >= 2^-25 gives |G| <= sqrt(50 ln 2)/sigma
// < 5.9/sigma; the phase b lies in [0, pi).  Both share the scale of G's copies.
float g_scale(double sigma) { return pow2_scale(std::max(5.9 / sigma, 3.1415927)); }

// Queries go through the same FP16 scaling as the training rows: |x| xscale must stay
// below 2^15 (queries up to 2^7 times the largest training |x|).
rff_status check_query_range(rff_admm_t h, int maxbits) {
  if (!h->tc_scores()) return RFF_OK;
  float qmax = 0.f;
  memcpy(&qmax, &maxbits, 4);
  if ((double)qmax * h->xscale < 32768.0) return RFF_OK;
  return h->fail(RFF_EINVAL, "query values up to " + std::to_string(qmax) +
                                 " exceed the split path's input range (|x| < " + std::to_string(32768.0 / h->xscale) +
                                 ", at least 128 times the largest training |x|)");
}

rff_status check_params(const rff_admm_params* p, std::string& why) {
  if (!p) { why = "params is NULL"; return RFF_EINVAL; }
  if (p->loss < 0 || p->loss > 5) { why = "unknown loss"; return RFF_EINVAL; }
  if (p->reg < 0 || p->reg > 1) { why = "unknown regulariser"; return RFF_EINVAL; }
  if (p->prec < 0 || p->prec > 2) { why = "unknown precision"; return RFF_EINVAL; }
  if (p->rho_scale < 0 || p->rho_scale > 1) { why = "unknown rho scale"; return RFF_EINVAL; }
  if (!(p->lambda > 0) || !std::isfinite(p->lambda)) { why = "lambda must be > 0"; return RFF_EINVAL; }
  if (!(p->sigma > 0) || !std::isfinite(p->sigma)) { why = "sigma must be > 0"; return RFF_EINVAL; }
  if (!(p->rho > 0) || !std::isfinite(p->rho)) { why = "rho must be > 0"; return RFF_EINVAL; }
  if (p->D < 1 || p->D > (int64_t)1 << 30) { why = "D out of range"; return RFF_EINVAL; }
  if (p->R < 1 || p->C < 1 || p->C > p->D) { why = "bad block grid"; return RFF_EINVAL; }
  if (p->m < 1 || p->m > 256) { why = "m must be in [1, 256]"; return RFF_EINVAL; }
  if (p->newton_iters < 0 || p->newton_iters > 100) { why = "newton_iters out of range"; return RFF_EINVAL; }
  if (p->prec != RFF_PREC_FP32 && p->C > 64) { why = "the split-BF16 and cached-Z paths support C <= 64"; return RFF_EINVAL; }
  if (p->feature_map < 0 || p->feature_map > 3) { why = "unknown feature map"; return RFF_EINVAL; }
  if (p->feature_map == RFF_MAP_TENSORSKETCH) {
    if (p->prec != RFF_PREC_CACHED_Z) {
      // a sketch is a whole vector per block, not a tile function: Z is formed once and kept
      why = "TensorSketch features run on the cached-Z precision";
      return RFF_EINVAL;
    }
    if (p->degree < 1 || p->degree > TS_MAX_DEGREE) { why = "TensorSketch degree must be in [1, 8]"; return RFF_EINVAL; }
    if (!(p->coef0 >= 0) || !std::isfinite(p->coef0)) { why = "TensorSketch coef0 must be >= 0"; return RFF_EINVAL; }
    if ((p->D + p->C - 1) / p->C > TS_MAX_BLOCK) {
      why = "TensorSketch column blocks hold at most 8192 features";
      return RFF_EINVAL;
    }
  }
  if (p->feature_map == RFF_MAP_LAPLACE && p->prec == RFF_PREC_SPLIT_BF16) {
    // W is Levy-distributed: its range spans far more than the FP16 split's 2^29
    why = "the random Laplace map runs on the FP32 and cached-Z precisions";
    return RFF_EINVAL;
  }
  return RFF_OK;
}

void partition(int64_t total, int parts, std::vector<int64_t>& start, std::vector<int64_t>& size) {
  start.assign(parts, 0);
  size.assign(parts, 0);
  const int64_t q = total / parts, rem = total % parts;
  int64_t s = 0;
  for (int i = 0; i < parts; ++i) {
    size[i] = q + (i < rem ? 1 : 0);
    start[i] = s;
    s += size[i];
  }
}

template <typename T>
rff_status dalloc(rff_admm_t h, T*& ptr, size_t count) {
  void* p = nullptr;
  const size_t bytes = std::max<size_t>(count * sizeof(T), 16);
  cudaError_t e = cudaMallocAsync(&p, bytes, h->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return h->fail(RFF_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  h->bufs.push_back(DevBuf{p, bytes});
  ptr = static_cast<T*>(p);
  return RFF_OK;
}

rff_status ensure_scratch(rff_admm_t h, size_t bytes) {
  if (h->scratch.bytes >= bytes) return RFF_OK;
  if (h->scratch.p) {
    cudaFreeAsync(h->scratch.p, h->st);
    h->scratch = DevBuf{};
  }
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, h->st) != cudaSuccess) {
    cudaGetLastError();
    return h->fail(RFF_ENOMEM, "scratch allocation failed");
  }
  h->scratch = DevBuf{p, bytes};
  return RFF_OK;
}

// bytes of device memory the working set needs (checked before allocating)
size_t working_set_bytes(const rff_admm_s& s) {
  const size_t f = sizeof(float), b2 = 2;
  size_t t = 0;
  t += (size_t)s.nslots * 4 + (size_t)s.fslots * 4 * 2;
  if (s.split_path()) t += (size_t)s.nslots * s.dld * b2 * 2 + (size_t)s.fslots * s.dld * b2 * 2;
  if (!s.split_path() || s.cached_z()) t += (size_t)s.nslots * s.dld * f + (size_t)s.fslots * s.dld * f;
  t += (size_t)s.fslots * f;
  t += (size_t)s.nslots * s.mpad * f * (4 + 2);                 // Y, O, Obar, nu, nu_old, Obar_old
  t += (size_t)s.C * s.nslots * s.mpad * f * (s.split_path() && !s.outer ? 1 : 2);   // Op (+ FP32 V)
  if (s.split_path()) t += (size_t)s.C * s.nslots * s.mpad * b2 * 2;
  t += (size_t)s.fslots * s.mpad * f * 5;                       // W, Wbar, mu, mu_old, Wbar_old
  t += (size_t)s.R * s.fslots * s.mpad * f * (3 + s.nsplit_max);    // What, muij, muij_old, Rpart
  if (s.split_path()) {
    t += (size_t)s.R * s.fslots * s.mpad * b2 * 2 + (size_t)s.fslots * s.mpad * b2 * 2;         // WT, WbT
    if (!s.outer) {
      t += (size_t)s.R * s.fslots * s.mpad * b2 * 3;                                          // rT
      t += (size_t)s.q_rows * s.ldq * b2 * 3 + (size_t)s.R * s.C * (s.ldq / 128 + 1) * sizeof(SgJob);   // Q splits
    }
    if (s.cached_z()) {
      t += (size_t)s.nslots * s.fslots * b2 * 4;                                                // Z, Z^T hi/lo
      t += (size_t)(s.nslots / 128 * s.C + s.fslots / 128 * s.R * s.nsplit_cz) * sizeof(SgJob);
      t += (size_t)s.R * s.fslots * s.mpad * f * (s.nsplit_cz > s.nsplit_max ? s.nsplit_cz - s.nsplit_max : 0);
    }
  }
  if (!s.split_path() || s.outer) {
    t += (size_t)s.R * s.fslots * s.mpad * f;                                                   // rhs
    t += (size_t)s.foff.back() * f + (size_t)s.R * s.C * sizeof(GemmDesc);                     // factors
  }
  if (s.outer) t += (size_t)s.C * s.nslots * s.mpad * f * 2;                                   // e = V - Z c, y
  if (s.tensorsketch()) t += (size_t)TS_SCORE_ROWS * s.fslots * f + 256;   // scoring rows
  return t + (64u << 20);
}

// relative weights lambda_c / lambda of the output columns (padding columns 0)
rff_status upload_lambdas(rff_admm_t h) {
  auto& s = *h;
  if (!s.lam_dev) return RFF_OK;
  std::vector<float> w(s.mpad, 0.f);
  for (int64_t c = 0; c < s.m; ++c)
    w[c] = s.lam_col.empty() ? 1.f : (float)(s.lam_col[c] / s.p.lambda);
  CK(cudaMemcpyAsync(s.lam_dev, w.data(), w.size() * 4, cudaMemcpyHostToDevice, s.st));
  CK(cudaStreamSynchronize(s.st));
  return RFF_OK;
}

// Block grid, slot layout and prox steps of a data set of n rows and d inputs.
void compute_geometry(rff_admm_s& s, int64_t n, int64_t d) {
  s.n = n;
  s.d = d;
  s.dld = round_up(d, 64);
  // the split path folds the phase b into the tensor-core product when column d is free
  s.bias_col = (s.p.prec == RFF_PREC_SPLIT_BF16 && round_up(d + 1, 64) == s.dld) ? d : -1;
  s.m = s.p.m;
  s.mpad = round_up(s.m, 16);
  s.D = s.p.D;
  s.R = s.p.R;
  s.C = s.p.C;
  partition(n, s.R, s.row_start, s.row_size);
  partition(s.D, s.C, s.col_start, s.col_size);
  s.row_slot.assign(s.R, 0);
  s.col_slot.assign(s.C, 0);
  int64_t acc = 0;
  for (int i = 0; i < s.R; ++i) { s.row_slot[i] = acc; acc += round_up(s.row_size[i], SLOT); }
  s.nslots = acc;
  acc = 0;
  for (int j = 0; j < s.C; ++j) { s.col_slot[j] = acc; acc += round_up(s.col_size[j], SLOT); }
  s.fslots = acc;
  // the projection's cached factor per block: (I + Z^T Z)^-1 (s_j x s_j) or, when every
  // block has fewer rows than features, (I + Z Z^T)^-1 (n_i x n_i); the cached-Z
  // precision streams Z through the Gram form only
  {
    const int64_t nmax = *std::max_element(s.row_size.begin(), s.row_size.end());
    const int64_t smin = *std::min_element(s.col_size.begin(), s.col_size.end());
    s.outer = s.p.prec != RFF_PREC_CACHED_Z && nmax < smin;
  }
  s.foff.assign((size_t)s.R * s.C + 1, 0);
  for (int i = 0; i < s.R; ++i)
    for (int j = 0; j < s.C; ++j) {
      const int64_t fd = s.outer ? s.row_size[i] : s.col_size[j];
      s.foff[(size_t)i * s.C + j + 1] = s.foff[(size_t)i * s.C + j] + fd * fd;
    }
  s.qrow.assign((size_t)s.R * s.C, 0);
  s.q_rows = 0;
  s.ldq = 0;
  if (s.split_path() && !s.outer) {
    int64_t smax = 0;
    for (int j = 0; j < s.C; ++j) smax = std::max(smax, s.col_size[j]);
    s.ldq = round_up(smax, 32);
    for (int64_t b = 0; b < (int64_t)s.R * s.C; ++b) {
      s.qrow[b] = s.q_rows;
      s.q_rows += round_up(s.col_size[b % s.C], SLOT);
    }
  }
  const double nn = (double)n;
  if (s.p.rho_scale == RFF_RHO_SUM) {
    s.t_loss = (float)(1.0 / s.p.rho);
    s.t_reg = (float)(nn * s.p.lambda / s.p.rho);
  } else {
    s.t_loss = (float)(1.0 / (nn * s.p.rho));
    s.t_reg = (float)(s.p.lambda / s.p.rho);
  }
  // pass-1 row splits: enough CTAs for two waves on the device and, on the tensor-core
  // path, at most ~6400 rows per split: the FP32 accumulator of the tensor cores rounds
  // toward zero at every accumulation, so its error grows with the chain length; the
  // partial sums of the splits are added in FP32 with round-to-nearest afterwards.  The
  // FP32 path splits into chains of at most ~1600 rows: its FP32 sums of Z^T V over a
  // whole 50k-row block moved the weights of the multiclass workload by 5.3e-5 from the
  // FP64 iterate, ~6,250-row chains by 1.3e-5, ~1,600-row chains by 1.1e-5 (measured)
  {
    int nsm = 148, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const int64_t tile = s.split_path() ? 128 : 64;   // pass-1 row step of a split
    const int64_t ftiles = s.fslots / 128;             // pass-1 CTAs per row block and split
    int64_t min_rows = n;
    for (int i = 0; i < s.R; ++i) min_rows = std::min(min_rows, s.row_size[i]);
    int64_t want = ceil_div(2 * (int64_t)nsm, ftiles * s.R);
    want = std::max<int64_t>(want, ceil_div(min_rows, s.split_path() ? 6400 : 1600));
    const int64_t cap = std::min<int64_t>(ceil_div(min_rows, tile), 64);
    s.nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(want, cap));
    // RFF_PASS1_SPLITS=k fixes the row splits of pass 1 (bounded by one 128-row tile each)
    if (const char* e = getenv("RFF_PASS1_SPLITS")) {
      const int k = atoi(e);
      if (k >= 1) s.nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(k, ceil_div(min_rows, tile)));
    }
    s.nsplit_max = s.nsplit;
    // cached-Z pass 1 (one CTA per 128 features x row range, two CTAs per SM): about
    // twelve waves of jobs, every split at least eight 128-row tiles of every row block
    s.nsplit_cz = 1;
    if (s.cached_z()) {
      const int64_t ft = s.fslots / 128;
      const int64_t nrt = ceil_div(min_rows, 128);
      const int64_t want_cz = ceil_div(24 * (int64_t)nsm, ft * s.R);
      s.nsplit_cz = (int)std::max<int64_t>(1, std::min<int64_t>({want_cz, nrt / 8, (int64_t)64}));
    }
  }

}

// Bytes of set-up scratch for one block batch (FP64 Gram and inverse of `batch`
// blocks, one materialised row chunk of Z, factorisation scratch).
// Split-path Gram on the tensor cores (Gram form): per row chunk of Z, Z^T as a scaled FP16
// hi/lo pair and 128 x 256 tiles of Z^T Z over 512-row pieces of K, GRAM_GROUP pieces per
// launch, their partial tiles summed into H in FP64.
constexpr int GRAM_KCH = 512, GRAM_GROUP = 16;

int64_t tc_gram_tiles(int64_t smax, std::vector<int2>* out = nullptr) {
  const int64_t spad = round_up(smax, 256);
  int64_t n = 0;
  for (int64_t a = 0; a < spad / 128; ++a)
    for (int64_t b = 0; b * 256 <= a * 128 + 127 && b < spad / 256; ++b) {
      if (out) out->push_back(make_int2((int)(a * 128), (int)(b * 256)));
      ++n;
    }
  return n;
}

size_t tc_gram_bytes(int64_t chunk_rows, int64_t smax) {
  const int64_t spad = round_up(smax, 256), kpad = round_up(chunk_rows, GRAM_KCH), nt = tc_gram_tiles(smax);
  return round_up((size_t)spad * kpad * 2, 256) * 2 + (size_t)GRAM_GROUP * nt * 128 * 256 * 4 +
         round_up((size_t)nt * sizeof(int2), 256) + round_up((size_t)(kpad / GRAM_KCH) * nt * sizeof(SgJob), 256) + 1024;
}

bool tc_gram(const rff_admm_s& s) { return s.split_path() && !s.outer; }

// rows of Z formed per chunk on the cached-Z precision (about 256 MB of FP32)
int64_t materialise_chunk(const rff_admm_s& s) {
  return std::max<int64_t>(128, ((int64_t)(256u << 20) / (s.fslots * 4)) / 128 * 128);
}

size_t setup_bytes(const rff_admm_s& s, int64_t batch) {
  int64_t smax = 0;
  for (int j = 0; j < s.C; ++j) smax = std::max(smax, s.col_size[j]);
  const int64_t chunk_rows = std::min<int64_t>(32768, round_up(*std::max_element(s.row_size.begin(), s.row_size.end()), SLOT));
  const size_t t = (size_t)batch * smax * smax * 8 * 2 + (size_t)chunk_rows * smax * 4 +
                   factor_scratch_bytes((int)batch, (int)smax) + (size_t)batch * 4 + 4096 +
                   (tc_gram(s) ? tc_gram_bytes(chunk_rows, smax) : 0);
  // the cached-Z precision forms Z in the same scratch first, in row chunks of ~256 MB
  return s.cached_z() ? std::max(t, (size_t)materialise_chunk(s) * s.fslots * 4) : t;
}

}  // namespace

extern "C" {

rff_status rff_admm_create(const rff_admm_params* params, void* stream, rff_admm_t* out) {
  if (!out) return RFF_EINVAL;
  *out = nullptr;
  std::string why;
  rff_status s = check_params(params, why);
  if (s != RFF_OK) return s;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return RFF_ECUDA;
  }
  rff_admm_t h = new rff_admm_s();
  h->p = *params;
  if (h->p.newton_iters == 0) h->p.newton_iters = 8;
  if (stream) {
    h->st = static_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&h->st, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete h;
      return RFF_ECUDA;
    }
    h->own_stream = true;
  }
  *out = h;
  return RFF_OK;
}

rff_status rff_admm_set_profiling(rff_admm_t h, int enable) {
  if (!h) return RFF_EINVAL;
  h->profiling = enable != 0;
  h->prof = rff_admm_profile{};
  h->launches = 0;
  return RFF_OK;
}

rff_status rff_admm_get_profile(rff_admm_t h, rff_admm_profile* out) {
  if (!h || !out) return RFF_EINVAL;
  *out = h->prof;
  out->launches = h->launches;
  out->tc_kchunk = h->split_path() ? (h->tc_kc ? h->tc_kc : 64) : 0;
  out->nsplit = h->cached_z() ? h->nsplit_cz : h->nsplit;
  out->tc_z_tmem = h->split_path() ? h->tc_zt : 0;
  out->tc_cta_pair = h->split_path() && h->tc_cg == 2 ? 1 : 0;
  return RFF_OK;
}

void rff_admm_destroy(rff_admm_t h) {
  if (!h) return;
  if (h->st) cudaStreamSynchronize(h->st);
  delete h;
}

const char* rff_admm_last_error(rff_admm_t h) { return h ? h->err.c_str() : "null handle"; }

}  // extern "C"

namespace {
// X as given by the caller: dense row-major n x d, or CSR (indptr n + 1, indices and values nnz)
struct XInput {
  const float* dense = nullptr;
  const int64_t* indptr = nullptr;
  const int32_t* indices = nullptr;
  const float* values = nullptr;
  int64_t nnz = 0;
};

rff_status set_data_impl(rff_admm_t h, const XInput& xin, const float* Yin, int64_t n, int64_t d,
                         int is_device_ptr) {
  if (!h) return RFF_EINVAL;
  h->err.clear();
  const bool csr = xin.dense == nullptr;
  if ((!csr && !xin.dense) || (csr && (!xin.indptr || (xin.nnz > 0 && (!xin.indices || !xin.values)))) || !Yin)
    return h->fail(RFF_EINVAL, "X or Y is NULL");
  if (csr && xin.nnz < 0) return h->fail(RFF_EINVAL, "nnz < 0");
  if (n < h->p.R || d < 1 || n > ((int64_t)1 << 31) - 1) return h->fail(RFF_EINVAL, "need R <= n < 2^31 and d >= 1");
  if (h->p.feature_map == RFF_MAP_FASTFOOD && d > 4096) return h->fail(RFF_EINVAL, "the Fastfood map takes d <= 4096");
  if (h->tensorsketch() &&
      tensorsketch_smem_bytes(h->p.degree, d, (h->p.D + h->p.C - 1) / h->p.C) > TS_MAX_SMEM)
    return h->fail(RFF_EINVAL, "TensorSketch: degree x d and the block size exceed the kernel's shared memory");
  CK(cudaStreamSynchronize(h->st));
  h->drop_graph();
  h->free_all();
  CK(cudaStreamSynchronize(h->st));   // the freed blocks return to the device before it is measured
  h->has_data = h->factored = false;
  h->features_released = false;
  h->iters_done = 0;

  auto& s = *h;
  compute_geometry(s, n, d);

  // memory check before any allocation
  size_t fr = 0, tot = 0;
  CK(cudaMemGetInfo(&fr, &tot));
  const size_t need = working_set_bytes(s) + setup_bytes(s, 1);
  const size_t avail = s.mem_limit ? std::min(fr, s.mem_limit) : fr;
  if (need > avail) {
    return h->fail(RFF_ENOMEM, "working set " + std::to_string(need >> 20) + " MiB exceeds the " +
                                   std::to_string(avail >> 20) + " MiB available");
  }

  rff_status st = RFF_OK;
#define AL(ptr, cnt) \
  if ((st = dalloc(h, ptr, (size_t)(cnt))) != RFF_OK) { h->free_all(); return st; }
  AL(s.row_of_slot, s.nslots);
  AL(s.feat_of_slot, s.fslots);
  AL(s.slot_of_feat, s.D);
  AL(s.d_row_slot, s.R);
  AL(s.d_row_size, s.R);
  AL(s.d_col_slot, s.C);
  AL(s.d_col_size, s.C);
  AL(s.d_zero, 2);
  if (s.tensorsketch()) AL(s.ts_buf, (int64_t)TS_SCORE_ROWS * s.fslots);
  AL(s.bmask, (int64_t)s.R * s.C);
  AL(s.bctr, 1);
  if (s.split_path()) {
    AL(s.Xhi, s.nslots * s.dld);
    AL(s.Xlo, s.nslots * s.dld);
    AL(s.Ghi, s.fslots * s.dld);
    AL(s.Glo, s.fslots * s.dld);
    AL(s.VThi, (int64_t)s.C * s.mpad * s.nslots);
    AL(s.VTlo, (int64_t)s.C * s.mpad * s.nslots);
    AL(s.WThi, (int64_t)s.R * s.mpad * s.fslots);
    AL(s.WTlo, (int64_t)s.R * s.mpad * s.fslots);
    AL(s.WbThi, s.mpad * s.fslots);
    AL(s.WbTlo, s.mpad * s.fslots);
  }
  // FP32 copies of X and G: the SIMT path's operands, and on the cached-Z path the inputs
  // of its one-time FP32 materialisation of Z (round-to-nearest FMA chains for X.G)
  if (!s.split_path() || s.cached_z()) {
    AL(s.X32, s.nslots * s.dld);
    AL(s.Gt32, s.fslots * s.dld);
  }
  AL(s.bias, s.fslots);
  AL(s.Y, s.nslots * s.mpad);
  AL(s.O, s.nslots * s.mpad);
  AL(s.Obar, s.nslots * s.mpad);
  AL(s.nu, s.nslots * s.mpad);
  AL(s.nu_old, s.nslots * s.mpad);
  AL(s.Obar_old, s.nslots * s.mpad);
  AL(s.Op, (int64_t)s.C * s.nslots * s.mpad);
  if (!s.split_path() || s.outer) AL(s.V32, (int64_t)s.C * s.nslots * s.mpad);   // FP32 V (outer form: U_i)
  AL(s.amax, AMAX_WORDS);
  AL(s.W, s.fslots * s.mpad);
  AL(s.Wbar, s.fslots * s.mpad);
  AL(s.mu, s.fslots * s.mpad);
  AL(s.mu_old, s.fslots * s.mpad);
  AL(s.Wbar_old, s.fslots * s.mpad);
  AL(s.What, (int64_t)s.R * s.fslots * s.mpad);
  AL(s.muij, (int64_t)s.R * s.fslots * s.mpad);
  AL(s.muij_old, (int64_t)s.R * s.fslots * s.mpad);
  AL(s.Rpart, (int64_t)std::max(s.nsplit_max, s.nsplit_cz) * s.R * s.fslots * s.mpad);
  if (s.split_path() && !s.outer) {
    AL(s.Q1, s.q_rows * s.ldq);
    AL(s.Q2, s.q_rows * s.ldq);
    AL(s.Q3, s.q_rows * s.ldq);
    AL(s.rT1, (int64_t)s.R * s.mpad * s.fslots);
    AL(s.rT2, (int64_t)s.R * s.mpad * s.fslots);
    AL(s.rT3, (int64_t)s.R * s.mpad * s.fslots);
    {
      int64_t nq = 0;
      for (int64_t b = 0; b < (int64_t)s.R * s.C; ++b) nq += ceil_div(s.col_size[b % s.C], 128);
      s.nqjobs = (int)nq;
      AL(s.qjobs, nq);
    }
  }
  if (s.split_path()) {
    if (s.cached_z()) {
      AL(s.Zhi, s.nslots * s.fslots);
      AL(s.Zlo, s.nslots * s.fslots);
      AL(s.ZThi, s.nslots * s.fslots);
      AL(s.ZTlo, s.nslots * s.fslots);
      s.np2 = (int)(s.nslots / 128 * s.C);
      s.np1 = (int)(s.fslots / 128 * s.R * s.nsplit_cz);
      AL(s.p1jobs, s.np1);
      AL(s.p2jobs, s.np2);
    }
  }
  if (!s.split_path() || s.outer) {
    AL(s.rhs, (int64_t)s.R * s.fslots * s.mpad);
    AL(s.Q32, s.foff.back());
    AL(s.gdesc, s.R * s.C);
  }
  if (s.outer) AL(s.U32, 2 * (int64_t)s.C * s.nslots * s.mpad);   // Z c and V - Z c, then -P (V - Z c)
  AL(s.lam_dev, s.mpad);
  AL(s.partials, 1024);
  AL(s.flag, 4);
#undef AL

  // slot tables
  std::vector<int32_t> ros(s.nslots, -1), fos(s.fslots, -1), sof(s.D, 0);
  for (int i = 0; i < s.R; ++i)
    for (int64_t r = 0; r < s.row_size[i]; ++r) ros[s.row_slot[i] + r] = (int32_t)(s.row_start[i] + r);
  for (int j = 0; j < s.C; ++j)
    for (int64_t k = 0; k < s.col_size[j]; ++k) {
      fos[s.col_slot[j] + k] = (int32_t)(s.col_start[j] + k);
      sof[s.col_start[j] + k] = (int32_t)(s.col_slot[j] + k);
    }
  CK(cudaMemcpyAsync(s.row_of_slot, ros.data(), ros.size() * 4, cudaMemcpyHostToDevice, s.st));
  CK(cudaMemcpyAsync(s.feat_of_slot, fos.data(), fos.size() * 4, cudaMemcpyHostToDevice, s.st));
  CK(cudaMemcpyAsync(s.slot_of_feat, sof.data(), sof.size() * 4, cudaMemcpyHostToDevice, s.st));
  CK(cudaMemcpyAsync(s.d_row_slot, s.row_slot.data(), s.R * 8, cudaMemcpyHostToDevice, s.st));
  CK(cudaMemcpyAsync(s.d_row_size, s.row_size.data(), s.R * 8, cudaMemcpyHostToDevice, s.st));
  CK(cudaMemcpyAsync(s.d_col_slot, s.col_slot.data(), s.C * 8, cudaMemcpyHostToDevice, s.st));
  CK(cudaMemcpyAsync(s.d_col_size, s.col_size.data(), s.C * 8, cudaMemcpyHostToDevice, s.st));
  CK(cudaMemsetAsync(s.d_zero, 0, 16, s.st));
  {
    rff_status lr = upload_lambdas(h);
    if (lr != RFF_OK) { h->free_all(); return lr; }
  }

  // data: stage (device), validate, scatter into slots.  Dense X is staged as n x d; CSR X as
  // its three arrays (values first, so that the value checks run on one contiguous range)
  const int64_t xcount = csr ? xin.nnz : (int64_t)n * d;   // the staged X values
  const size_t xb = (size_t)xcount * 4, yb = (size_t)n * s.m * 4;
  const size_t csrb = csr ? round_up((n + 1) * 8, 256) + round_up(xin.nnz * 4, 256) : 0;
  const size_t slotb = (s.split_path() && !s.cached_z()) ? (size_t)s.nslots * s.dld * 4 : 0;
  if ((st = ensure_scratch(h, round_up(xcount, 64) * 4 + round_up((int64_t)n * s.m, 64) * 4 + csrb + slotb + 1024)) !=
      RFF_OK) {
    h->free_all();
    return st;
  }
  float* sx = static_cast<float*>(h->scratch.p);
  float* sy = sx + round_up(xcount, 64);
  char* cbase = reinterpret_cast<char*>(sy + round_up((int64_t)n * s.m, 64));
  int64_t* sindptr = reinterpret_cast<int64_t*>(cbase);
  int32_t* sindices = reinterpret_cast<int32_t*>(cbase + (csr ? round_up((n + 1) * 8, 256) : 0));
  const cudaMemcpyKind kind = is_device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (xb) CK(cudaMemcpyAsync(sx, csr ? xin.values : xin.dense, xb, kind, s.st));
  CK(cudaMemcpyAsync(sy, Yin, yb, kind, s.st));
  CK(cudaMemsetAsync(s.flag, 0, 16, s.st));
  if (csr) {
    CK(cudaMemcpyAsync(sindptr, xin.indptr, (n + 1) * 8, kind, s.st));
    if (xin.nnz) CK(cudaMemcpyAsync(sindices, xin.indices, xin.nnz * 4, kind, s.st));
    CK(launch_csr_check(sindptr, sindices, n, d, xin.nnz, s.flag + 3, s.st));
  }
  CK(launch_finite_check(sx, xcount, s.p.feature_map == RFF_MAP_LAPLACE ? 2 : 0, s.flag, s.st,
                         reinterpret_cast<unsigned*>(s.flag + 2)));
  const int pm1 = (s.p.loss == RFF_LOSS_HINGE || s.p.loss == RFF_LOSS_LOGISTIC) ? 1 : 0;
  CK(launch_finite_check(sy, (int64_t)n * s.m, pm1, s.flag + 1, s.st));
  int fl[4] = {0, 0, 0, 0};
  CK(cudaMemcpyAsync(fl, s.flag, 16, cudaMemcpyDeviceToHost, s.st));
  CK(cudaStreamSynchronize(s.st));
  if (fl[3]) { h->free_all(); return h->fail(RFF_EINVAL, "CSR X: indptr not non-decreasing from 0 to nnz, or a column index outside [0, d)"); }
  {
    float xmax = 0.f;
    memcpy(&xmax, &fl[2], 4);
    s.xscale = pow2_scale(std::max<double>(xmax, s.bias_col >= 0 ? 1.0 : 0.0));
    s.gscale = g_scale(s.p.sigma);
  }
  if (fl[0] & 1) { h->free_all(); return h->fail(RFF_EINVAL, "X contains NaN or Inf"); }
  if (fl[0] & 4) { h->free_all(); return h->fail(RFF_EINVAL, "the random Laplace map takes nonnegative X"); }
  if (fl[1] & 1) { h->free_all(); return h->fail(RFF_EINVAL, "Y contains NaN or Inf"); }
  if (fl[1] & 2) { h->free_all(); return h->fail(RFF_EINVAL, "hinge/logistic targets must be -1 or +1"); }

  float* Xs = s.X32;
  if (s.split_path() && !s.cached_z())   // the float32 slot copy lives in scratch only long enough to split it
    Xs = reinterpret_cast<float*>(cbase + round_up(csrb, 256));
  if (csr)
    CK(launch_scatter_csr(sindptr, sindices, sx, s.row_of_slot, s.nslots, Xs, s.dld, s.st));
  else
    CK(launch_gather_rows(sx, d, d, s.row_of_slot, s.nslots, Xs, s.dld, s.st));
  CK(launch_gather_rows(sy, s.m, s.m, s.row_of_slot, s.nslots, s.Y, s.mpad, s.st));
  if (s.bias_col >= 0) CK(launch_set_column(Xs, s.dld, s.nslots, s.bias_col, 1.f, s.st));
  if (s.split_path()) CK(launch_split_f16(Xs, s.nslots * s.dld, s.xscale, s.Xhi, s.Xlo, s.st));

  // ADMM state: all zero (Sec. 3: "initialize to zero"), then O = prox(Obar - nu) = prox(0)
  const size_t rowb = (size_t)s.nslots * s.mpad * 4, colb = (size_t)s.fslots * s.mpad * 4;
  for (float* b : {s.O, s.Obar, s.nu}) CK(cudaMemsetAsync(b, 0, rowb, s.st));
  if (s.V32) CK(cudaMemsetAsync(s.V32, 0, rowb * s.C, s.st));
  CK(cudaMemsetAsync(s.amax, 0, AMAX_WORDS * 4, s.st));
  CK(cudaMemsetAsync(s.Op, 0, rowb * s.C, s.st));
  for (float* b : {s.W, s.Wbar, s.mu}) CK(cudaMemsetAsync(b, 0, colb, s.st));
  for (float* b : {s.What, s.muij}) CK(cudaMemsetAsync(b, 0, colb * s.R, s.st));
  if (s.rhs) CK(cudaMemsetAsync(s.rhs, 0, colb * s.R, s.st));
  if (s.U32) CK(cudaMemsetAsync(s.U32, 0, rowb * s.C, s.st));
  CK(cudaMemsetAsync(s.Rpart, 0, colb * s.R * std::max(s.nsplit_max, s.nsplit_cz), s.st));
  if (s.split_path()) {
    CK(cudaMemsetAsync(s.VThi, 0, rowb / 2 * s.C, s.st));
    CK(cudaMemsetAsync(s.VTlo, 0, rowb / 2 * s.C, s.st));
    CK(cudaMemsetAsync(s.WThi, 0, colb / 2 * s.R, s.st));
    CK(cudaMemsetAsync(s.WTlo, 0, colb / 2 * s.R, s.st));
    for (__nv_bfloat16* b : {s.rT1, s.rT2, s.rT3})
      if (b) CK(cudaMemsetAsync(b, 0, colb / 2 * s.R, s.st));
  }
  CK(launch_prox_loss(s.p.loss, s.O, s.Y, s.nslots, (int)s.m, s.mpad, s.t_loss, s.p.newton_iters, s.O, s.st));
  // max |O| of the initial state (nu = 0, V = 0): the first exchange's bound of |V|
  if (s.split_path())
    CK(launch_finite_check(s.O, s.nslots * s.mpad, 0, reinterpret_cast<int*>(s.amax + AMAX_FLAG), s.st,
                           s.amax + AMAX_O));
  // zero O on padding rows (prox(0) with y = 0 is not zero for the squared loss only if y != 0; y = 0 there)
  CK(cudaStreamSynchronize(s.st));
  h->has_data = true;
  return RFF_OK;
}
}  // namespace

extern "C" {
rff_status rff_admm_set_data(rff_admm_t h, const float* X, const float* Yin, int64_t n, int64_t d,
                             int is_device_ptr) {
  XInput xin;
  xin.dense = X;
  if (!X) return h ? h->fail(RFF_EINVAL, "X or Y is NULL") : RFF_EINVAL;
  return set_data_impl(h, xin, Yin, n, d, is_device_ptr);
}

rff_status rff_admm_set_data_csr(rff_admm_t h, const int64_t* indptr, const int32_t* indices, const float* values,
                                 int64_t nnz, const float* Y, int64_t n, int64_t d, int is_device_ptr) {
  XInput xin;
  xin.indptr = indptr;
  xin.indices = indices;
  xin.values = values;
  xin.nnz = nnz;
  return set_data_impl(h, xin, Y, n, d, is_device_ptr);
}

}  // extern "C"

// ------------------------------------------------------------------ set-up
namespace {

// Tile-shape autotuner of the tensor-core passes: times pass 2 for each ring geometry
// (K chunk 64 or 32; Z tile in shared or tensor memory; the wide products) on the handle's
// own data, over the first 128-row tiles of the first row block (about two waves of work
// items; pass 1 runs the same X.G tiles and chained products and ranks the geometries the
// same way), and keeps the fastest.  All geometries issue the same products in the same order for every output
// element, so the choice changes speed, never results (a run is reproducible whatever
// the timing).  The passes only write their scratch outputs (R partials, O'), which
// every iteration recomputes.
rff_status autotune(rff_admm_t h) {
  NvtxRange range("rff set-up: autotune");
  auto& s = *h;
  if (!s.split_path() || s.cached_z()) return RFF_OK;
  // RFF_TC_GEOMETRY="kc,zt" or "kc,zt,cg" (kc 64 or 32; zt 0, 1, or 2 when m_pad <= 128;
  // cg 1, or 2 with zt 1 or 2) fixes the geometry instead
  if (const char* g = getenv("RFF_TC_GEOMETRY")) {
    int kc = 0, zt = -1, cg = 1;
    const int nf = sscanf(g, "%d,%d,%d", &kc, &zt, &cg);
    if (nf >= 2 && (kc == 64 || kc == 32) &&
        (zt == 0 || zt == 1 || (zt == 2 && s.mpad <= 128) || (zt == 3 && s.mpad <= 192)) &&
        (cg == 1 || (cg == 2 && (zt == 1 || zt == 2)))) {
      s.tc_kc = kc;
      s.tc_zt = zt;
      s.tc_cg = cg;
      return RFF_OK;
    }
    return h->fail(RFF_EINVAL,
                   "RFF_TC_GEOMETRY must be \"kc,zt\" or \"kc,zt,cg\" with kc 64 or 32, zt 0, 1, 2 (m_pad <= "
                   "128) or 3 (m_pad <= 192), cg 1 or 2 (2 needs zt 1 or 2)");
  }
  std::vector<int> splits{s.nsplit};   // pass 1's row splits are not timed: kept as chosen
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_kc = 64, best_ns = s.nsplit, best_zt = 0, best_cg = 1;
  bool warm = false;
  int nsm = 148, dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // (Z in smem), (Z in TMEM), the wide N = 256 geometry (m_pad <= 192), and with m_pad <= 128
  // the double-buffered acc1 beside Z in TMEM.  The CTA-pair geometries are selectable through
  // RFF_TC_GEOMETRY but not timed here: they measured 6-15 % slower on every workload tried
  std::vector<std::pair<int, int>> geos{{0, 1}, {1, 1}};   // (zt, cg)
  if (s.mpad <= 192) geos.push_back({3, 1});
  if (s.mpad <= 128) geos.push_back({2, 1});
  for (const auto& geo : geos)
  for (int kc : {64, 32}) {
    const int zt = geo.first, cg = geo.second;
    for (int ns : splits) {
      s.tc_kc = kc;
      s.tc_zt = zt;
      s.tc_cg = cg;
      s.nsplit = ns;
      float ms = 0.f;
      TcView tv = tc_view(s);
      tv.R = 1;
      tv.row_tiles = std::min<int64_t>(ceil_div(s.row_size[0], 128), std::max<int64_t>(16, ceil_div(2 * nsm, s.C)));
      for (int rep = warm ? 1 : 0; rep < 2; ++rep) {   // one untimed run warms caches and descriptors
        CK(cudaEventRecord(e0, s.st));
        CK(tc_pass2(tv, s.WThi, s.WTlo, s.mpad * s.fslots, s.Op, 1, s.amax + AMAX_W));
        CK(cudaEventRecord(e1, s.st));
        CK(cudaEventSynchronize(e1));
        CK(cudaEventElapsedTime(&ms, e0, e1));
      }
      warm = true;
      if (ms < best) {
        best = ms;
        best_kc = kc;
        best_ns = ns;
        best_zt = zt;
        best_cg = cg;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  s.tc_kc = best_kc;
  s.tc_zt = best_zt;
  s.tc_cg = best_cg;
  s.nsplit = best_ns;
  // the timing runs wrote O'_ij, which starts at zero: a block that sits out the first
  // iterations of a stochastic solve reads it as it is
  CK(cudaMemsetAsync(s.Op, 0, (size_t)s.C * s.nslots * s.mpad * sizeof(float), s.st));
  if (tc_error_word() != 0) return h->fail(RFF_ETIMEOUT, "a tensor-core pass gave up waiting during tuning");
  return RFF_OK;
}

// Cached-Z precision: Z (all row slots x all feature slots) and its transpose as scaled
// FP16 hi/lo pairs, computed once in FP32 on the SIMT pipes (X.G as round-to-nearest
// FMA chains: the tensor cores' accumulator rounds toward zero at every step, which
// for X.G costs accuracy that one-time work need not give up), staged in row chunks,
// and the job tables of the two streamed passes.
// TensorSketch over rows [r0, r0 + nr) of X (ld ldx, slot layout) for every column block of
// the handle; the caller sets the output (or the maximum) and the block range
TsArgs ts_args(const rff_admm_s& s, const float* X, int64_t ldx, const int32_t* row_ok, int64_t r0, int64_t nr) {
  TsArgs a{};
  a.X = X;
  a.ldx = ldx;
  a.d = (int)s.d;
  a.row_ok = row_ok;
  a.r0 = r0;
  a.nr = nr;
  a.q = s.p.degree;
  a.inv_sigma = (float)(1.0 / s.p.sigma);
  a.sqrt_c = (float)std::sqrt(s.p.coef0);
  a.k0 = (uint32_t)s.p.seed;
  a.k1 = (uint32_t)(s.p.seed >> 32);
  a.col_slot = s.d_col_slot;
  a.col_size = s.d_col_size;
  a.D = s.D;
  return a;
}

int64_t ts_block_max(const rff_admm_s& s) { return *std::max_element(s.col_size.begin(), s.col_size.end()); }

rff_status materialise_z(rff_admm_t h) {
  NvtxRange range("rff set-up: materialise Z");
  auto& s = *h;
  const int64_t chunk = materialise_chunk(s);
  rff_status rs = ensure_scratch(h, (size_t)chunk * s.fslots * 4);
  if (rs != RFF_OK) return rs;
  float* zc = static_cast<float*>(s.scratch.p);
  s.zscale = pow2_scale(s.zmap_scale());   // |Z| <= sqrt(2/D) (cos) or 1/sqrt(D) (exp(-T))
  for (int64_t r0 = 0; r0 < s.nslots; r0 += chunk) {
    const int64_t nr = std::min(chunk, s.nslots - r0);
    if (s.tensorsketch()) {
      TsArgs ta = ts_args(s, s.X32, s.dld, s.row_of_slot, r0, nr);
      ta.out = zc;
      ta.ldo = s.fslots;
      ta.out_elems = nr * s.fslots;
      ta.pad = 1;
      CK(launch_tensorsketch(ta, s.C, ts_block_max(s), s.st));
    } else {
      ZArgs za{s.X32, s.dld, s.Gt32, s.dld, (int)s.dld, s.bias, s.zmap_scale(), s.row_of_slot,
               s.feat_of_slot, r0, nr, 0, s.fslots, zc, s.fslots, s.p.feature_map};
      CK(launch_write_z_simt(za, s.st));
    }
    CK(launch_split_f16(zc, nr * s.fslots, s.zscale, s.Zhi + r0 * s.fslots, s.Zlo + r0 * s.fslots, s.st));
    CK(launch_transpose_split_f16(zc, nr, (int)s.fslots, 1, 0, s.ZThi + r0, s.ZTlo + r0, s.nslots, 0, s.zscale,
                                  nullptr, s.st));
  }
  // pass 2: one job per (128-row tile, column block j), K = the features of block j
  std::vector<SgJob> j2, j1;
  for (int64_t rt = 0; rt < s.nslots / 128; ++rt) {
    int i = 0;
    while (i + 1 < s.R && s.row_slot[i + 1] <= rt * 128) ++i;
    for (int j = 0; j < s.C; ++j) {
      SgJob jb{};
      jb.a_row = (int32_t)(rt * 128);
      jb.a_k0 = (int32_t)s.col_slot[j];
      jb.b_row = (int32_t)(i * s.mpad);
      jb.b_k0 = (int32_t)s.col_slot[j];
      jb.nk = (int32_t)ceil_div(s.col_size[j], 32);
      jb.blk = i * s.C + j;
      jb.out = ((int64_t)j * s.nslots + rt * 128) * s.mpad;
      j2.push_back(jb);
    }
  }
  // pass 1: one job per (128-feature tile, row block i, row split), K = the split's rows
  for (int sp = 0; sp < s.nsplit_cz; ++sp)
    for (int i = 0; i < s.R; ++i) {
      const int64_t nrt = ceil_div(s.row_size[i], 128);
      const int64_t t0 = sp * nrt / s.nsplit_cz, t1 = (sp + 1) * nrt / s.nsplit_cz;
      for (int64_t ft = 0; ft < s.fslots / 128; ++ft) {
        int j = 0;
        while (j + 1 < s.C && s.col_slot[j + 1] <= ft * 128) ++j;
        SgJob jb{};
        jb.a_row = (int32_t)(ft * 128);
        jb.a_k0 = (int32_t)(s.row_slot[i] + t0 * 128);
        jb.b_row = (int32_t)(s.incremental() ? 0 : j * s.mpad);   // the shared U_i, or V_ij
        jb.b_k0 = jb.a_k0;
        jb.nk = (int32_t)((t1 - t0) * 4);
        jb.blk = i * s.C + j;
        jb.out = (((int64_t)sp * s.R + i) * s.fslots + ft * 128) * s.mpad;
        j1.push_back(jb);
      }
    }
  if ((int)j1.size() != s.np1 || (int)j2.size() != s.np2) return h->fail(RFF_ECUDA, "internal: cached-Z job count");
  CK(cudaMemcpyAsync(s.p1jobs, j1.data(), j1.size() * sizeof(SgJob), cudaMemcpyHostToDevice, s.st));
  CK(cudaMemcpyAsync(s.p2jobs, j2.data(), j2.size() * sizeof(SgJob), cudaMemcpyHostToDevice, s.st));
  CK(cudaStreamSynchronize(s.st));
  return RFF_OK;
}

// Fastfood: V (the projection, in G's place) and b from Philox on the device; its split
// copies take their scale from the measured max |V| (V has no a-priori bound like
// Box-Muller's).  Tables and, on the split path, the FP32 V live in the set-up scratch.
rff_status fastfood_features(rff_admm_t h) {
  auto& s = *h;
  const size_t tb = round_up(fastfood_table_bytes(s.D, fastfood_dim(s.d)), 256);
  const bool keep32 = s.Gt32 != nullptr;
  const size_t vb = keep32 ? 0 : (size_t)s.fslots * s.dld * 4;
  rff_status rs = ensure_scratch(h, tb + vb + 256);
  if (rs != RFF_OK) return rs;
  char* base = static_cast<char*>(s.scratch.p);
  float* V = keep32 ? s.Gt32 : reinterpret_cast<float*>(base + tb);
  unsigned* maxbits = reinterpret_cast<unsigned*>(s.flag + 3);
  CK(cudaMemsetAsync(maxbits, 0, 4, s.st));
  CK(launch_fastfood_params(s.p.seed, s.p.sigma, s.d, s.dld, s.D, s.fslots, s.feat_of_slot, V, s.bias, maxbits, base,
                            s.st));
  if (s.tc_scores()) {
    unsigned bits = 0;
    CK(cudaMemcpyAsync(&bits, maxbits, 4, cudaMemcpyDeviceToHost, s.st));
    CK(cudaStreamSynchronize(s.st));
    float vmax = 0.f;
    memcpy(&vmax, &bits, 4);
    s.gscale = pow2_scale(std::max<double>(vmax, 3.1415927));   // b in [0, pi) shares the scale
    CK(launch_split_g_bias(V, s.fslots, s.dld, s.bias, s.bias_col, s.gscale, s.Ghi, s.Glo, s.st));
  }
  return RFF_OK;
}

// H (s x s FP64, ld s) += Z^T Z for one row chunk Z (nr x s FP32, ld s) on the tensor cores:
// Z^T split into scaled FP16 hi/lo (three products, the hi.hi ones in an accumulator of their
// own), 128 x 256 tiles of the lower triangle over 512-row pieces of K (32 accumulations of
// the dominant products per tile: the accumulator's round-toward-zero bias stays ~2e-6 of a
// piece's sum), the pieces' tiles added in FP64 in order.  buf: tc_gram_bytes(chunk, smax).
// With Zc null the chunk is regenerated straight into that split by the tensor-core write mode
// (rows zr0.., features zf0.. of the view zv), with the same roundings as splitting the FP32 Z;
// on the cached-Z precision (zv null too) it is copied from the stored split of Z^T.
rff_status tc_gram_accumulate(rff_admm_t h, const float* Zc, int64_t nr, int64_t sj, double* H, char* buf,
                              int64_t chunk_rows, int64_t smax, const TcView* zv = nullptr, int64_t zr0 = 0,
                              int64_t zf0 = 0) {
  auto& s = *h;
  const int64_t spad = round_up(smax, 256), kpad = round_up(chunk_rows, GRAM_KCH);
  std::vector<int2> tiles;
  const int64_t nt = tc_gram_tiles(sj, &tiles);
  // the split's scale: the stored Z's on the cached-Z precision, else that of |Z| <= sqrt(2/D)
  const float zs = s.cached_z() ? s.zscale : pow2_scale(std::sqrt(2.0 / (double)s.D));
  __half* hi = reinterpret_cast<__half*>(buf);
  __half* lo = reinterpret_cast<__half*>(buf + round_up((size_t)spad * kpad * 2, 256));
  float* P = reinterpret_cast<float*>(buf + 2 * round_up((size_t)spad * kpad * 2, 256));
  int2* dtiles = reinterpret_cast<int2*>(reinterpret_cast<char*>(P) + (size_t)GRAM_GROUP * tc_gram_tiles(smax) * 128 * 256 * 4);
  SgJob* djobs = reinterpret_cast<SgJob*>(reinterpret_cast<char*>(dtiles) + round_up((size_t)tc_gram_tiles(smax) * sizeof(int2), 256));
  const int64_t kn = round_up(nr, GRAM_KCH);   // this chunk's K, zero-padded
  CK(cudaMemsetAsync(hi, 0, (size_t)spad * kn * 2, s.st));
  CK(cudaMemsetAsync(lo, 0, (size_t)spad * kn * 2, s.st));
  if (Zc) {
    CK(launch_transpose_split_f16(Zc, nr, (int)sj, 1, 0, hi, lo, kn, 0, zs, nullptr, s.st));
  } else if (zv) {
    CK(tc_write_zt_split(*zv, zr0, nr, zf0, sj, zs, hi, lo, kn));
  } else {   // features zf0.. and rows zr0.. of the stored Z^T split (ld nslots)
    CK(cudaMemcpy2DAsync(hi, kn * 2, s.ZThi + zf0 * s.nslots + zr0, s.nslots * 2, nr * 2, sj,
                         cudaMemcpyDeviceToDevice, s.st));
    CK(cudaMemcpy2DAsync(lo, kn * 2, s.ZTlo + zf0 * s.nslots + zr0, s.nslots * 2, nr * 2, sj,
                         cudaMemcpyDeviceToDevice, s.st));
  }
  CK(cudaMemcpyAsync(dtiles, tiles.data(), nt * sizeof(int2), cudaMemcpyHostToDevice, s.st));
  const int64_t npieces = kn / GRAM_KCH;
  // every group's job table in one copy: stream order alone keeps P and the tables of one
  // group from being overwritten before its reduction has read them
  std::vector<SgJob> jobs;
  jobs.reserve((size_t)npieces * nt);
  for (int64_t k = 0; k < npieces; ++k)
    for (int64_t t = 0; t < nt; ++t) {
      SgJob jb{};
      jb.a_row = tiles[t].x;
      jb.a_k0 = (int32_t)(k * GRAM_KCH);
      jb.b_row = tiles[t].y;
      jb.b_k0 = jb.a_k0;
      jb.nk = GRAM_KCH / 32;
      jb.blk = 0;
      jb.out = ((k % GRAM_GROUP) * nt + t) * 128 * 256;
      jobs.push_back(jb);
    }
  // the host vector is read by the copy: pageable memory is staged before the call returns
  CK(cudaMemcpyAsync(djobs, jobs.data(), jobs.size() * sizeof(SgJob), cudaMemcpyHostToDevice, s.st));
  for (int64_t g0 = 0; g0 < npieces; g0 += GRAM_GROUP) {
    const int64_t g1 = std::min<int64_t>(npieces, g0 + GRAM_GROUP);
    SgView v{};
    v.A[0] = hi;
    v.A[1] = lo;
    v.a_rows = spad;
    v.a_cols = kn;
    v.B[0] = hi;
    v.B[1] = lo;
    v.b_rows = spad;
    v.b_cols = kn;
    v.na = v.nb = 2;
    v.f16 = 1;
    v.jobs = djobs + g0 * nt;
    v.njobs = (int)((g1 - g0) * nt);
    v.mpad = 256;
    v.out = P;
    v.out_elems = (int64_t)GRAM_GROUP * tc_gram_tiles(smax) * 128 * 256;
    v.out_scale = 1.f / (zs * zs);
    v.two_acc = 1;
    v.persistent = 1;
    v.kc = 64;   // K = kn, a multiple of 512
    v.st = s.st;
    CK(split_gemm(v));
    CK(launch_gram_reduce(P, (int)(g1 - g0), (int)nt, dtiles, sj, H, sj, s.st));
  }
  return RFF_OK;
}

// Random features: G and b (or the Laplace map's W, or the Fastfood V) from Philox (Sec. 4),
// into the handle's copies: FP32 where SIMT kernels read them, the FP16 split where the
// tensor cores form X.G
rff_status generate_features(rff_admm_t h) {
  auto& s = *h;
  if (s.p.feature_map == RFF_MAP_FASTFOOD) return fastfood_features(h);
  const bool g16 = s.tc_scores();
  CK(launch_params_slots(s.p.seed, s.p.sigma, s.d, s.dld, s.fslots, s.feat_of_slot, s.Gt32, g16 ? s.Ghi : nullptr,
                         g16 ? s.Glo : nullptr, s.gscale, s.bias, s.bias_col, s.st, s.p.feature_map));
  return RFF_OK;
}

void free_buf(rff_admm_t h, void* p) {
  for (size_t i = 0; i < h->bufs.size(); ++i)
    if (h->bufs[i].p == p) {
      cudaFreeAsync(p, h->st);
      h->bufs.erase(h->bufs.begin() + (long)i);
      return;
    }
}

// Give back the feature parameters' copies (the paper keeps omega implicit as the state of
// the generator, Sec. 4); *bytes receives what was freed
rff_status release_features(rff_admm_t h, size_t* bytes) {
  auto& s = *h;
  size_t freed = 0;
  if (!s.features_released) {
    for (void* p : {(void*)s.Gt32, (void*)s.Ghi, (void*)s.Glo})
      if (p) {
        for (auto& b : s.bufs)
          if (b.p == p) freed += b.bytes;
        free_buf(h, p);
      }
    s.Gt32 = nullptr;
    s.Ghi = s.Glo = nullptr;
    s.features_released = true;
    s.drop_graph();   // a captured iteration holds the old addresses
  }
  if (bytes) *bytes = freed;
  return RFF_OK;
}

// Bring them back: allocate and draw again (bit-identical to the first draw)
rff_status regenerate_features(rff_admm_t h) {
  auto& s = *h;
  if (!s.features_released) return RFF_OK;
  rff_status st = RFF_OK;
  if (s.split_path()) {
    if ((st = dalloc(h, s.Ghi, (size_t)(s.fslots * s.dld))) != RFF_OK) return st;
    if ((st = dalloc(h, s.Glo, (size_t)(s.fslots * s.dld))) != RFF_OK) return st;
  }
  if (!s.split_path() || s.cached_z())
    if ((st = dalloc(h, s.Gt32, (size_t)(s.fslots * s.dld))) != RFF_OK) return st;
  s.features_released = false;
  s.drop_graph();
  return generate_features(h);
}

rff_status setup_factors(rff_admm_t h) {
  NvtxRange range("rff set-up: features, Gram, factors");
  auto& s = *h;
  {
    rff_status r = generate_features(h);
    if (r != RFF_OK) return r;
  }
  if (s.tensorsketch()) {
    // the sketches have no a-priori bound: one pass over the training rows measures max |z|,
    // the scale of Z's FP16 split (and of the Gram's)
    unsigned* bits = reinterpret_cast<unsigned*>(s.flag + 3);
    CK(cudaMemsetAsync(bits, 0, 4, s.st));
    TsArgs ta = ts_args(s, s.X32, s.dld, s.row_of_slot, 0, s.nslots);
    ta.amax = bits;
    CK(launch_tensorsketch(ta, s.C, ts_block_max(s), s.st));
    unsigned hb = 0;
    CK(cudaMemcpyAsync(&hb, bits, 4, cudaMemcpyDeviceToHost, s.st));
    CK(cudaStreamSynchronize(s.st));
    memcpy(&s.ts_zmax, &hb, 4);
  }
  const float scale = s.zmap_scale();
  // Gram matrices H_ij = I + Z_ij^T Z_ij (eq. (cache)), or I + Z_ij Z_ij^T in the outer
  // form, in FP64, batched by memory
  int64_t smax = 0;
  for (int j = 0; j < s.C; ++j) smax = std::max(smax, s.col_size[j]);
  const int64_t nmax = *std::max_element(s.row_size.begin(), s.row_size.end());
  const int64_t fmax = s.outer ? nmax : smax;          // factor dimension
  const int64_t nblocks = (int64_t)s.R * s.C;
  size_t fr = 0, tot = 0;
  CK(cudaMemGetInfo(&fr, &tot));
  const size_t per_block = (size_t)fmax * fmax * 8 * 2;
  const int64_t chunk_rows = std::min<int64_t>(32768, round_up(nmax, SLOT));
  // outer form: Z_ij in chunks of feature columns, each transposed for the Gram kernel
  const int64_t chunk_feat = std::min<int64_t>(2048, round_up(smax, SLOT));
  const size_t zbytes = (s.outer ? (size_t)nmax * chunk_feat * 4 * 2 : (size_t)chunk_rows * smax * 4) +
                        (tc_gram(s) ? tc_gram_bytes(chunk_rows, smax) : 0);
  size_t budget = (size_t)(fr * 0.6);
  if (s.mem_limit) {
    const size_t ws = working_set_bytes(s);
    budget = std::min(budget, s.mem_limit > ws ? s.mem_limit - ws : (size_t)0);
  }
  budget = budget > zbytes + (256u << 20) ? budget - zbytes - (256u << 20) : 0;
  int64_t batch = std::max<int64_t>(1, std::min<int64_t>(nblocks, (int64_t)(budget / std::max<size_t>(per_block + factor_scratch_bytes(1, (int)fmax), 1))));
  size_t need = (size_t)batch * per_block + zbytes + factor_scratch_bytes((int)batch, (int)fmax) + (size_t)batch * 4 + 4096;
  if (s.cached_z()) need = std::max(need, (size_t)materialise_chunk(s) * s.fslots * 4);
  rff_status rs = ensure_scratch(h, need);
  if (rs != RFF_OK) return rs;
  if (s.cached_z()) {   // Z and Z^T's splits first: the Gram below reads the stored Z^T
    rff_status zr = materialise_z(h);
    if (zr != RFF_OK) return zr;
  }
  char* base = static_cast<char*>(s.scratch.p);
  double* H64 = reinterpret_cast<double*>(base);
  double* Q64 = H64 + batch * fmax * fmax;
  float* Zc = reinterpret_cast<float*>(Q64 + batch * fmax * fmax);
  float* Zt = Zc + (s.outer ? nmax * chunk_feat : 0);   // transposed chunk (outer form)
  // tensor-core Gram buffers after the row chunk, on a 256-byte boundary (tc_gram_bytes keeps 1 KB of slack)
  char* gbase = reinterpret_cast<char*>(
      round_up((uintptr_t)(reinterpret_cast<char*>(Zc) + (size_t)chunk_rows * smax * 4), (uintptr_t)256));
  int32_t* info = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(Zc) + zbytes);
  void* fscr = reinterpret_cast<char*>(info) + round_up(batch * 4, 256);

  if (s.split_path() && !s.outer)   // padding rows and columns of the split inverses stay zero
    for (__nv_bfloat16* q : {s.Q1, s.Q2, s.Q3}) CK(cudaMemsetAsync(q, 0, (size_t)s.q_rows * s.ldq * 2, s.st));
  for (int64_t b0 = 0; b0 < nblocks; b0 += batch) {
    const int64_t nb = std::min(batch, nblocks - b0);
    std::vector<MatJob> jobs;
    CK(cudaMemsetAsync(info, 0, nb * 4, s.st));
    for (int64_t bb = 0; bb < nb; ++bb) {
      const int64_t blk = b0 + bb;
      const int i = (int)(blk / s.C), j = (int)(blk % s.C);
      const int64_t sj = s.col_size[j], ni = s.row_size[i];
      const int64_t fd = s.outer ? ni : sj;
      double* Hb = H64 + bb * fmax * fmax;
      double* Qb = Q64 + bb * fmax * fmax;
      CK(cudaMemsetAsync(Hb, 0, fd * fd * 8, s.st));
      // outer form: H = I + Z Z^T accumulated over feature chunks (the rows of Z^T)
      for (int64_t f0 = 0; s.outer && f0 < sj; f0 += chunk_feat) {
        const int64_t nf = std::min(chunk_feat, sj - f0);
        if (s.split_path()) {
          CK(tc_write_z(tc_view(s), s.row_slot[i], ni, s.col_slot[j] + f0, nf, Zc, nf));
        } else {
          ZArgs za{s.X32, s.dld, s.Gt32, s.dld, (int)s.dld, s.bias, scale, s.row_of_slot, s.feat_of_slot,
                   s.row_slot[i], ni, s.col_slot[j] + f0, nf, Zc, nf, s.p.feature_map};
          CK(launch_write_z_simt(za, s.st));
        }
        CK(launch_transpose_f32(Zc, ni, nf, Zt, ni, s.st));
        CK(launch_gram_f32_to_f64(Zt, ni, nf, ni, Hb, ni, s.st));
      }
      for (int64_t r = 0; !s.outer && r < s.row_size[i]; r += chunk_rows) {
        const int64_t nr = std::min(chunk_rows, s.row_size[i] - r);
        if (s.split_path() && getenv("RFF_DIAG_SIMT_GRAM")) {
          CK(tc_write_z(tc_view(s), s.row_slot[i] + r, nr, s.col_slot[j], sj, Zc, sj));
          CK(launch_gram_f32_to_f64(Zc, sj, nr, sj, Hb, sj, s.st));
          continue;
        }
        if (tc_gram(s)) {   // Z^T's split written by the regeneration itself, or the stored one
          const TcView zv = tc_view(s);
          rff_status gr = tc_gram_accumulate(h, nullptr, nr, sj, Hb, gbase, chunk_rows, smax,
                                             s.cached_z() ? nullptr : &zv, s.row_slot[i] + r, s.col_slot[j]);
          if (gr != RFF_OK) return gr;
          continue;
        }
        // FP32 precision: Z on the SIMT pipes, its Gram from FP32 products with float-float sums
        ZArgs za{s.X32, s.dld, s.Gt32, s.dld, (int)s.dld, s.bias, scale, s.row_of_slot, s.feat_of_slot,
                 s.row_slot[i] + r, nr, s.col_slot[j], sj, Zc, sj, s.p.feature_map};
        CK(launch_write_z_simt(za, s.st));
        CK(launch_gram_f32_to_f64(Zc, sj, nr, sj, Hb, sj, s.st));
      }
      CK(launch_add_identity_and_mirror(Hb, fd, fd, s.st));
      CK(cudaMemsetAsync(Qb, 0, fd * fd * 8, s.st));
      CK(launch_set_diag(Qb, fd, fd, 1.0, s.st));
      jobs.push_back(MatJob{Hb, fd, (int)fd, Qb, fd, info + bb});
    }
    // Q is stored to 24 bits (FP32, or three BF16 pieces): updates that keep 40 bits of every
    // operand leave it within cond(H) 2^-40 (about 2e-9 at cond 2.3e3), far inside that
    CK(factor_and_invert_f64(jobs, true, fscr, s.st, true, 40));
    for (int64_t bb = 0; bb < nb; ++bb) {
      const int64_t blk = b0 + bb;
      const int64_t fd = s.outer ? s.row_size[blk / s.C] : s.col_size[blk % s.C];
      if (s.split_path() && !s.outer)
        CK(launch_split3_q(Q64 + bb * fmax * fmax, (int)fd, s.ldq, s.qrow[blk], s.Q1, s.Q2, s.Q3, s.st));
      else
        CK(launch_convert_f64_f32(Q64 + bb * fmax * fmax, s.Q32 + s.foff[blk], fd * fd, s.st));
    }
    std::vector<int32_t> hinfo(nb);
    CK(cudaMemcpyAsync(hinfo.data(), info, nb * 4, cudaMemcpyDeviceToHost, s.st));
    CK(cudaStreamSynchronize(s.st));
    for (int64_t bb = 0; bb < nb; ++bb)
      if (hinfo[bb] != 0)
        return h->fail(RFF_ENUMERIC, "Gram matrix of block " + std::to_string(b0 + bb) +
                                         " not positive definite at column " + std::to_string(hinfo[bb] - 1));
  }
  // iteration GEMM descriptors: x = Q rhs
  std::vector<GemmDesc> g(nblocks);
  std::vector<SgJob> qj;
  for (int i = 0; i < s.R; ++i)
    for (int j = 0; j < s.C; ++j) {
      const int64_t blk = (int64_t)i * s.C + j, sj = s.col_size[j];
      const int64_t off = ((int64_t)i * s.fslots + s.col_slot[j]) * s.mpad;
      if (s.outer) {
        // O'_ij = (I + Z_ij Z_ij^T)^-1 u_ij, rows of block i in column block j
        const int64_t ni = s.row_size[i], roff = ((int64_t)j * s.nslots + s.row_slot[i]) * s.mpad;
        float* yb = s.U32 + (int64_t)s.C * s.nslots * s.mpad;   // y_ij = -P_ij e_ij (alpha = -1)
        g[blk] = GemmDesc{s.Q32 + s.foff[blk], s.U32 + roff, nullptr, yb + roff, (int)ni, (int)s.mpad, (int)ni, ni,
                          s.mpad, 0, s.mpad};
      } else if (s.split_path()) {
        // one job per 128-row tile of Q_ij: rows of W'_ij, all m_pad columns, K = s_j
        for (int64_t m0 = 0; m0 < sj; m0 += 128) {
          SgJob jb{};
          jb.a_row = (int32_t)(s.qrow[blk] + m0);
          jb.a_k0 = 0;
          jb.b_row = (int32_t)(i * s.mpad);
          jb.b_k0 = (int32_t)s.col_slot[j];
          jb.nk = (int32_t)ceil_div(sj, 32);
          jb.blk = (int32_t)blk;
          jb.out = ((int64_t)i * s.fslots + s.col_slot[j] + m0) * s.mpad;
          qj.push_back(jb);
        }
      } else {
        float* Qb = s.Q32 + s.foff[blk];   // W'_ij += Q_ij rhs_ij (the incremental projection)
        g[blk] = GemmDesc{Qb, s.rhs + off, s.What + off, s.What + off, (int)sj, (int)s.mpad, (int)sj, sj, s.mpad,
                          s.mpad, s.mpad};
      }
    }
  if (s.split_path() && !s.outer) {
    if ((int)qj.size() != s.nqjobs) return h->fail(RFF_ECUDA, "internal: projection job count");
    CK(cudaMemcpyAsync(s.qjobs, qj.data(), qj.size() * sizeof(SgJob), cudaMemcpyHostToDevice, s.st));
  } else
    CK(cudaMemcpyAsync(s.gdesc, g.data(), g.size() * sizeof(GemmDesc), cudaMemcpyHostToDevice, s.st));
  CK(cudaStreamSynchronize(s.st));
  // the set-up scratch (FP64 Gram and inverse batches) is released
  CK(cudaFreeAsync(s.scratch.p, s.st));
  s.scratch = DevBuf{};
  s.factored = true;
  return autotune(h);
}

// ------------------------------------------------------------------ iteration
PassArgs base_pass_args(const rff_admm_s& s) {
  PassArgs a{};
  a.X = s.X32;
  a.ldx = s.dld;
  a.Gt = s.Gt32;
  a.ldg = s.dld;
  a.K = (int)s.dld;
  a.bias = s.bias;
  a.scale = s.zmap_scale();
  a.map = s.p.feature_map;
  a.row_ok = s.row_of_slot;
  a.feat_ok = s.feat_of_slot;
  a.row_slot = s.d_row_slot;
  a.row_size = s.d_row_size;
  a.R = s.R;
  a.col_slot = s.d_col_slot;
  a.col_size = s.d_col_size;
  a.C = s.C;
  a.mpad = (int)s.mpad;
  a.nsplit = s.nsplit;
  a.x_rows = s.nslots;
  a.g_rows = s.fslots;
  return a;
}

// W'_ij = Q_ij rhs_ij for all blocks: Q and rhs split three ways into BF16 (six
// products); W' is written row-major and max |W'| reduced for its FP16 split
SgView qgemm_view(const rff_admm_s& s) {
  SgView v{};
  v.A[0] = s.Q1;
  v.A[1] = s.Q2;
  v.A[2] = s.Q3;
  v.a_rows = s.q_rows;
  v.a_cols = s.ldq;
  v.B[0] = s.rT1;
  v.B[1] = s.rT2;
  v.B[2] = s.rT3;
  v.b_rows = (int64_t)s.R * s.mpad;
  v.b_cols = s.fslots;
  v.na = v.nb = 3;
  v.jobs = s.qjobs;
  v.njobs = s.nqjobs;
  v.mpad = (int)s.mpad;
  v.out = s.What;
  v.out_elems = (int64_t)s.R * s.fslots * s.mpad;
  v.out_scale = 1.f;
  v.amax = s.amax + AMAX_W;
  v.two_acc = 1;
  v.bmask = s.act();
  v.accumulate = 1;   // W'_ij += Q_ij rhs_ij (the incremental projection)
  v.kc = 64;          // the split inverses are zero past s_j columns
  v.st = s.st;        // one job per CTA: the hardware hands the 3.4 waves of jobs to whichever SM is free
  return v;
}

// cached-Z pass 1: R partials [split][i][feature slot][c] = sum over the split's rows of
// block i of Z^T[f][r] V_ij[r][c]  (A = Z^T hi/lo, B = V^T hi/lo of block j)
SgView cz_pass1_view(const rff_admm_s& s) {
  SgView v{};
  v.A[0] = s.ZThi;
  v.A[1] = s.ZTlo;
  v.a_rows = s.fslots;
  v.a_cols = s.nslots;
  v.B[0] = s.VThi;
  v.B[1] = s.VTlo;
  v.b_rows = (int64_t)s.C * s.mpad;
  v.b_cols = s.nslots;
  v.na = v.nb = 2;
  v.f16 = 1;
  v.jobs = s.p1jobs;
  v.njobs = s.np1;
  v.mpad = (int)s.mpad;
  v.out = s.Rpart;
  v.out_elems = s.rpart_elems();
  v.out_scale = 1.f / s.zscale;
  v.b_amax = s.amax;
  v.smem_budget = 110 * 1024;   // two CTAs per SM: one's epilogue overlaps the other's stream
  v.bmask = s.act();
  v.st = s.st;
  return v;
}

// cached-Z pass 2: O'_ij[r][c] = sum over features of block j of Z[r][f] W'_ij[f][c]
SgView cz_pass2_view(const rff_admm_s& s) {
  SgView v{};
  v.A[0] = s.Zhi;
  v.A[1] = s.Zlo;
  v.a_rows = s.nslots;
  v.a_cols = s.fslots;
  v.B[0] = s.WThi;
  v.B[1] = s.WTlo;
  v.b_rows = (int64_t)s.R * s.mpad;
  v.b_cols = s.fslots;
  v.na = v.nb = 2;
  v.f16 = 1;
  v.jobs = s.p2jobs;
  v.njobs = s.np2;
  v.mpad = (int)s.mpad;
  v.out = s.Op;
  v.out_elems = (int64_t)s.C * s.nslots * s.mpad;
  v.out_scale = 1.f / s.zscale;
  v.b_amax = s.amax + AMAX_W;
  v.amax = s.amax + AMAX_OP;
  v.smem_budget = 110 * 1024;
  v.bmask = s.act();
  v.st = s.st;
  return v;
}

// kernel launches of one iteration (the count a captured iteration replays)
int iter_launches(const rff_admm_s& s) {
  int n = s.outer ? (s.split_path() ? 14 : 10) : (s.split_path() ? 8 : 7);
  if (s.stochastic()) n += 1 + (s.split_path() && !s.outer ? 1 : 0);   // the mask; max |O'| of all blocks
  return n;
}

// the tensor-core view of an iteration's passes: the block mask of a stochastic iteration
TcView iter_view(const rff_admm_s& s) {
  TcView v = tc_view(s);
  v.bmask = s.act();
  return v;
}

// phase boundaries of one iteration; with profiling on, events k*7 .. k*7+6
rff_status mark(rff_admm_t h, int k, int phase) {
  if (!h->profiling) return RFF_OK;
  CK(cudaEventRecord(h->ev[(size_t)k * 7 + phase], h->st));
  return RFF_OK;
}

// The row exchange, the next loss prox, V_ij and (tensor-core path) its FP16 split, then
// the averaging and dual updates: the end of every iteration (phases 4..6).
rff_status exchange_and_average(rff_admm_t h, int k) {
  auto& s = *h;
  const int64_t nfe = s.fslots * s.mpad;
  rff_status r;
  RowEpiArgs e{s.Op, s.O, s.Obar, s.nu, s.Y, s.V32, nullptr, nullptr, nullptr, s.row_of_slot, s.nslots,
               s.C, (int)s.m, (int)s.mpad, s.p.loss, s.p.newton_iters, s.t_loss};
  const bool vsplit = s.split_path() && !s.outer;   // the outer form reads U_i in FP32
  if (vsplit) {
    // U^T as a scaled FP16 pair straight from the exchange (scale from the bound of |U|)
    e.V32 = nullptr;
    e.VThi = s.VThi;
    e.VTlo = s.VTlo;
    e.amax = s.amax;
    CK(cudaMemsetAsync(s.amax + AMAX_V, 0, 4, s.st));
    CK(cudaMemsetAsync(s.amax + AMAX_O_NEXT, 0, 8, s.st));
  }
  CK(launch_row_epilogue(e, s.st));
  if (vsplit)   // the outputs' maxima become the next exchange's inputs
    CK(cudaMemcpyAsync(s.amax + AMAX_O, s.amax + AMAX_O_NEXT, 8, cudaMemcpyDeviceToDevice, s.st));
  if ((r = mark(h, k, 5)) != RFF_OK) return r;
  CK(launch_avg_dual(s.W, s.What, s.R, nfe, s.Wbar, s.mu, s.muij, s.st));
  return mark(h, k, 6);
}

// One iteration with the outer form of the graph projection (every block has fewer rows
// than features): with c_ij = Wbar_j - mu'_ij, V_ij = Obar_ij + nu_i = O'_ij + U_i and
// P_ij = (I + Z_ij Z_ij^T)^-1 (n_i x n_i), eq. (gpWij) and (gpOij) read
//   W'_ij = (I + Z^T Z)^-1 (c + Z^T V) = c + Z^T P (V - Z c),   O'_ij = Z W'_ij = V - P (V - Z c)
// ((I + Z^T Z)^-1 Z^T = Z^T P and Z Z^T P = I - P): two regenerations of Z_ij per iteration
// (Z c and Z^T y), and no cancellation between two terms of the size of c.  In order:
// c; u = Z c (pass 2); e = V - u; y = -P e (GEMM); W' = c - Z^T y (pass 1); O' += U + y.
// Phases: ms_project covers c, Z c, P and Z^T y; ms_pass2 is empty.
rff_status iterate_outer(rff_admm_t h, int k) {
  auto& s = *h;
  const int64_t nfe = s.fslots * s.mpad;
  const int64_t nmax = *std::max_element(s.row_size.begin(), s.row_size.end());
  const int64_t nop = (int64_t)s.C * s.nslots * s.mpad;
  float* y = s.U32 + nop;
  int* scratch_flag = reinterpret_cast<int*>(s.amax + AMAX_FLAG);
  rff_status r;
  if ((r = mark(h, k, 0)) != RFF_OK) return r;
  if (s.stochastic()) CK(launch_block_mask(s.p.seed, s.bthr, s.R * s.C, s.bctr, s.bmask, s.st));
  CK(launch_prox_reg(s.p.reg, s.Wbar, s.mu, nfe, s.t_reg, s.W, s.st, s.lam_dev, (int)s.mpad));
  if ((r = mark(h, k, 1)) != RFF_OK) return r;
  if ((r = mark(h, k, 2)) != RFF_OK) return r;
  // c_ij, then u_ij = Z_ij c_ij into U32 (inactive blocks of a stochastic iteration are
  // skipped by every per-block kernel below and keep their W'_ij and O'_ij)
  CK(launch_rhs(s.Wbar, s.muij, s.Rpart, 0, s.R, nfe, s.rhs, s.st, s.feat_of_slot, (int)s.mpad));
  if (s.split_path()) {
    CK(cudaMemsetAsync(s.amax + AMAX_W, 0, 4, s.st));
    CK(launch_finite_check(s.rhs, s.R * nfe, 0, scratch_flag, s.st, s.amax + AMAX_W));
    CK(launch_transpose_split_f16(s.rhs, s.fslots, (int)s.mpad, s.R, nfe, s.WThi, s.WTlo, s.fslots,
                                  s.mpad * s.fslots, 1.f, s.amax + AMAX_W, s.st));
    CK(tc_pass2(iter_view(s), s.WThi, s.WTlo, s.mpad * s.fslots, s.U32, 1, s.amax + AMAX_W));
  } else {
    PassArgs b = base_pass_args(s);
    b.bmask = s.act();
    b.M = s.rhs;
    b.m_block_stride = nfe;
    b.m_elems = (int64_t)s.R * nfe;
    b.out = s.U32;
    b.out_block_stride = s.nslots * s.mpad;
    b.out_elems = nop;
    b.per_block = 1;
    CK(launch_pass2_simt(b, s.nslots, s.st));
  }
  // e_ij = V_ij - u_ij (in place), y_ij = -P_ij e_ij
  CK(launch_outer_residual(s.U32, s.Op, s.V32, s.nslots, (int)s.mpad, s.C, s.st));
  CK(launch_gemm_f32_nn(s.gdesc, s.R * s.C, (int)nmax, (int)s.mpad, -1.f, 0.f, s.st, s.act()));
  // W'_ij = c_ij - Z_ij^T y_ij (operand per block)
  PassArgs a = base_pass_args(s);
  a.bmask = s.act();
  if (s.split_path()) {
    // y^T as a scaled FP16 pair in the V^T buffers
    CK(cudaMemsetAsync(s.amax + AMAX_OINC, 0, 4, s.st));
    CK(launch_finite_check(y, nop, 0, scratch_flag, s.st, s.amax + AMAX_OINC));
    CK(launch_transpose_split_f16(y, s.nslots, (int)s.mpad, s.C, s.nslots * s.mpad, s.VThi, s.VTlo, s.nslots,
                                  s.mpad * s.nslots, 1.f, s.amax + AMAX_OINC, s.st));
    TcView vo = iter_view(s);
    vo.v_amax = s.amax + AMAX_OINC;
    CK(tc_pass1(vo, s.Rpart));
  } else {
    a.M = y;
    a.m_block_stride = s.nslots * s.mpad;
    a.m_elems = nop;
    a.out = s.Rpart;
    a.out_block_stride = nfe;
    a.out_elems = s.rpart_elems();
    CK(launch_pass1_simt(a, s.fslots, s.st));
  }
  CK(launch_sub_partials(s.rhs, s.Rpart, s.nsplit, s.R, nfe, s.feat_of_slot, (int)s.mpad, s.What, s.st, s.act(),
                         s.d_col_slot, s.C));
  // O'_ij = V_ij - P_ij e_ij = O'_ij + U_i + y_ij
  CK(launch_outer_update(s.Op, s.V32, y, s.nslots, (int)s.mpad, s.R, s.C, s.d_row_slot, s.act(), s.st));
  if ((r = mark(h, k, 3)) != RFF_OK) return r;
  if ((r = mark(h, k, 4)) != RFF_OK) return r;
  if ((r = exchange_and_average(h, k)) != RFF_OK) return r;
  s.launches += iter_launches(s);
  return RFF_OK;
}

// One iteration in phases: before pass 1 (mask, regulariser prox), pass 1, the projection,
// pass 2 and after it (exchange, averaging, duals).  iterate() runs them in order; a sweep
// may run the passes of several solves as one launch between the solves' other phases.
rff_status phase_pre(rff_admm_t h, int k) {
  auto& s = *h;
  const int64_t nfe = s.fslots * s.mpad;
  rff_status r;
  if ((r = mark(h, k, 0)) != RFF_OK) return r;
  // stochastic variant: this iteration's active blocks; the per-block kernels below skip the
  // others, which keep W'_ij and O'_ij (every dual still updates)
  if (s.stochastic()) CK(launch_block_mask(s.p.seed, s.bthr, s.R * s.C, s.bctr, s.bmask, s.st));
  // W_j <- prox_{(n lam / rho) r}(Wbar_j - mu_j)
  CK(launch_prox_reg(s.p.reg, s.Wbar, s.mu, nfe, s.t_reg, s.W, s.st, s.lam_dev, (int)s.mpad));
  return mark(h, k, 1);
}

// pass 1: R_ij = Z_ij^T U_i with U_i = Delta_i/(C+1) + nu_i = Obar_ij + nu_i - O'_ij, one
// operand for every column block (the incremental projection below)
rff_status phase_pass1(rff_admm_t h) {
  auto& s = *h;
  PassArgs a = base_pass_args(s);
  a.bmask = s.act();
  if (s.cached_z()) {
    CK(split_gemm(cz_pass1_view(s)));
  } else if (s.split_path()) {
    CK(tc_pass1(iter_view(s), s.Rpart));
  } else {
    a.M = s.V32;
    a.m_block_stride = 0;   // the shared U_i
    a.m_elems = (int64_t)s.C * s.nslots * s.mpad;
    a.out = s.Rpart;
    a.out_block_stride = s.fslots * s.mpad;
    a.out_elems = s.rpart_elems();
    CK(launch_pass1_simt(a, s.fslots, s.st));
  }
  return RFF_OK;
}

rff_status phase_project(rff_admm_t h, int k) {
  auto& s = *h;
  const int64_t nfe = s.fslots * s.mpad;
  const int64_t nblocks = (int64_t)s.R * s.C;
  int64_t smax = 0;
  for (int j = 0; j < s.C; ++j) smax = std::max(smax, s.col_size[j]);
  rff_status r;
  if ((r = mark(h, k, 2)) != RFF_OK) return r;
  // graph projection, eq. (gpWij): W'_ij = Q_ij (Wbar_j - mu'_ij + Z_ij^T (Obar_ij + nu_i)) with
  // the cached inverse Q_ij = (I + Z_ij^T Z_ij)^-1, taken incrementally from the previous
  // W'_ij and O'_ij = Z_ij W'_ij (Q_ij (I + Z_ij^T Z_ij) = I makes it the same map):
  //   W'_ij <- W'_ij + Q_ij (Wbar_j - mu'_ij - W'_ij + Z_ij^T U_i),  U_i = Obar_ij + nu_i - O'_ij.
  // Q_ij has gain up to 1 where I + Z_ij^T Z_ij has its small eigenvalues while it shrinks the
  // right-hand side by the largest ones (about 2e3 for correlated kernels), so a rounding of the
  // right-hand side reaches W'_ij amplified by up to that condition number: the increment's
  // right-hand side, and with it that rounding, is the smaller, and U_i is smaller than
  // Obar_ij + nu_i by O'_ij.
  if (s.split_path()) {
    // six-product split-BF16 GEMM on the tensor cores added into W' (reducing max |W'|), then
    // the transposed FP16 split of W' that pass 2 reads
    CK(launch_rhs_split3T(s.Wbar, s.muij, s.Rpart, s.cached_z() ? s.nsplit_cz : s.nsplit, s.R, s.fslots,
                          (int)s.mpad, s.feat_of_slot, s.rT1, s.rT2, s.rT3, s.st, s.What));
    CK(cudaMemsetAsync(s.amax + AMAX_W, 0, 4, s.st));
    CK(split_gemm(qgemm_view(s)));
    CK(launch_transpose_split_f16(s.What, s.fslots, (int)s.mpad, s.R, s.fslots * s.mpad, s.WThi, s.WTlo, s.fslots,
                                  s.mpad * s.fslots, 1.f, s.amax + AMAX_W, s.st));
  } else {
    CK(launch_rhs(s.Wbar, s.muij, s.Rpart, s.nsplit, s.R, nfe, s.rhs, s.st, nullptr, 0, s.What));
    CK(launch_gemm_f32_nn(s.gdesc, (int)nblocks, (int)smax, (int)s.mpad, 1.f, 1.f, s.st, s.act()));
  }
  if ((r = mark(h, k, 3)) != RFF_OK) return r;
  if (s.split_path()) CK(cudaMemsetAsync(s.amax + AMAX_OP, 0, 4, s.st));   // max |O'| for the exchange
  return RFF_OK;
}

// pass 2: O'_ij = Z_ij W'_ij (eq. (gpOij))
rff_status phase_pass2(rff_admm_t h) {
  auto& s = *h;
  PassArgs a = base_pass_args(s);
  a.bmask = s.act();
  if (s.cached_z()) {
    CK(split_gemm(cz_pass2_view(s)));
  } else if (s.split_path()) {
    CK(tc_pass2(iter_view(s), s.WThi, s.WTlo, s.mpad * s.fslots, s.Op, 1, s.amax + AMAX_W, s.amax + AMAX_OP));
  } else {
    a.M = s.What;
    a.m_block_stride = s.fslots * s.mpad;
    a.m_elems = (int64_t)s.R * s.fslots * s.mpad;
    a.out = s.Op;
    a.out_block_stride = s.nslots * s.mpad;
    a.out_elems = (int64_t)s.C * s.nslots * s.mpad;
    a.per_block = 1;
    CK(launch_pass2_simt(a, s.nslots, s.st));
  }
  return RFF_OK;
}

rff_status phase_post(rff_admm_t h, int k) {
  auto& s = *h;
  rff_status r;
  if (s.split_path() && s.stochastic())   // max |O'| over every block, the kept ones included
    CK(launch_finite_check(s.Op, s.C * s.nslots * s.mpad, 0, reinterpret_cast<int*>(s.amax + AMAX_FLAG), s.st,
                           s.amax + AMAX_OP));
  if ((r = mark(h, k, 4)) != RFF_OK) return r;
  // exchange, nu update, next loss prox, next V_ij (the tensor-core path reads V^T as a
  // scaled FP16 hi/lo pair), averaging and dual updates
  return exchange_and_average(h, k);
}

rff_status iterate(rff_admm_t h, int k) {
  auto& s = *h;
  if (s.outer) return iterate_outer(h, k);
  rff_status r;
  if ((r = phase_pre(h, k)) != RFF_OK) return r;
  if ((r = phase_pass1(h)) != RFF_OK) return r;
  if ((r = phase_project(h, k)) != RFF_OK) return r;
  if ((r = phase_pass2(h)) != RFF_OK) return r;
  if ((r = phase_post(h, k)) != RFF_OK) return r;
  s.launches += iter_launches(s);
  return RFF_OK;
}

// Capture one iteration (the same launches as iterate()) into an executable graph.
rff_status capture_iteration(rff_admm_t h) {
  auto& s = *h;
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(s.st, cudaStreamCaptureModeThreadLocal));
  const int64_t saved = s.launches;
  rff_status r = iterate(h, 0);
  s.launches = saved;
  cudaError_t e = cudaStreamEndCapture(s.st, &g);
  if (r != RFF_OK) {
    if (g) cudaGraphDestroy(g);
    return r;
  }
  if (e != cudaSuccess) return h->cuda_fail(e, "cudaStreamEndCapture");
  e = cudaGraphInstantiate(&s.gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    s.gexec = nullptr;
    return h->cuda_fail(e, "cudaGraphInstantiate");
  }
  return RFF_OK;
}

// Enqueue `iters` iterations on the handle's stream (no host synchronisation).
// copy_old: keep nu, Obar, mu, Wbar, mu' of the iteration before the last (residuals).
rff_status enqueue_iterations(rff_admm_t h, int iters, bool copy_old) {
  NvtxRange range("rff iterations");
  auto& s = *h;
  if (s.features_released) {   // a solve keeps them resident again
    rff_status r = regenerate_features(h);
    if (r != RFF_OK) return r;
  }
  const int64_t rowb = s.nslots * s.mpad * 4, colb = s.fslots * s.mpad * 4;
  const int base = s.pending_profiled;   // profiled iterations not yet accumulated
  if (s.profiling && (size_t)(base + iters) * 7 > s.ev.size()) {
    const size_t old = s.ev.size();
    s.ev.resize((size_t)(base + iters) * 7);
    for (size_t e = old; e < s.ev.size(); ++e) CK(cudaEventCreate(&s.ev[e]));
  }
  if (s.stochastic() && iters > 0) {   // the masks continue from the iteration count
    s.bctr_host = s.iters_done;
    CK(cudaMemcpyAsync(s.bctr, &s.bctr_host, sizeof(int64_t), cudaMemcpyHostToDevice, s.st));
  }
  for (int k = 0; k < iters; ++k) {
    if (copy_old && k == iters - 1) {
      CK(cudaMemcpyAsync(s.nu_old, s.nu, rowb, cudaMemcpyDeviceToDevice, s.st));
      CK(cudaMemcpyAsync(s.Obar_old, s.Obar, rowb, cudaMemcpyDeviceToDevice, s.st));
      CK(cudaMemcpyAsync(s.mu_old, s.mu, colb, cudaMemcpyDeviceToDevice, s.st));
      CK(cudaMemcpyAsync(s.Wbar_old, s.Wbar, colb, cudaMemcpyDeviceToDevice, s.st));
      CK(cudaMemcpyAsync(s.muij_old, s.muij, colb * s.R, cudaMemcpyDeviceToDevice, s.st));
    }
    rff_status r = RFF_OK;
    if (s.profiling || s.iters_done == 0) {
      r = iterate(h, base + k);
    } else {
      if (!s.gexec && (r = capture_iteration(h)) != RFF_OK) return r;
      CK(cudaGraphLaunch(s.gexec, s.st));
      s.launches += iter_launches(s);
    }
    if (r != RFF_OK) return r;
    s.iters_done++;
  }
  s.pending_profiled += s.profiling ? iters : 0;
  return RFF_OK;
}

// After the stream has drained: tensor-core error word, profiling accumulation.
rff_status finish_iterations(rff_admm_t h) {
  auto& s = *h;
  if (s.split_path() && tc_error_word() != 0)
    return h->fail(RFF_ETIMEOUT, "a tensor-core pass gave up waiting (device error word set)");
  if (s.pending_profiled > 0) {
    double* acc[6] = {&s.prof.ms_prox_reg, &s.prof.ms_pass1, &s.prof.ms_project, &s.prof.ms_pass2,
                      &s.prof.ms_exchange, &s.prof.ms_average};
    for (int k = 0; k < s.pending_profiled; ++k)
      for (int ph = 0; ph < 6; ++ph) {
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, s.ev[(size_t)k * 7 + ph], s.ev[(size_t)k * 7 + ph + 1]));
        *acc[ph] += ms;
      }
    s.prof.iters += s.pending_profiled;
    s.pending_profiled = 0;
  }
  return RFF_OK;
}

rff_status sum_partials(rff_admm_t h, double& out) {
  std::vector<double> hp(1024);
  CK(cudaMemcpyAsync(hp.data(), h->partials, 1024 * 8, cudaMemcpyDeviceToHost, h->st));
  CK(cudaStreamSynchronize(h->st));
  double sacc = 0.0;
  for (double v : hp) sacc += v;
  out = sacc;
  return RFF_OK;
}

rff_status sqdiff(rff_admm_t h, const float* a, const float* b, int64_t n, double& out) {
  CK(launch_sqdiff_partials(a, b, n, h->partials, 1024, h->st));
  return sum_partials(h, out);
}

// scores S (slots x m_pad) = Z(rows) Wbar, on the handle's training rows or a query batch
rff_status scores_pass(rff_admm_t h, const float* Xrows32, const __half* Xh, const __half* Xl,
                       int64_t nrows, const int32_t* row_ok, float* out) {
  auto& s = *h;
  if (s.tc_scores()) {
    CK(cudaMemsetAsync(s.amax + AMAX_WB, 0, 4, s.st));
    CK(launch_finite_check(s.Wbar, s.fslots * s.mpad, 0, reinterpret_cast<int*>(s.amax + AMAX_FLAG), s.st, s.amax + AMAX_WB));
    CK(launch_transpose_split_f16(s.Wbar, s.fslots, (int)s.mpad, 1, 0, s.WbThi, s.WbTlo, s.fslots, 0, 1.f,
                                  s.amax + AMAX_WB, s.st));
    CK(tc_predict(tc_view(s), Xh, Xl, nrows, s.WbThi, s.WbTlo, s.amax + AMAX_WB, out));
  } else if (s.tensorsketch()) {
    // the rows' sketches, TS_SCORE_ROWS at a time, then their product with Wbar in FP32
    for (int64_t r0 = 0; r0 < nrows; r0 += TS_SCORE_ROWS) {
      const int64_t nr = std::min<int64_t>(TS_SCORE_ROWS, nrows - r0);
      TsArgs ta = ts_args(s, Xrows32, s.dld, row_ok, r0, nr);
      ta.out = s.ts_buf;
      ta.ldo = s.fslots;
      ta.out_elems = nr * s.fslots;
      ta.pad = 1;
      CK(launch_tensorsketch(ta, s.C, ts_block_max(s), s.st));
      const GemmDesc g{s.ts_buf, s.Wbar, nullptr, out + r0 * s.mpad, (int)nr, (int)s.mpad, (int)s.fslots,
                       s.fslots, s.mpad, s.mpad, s.mpad};
      CK(launch_gemm_f32_nn_one(g, 1.f, 0.f, s.st));
    }
  } else {
    PassArgs a = base_pass_args(s);
    a.X = Xrows32;
    a.row_ok = row_ok;
    a.row_slot = s.d_zero;
    a.R = 1;
    a.M = s.Wbar;
    a.m_block_stride = 0;
    a.m_elems = s.fslots * s.mpad;
    a.x_rows = nrows;
    a.out = out;
    a.out_block_stride = 0;
    a.out_elems = nrows * s.mpad;
    a.per_block = 0;
    CK(launch_pass2_simt(a, nrows, s.st));
  }
  return RFF_OK;
}

}  // namespace

// ------------------------------------------------------------------ tc.h glue used by tc.cu
namespace rff {
TcView tc_view(const rff_admm_s& s) {
  TcView v{};
  v.Xhi = s.Xhi; v.Xlo = s.Xlo; v.Ghi = s.Ghi; v.Glo = s.Glo;
  v.VThi = s.VThi; v.VTlo = s.VTlo; v.v_amax = s.amax;
  v.bias = s.bias; v.row_ok = s.row_of_slot; v.feat_ok = s.feat_of_slot;
  v.nslots = s.nslots; v.fslots = s.fslots; v.dld = s.dld; v.mpad = s.mpad;
  v.R = s.R; v.C = s.C; v.nsplit = s.nsplit;
  v.row_slot = s.row_slot.data(); v.row_size = s.row_size.data();
  v.col_slot = s.col_slot.data(); v.col_size = s.col_size.data();
  v.d_row_slot = s.d_row_slot; v.d_row_size = s.d_row_size; v.d_col_slot = s.d_col_slot; v.d_col_size = s.d_col_size;
  v.scale = (float)std::sqrt(2.0 / (double)s.D);
  v.inv_xg = 1.f / (s.xscale * s.gscale);
  v.bias_in_mma = s.bias_col >= 0 ? 1 : 0;
  v.kc = s.tc_kc;
  v.zt = s.tc_zt;
  v.cg = s.tc_cg;
  v.v_shared = s.incremental() ? 1 : 0;
  v.st = s.st;
  return v;
}
}  // namespace rff

extern "C" {

rff_status rff_admm_solve(rff_admm_t h, int32_t iters, rff_admm_stats* stats) {
  if (!h) return RFF_EINVAL;
  h->err.clear();
  if (!h->has_data) return h->fail(RFF_ENOTREADY, "no data: call rff_admm_set_data first");
  if (iters < 0) return h->fail(RFF_EINVAL, "iters must be >= 0");
  auto& s = *h;
  cudaEvent_t e0, e1, e2;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventCreate(&e2));
  CK(cudaEventRecord(e0, s.st));
  if (!s.factored) {
    rff_status r = setup_factors(h);
    if (r != RFF_OK) return r;
  }
  CK(cudaEventRecord(e1, s.st));
  {
    rff_status r = enqueue_iterations(h, iters, stats != nullptr);
    if (r != RFF_OK) return r;
  }
  CK(cudaEventRecord(e2, s.st));
  CK(cudaEventSynchronize(e2));
  {
    rff_status r = finish_iterations(h);
    if (r != RFF_OK) return r;
  }
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    float ms0 = 0, ms1 = 0;
    cudaEventElapsedTime(&ms0, e0, e1);
    cudaEventElapsedTime(&ms1, e1, e2);
    stats->ms_setup = ms0;
    stats->ms_iterations = ms1;
    stats->iters_done = s.iters_done;
    rff_status r;
    if (iters > 0) {
      // primal: |O - Obar| = |nu^k - nu^{k-1}|, |W - Wbar| = |mu^k - mu^{k-1}|, |W'_ij - Wbar| likewise
      double a1, a2, a3, b1, b2;
      if ((r = sqdiff(h, s.nu, s.nu_old, s.nslots * s.mpad, a1)) != RFF_OK) return r;
      if ((r = sqdiff(h, s.mu, s.mu_old, s.fslots * s.mpad, a2)) != RFF_OK) return r;
      if ((r = sqdiff(h, s.muij, s.muij_old, s.R * s.fslots * s.mpad, a3)) != RFF_OK) return r;
      if ((r = sqdiff(h, s.Wbar, s.Wbar_old, s.fslots * s.mpad, b1)) != RFF_OK) return r;
      if ((r = sqdiff(h, s.Obar, s.Obar_old, s.nslots * s.mpad, b2)) != RFF_OK) return r;
      stats->primal_res = std::sqrt(a1 + a2 + a3);
      stats->dual_res = s.p.rho * std::sqrt(b1 + b2);
    }
    // objective at Wbar: the training rows scored in chunks into a buffer that no iteration
    // carries over (O'_ij is: the outer form updates it, and a stochastic iteration's inactive
    // blocks keep it): the outer form's product scratch, else the pass-1 partials
    double loss = 0, reg = 0;
    float* sc = s.outer ? s.U32 : s.Rpart;
    const int64_t chunk = s.outer ? s.nslots
                                  : std::min<int64_t>(s.nslots, std::max<int64_t>(SLOT, s.rpart_elems() / s.mpad / SLOT * SLOT));
    for (int64_t r0 = 0; r0 < s.nslots; r0 += chunk) {
      const int64_t nr = std::min(chunk, s.nslots - r0);
      if ((r = scores_pass(h, s.X32 ? s.X32 + r0 * s.dld : nullptr, s.Xhi ? s.Xhi + r0 * s.dld : nullptr,
                           s.Xlo ? s.Xlo + r0 * s.dld : nullptr, nr, s.row_of_slot + r0, sc)) != RFF_OK)
        return r;
      CK(launch_loss_partials(s.p.loss, s.Y + r0 * s.mpad, sc, s.row_of_slot + r0, nr, (int)s.m, (int)s.mpad,
                              s.partials, 1024, s.st));
      double part = 0;
      if ((r = sum_partials(h, part)) != RFF_OK) return r;
      loss += part;
    }
    CK(launch_reg_partials(s.p.reg, s.Wbar, s.fslots * s.mpad, s.partials, 1024, s.st, s.lam_dev, (int)s.mpad));
    if ((r = sum_partials(h, reg)) != RFF_OK) return r;
    stats->objective = loss + (double)s.n * s.p.lambda * reg;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaEventDestroy(e2);
  return RFF_OK;
}

rff_status rff_admm_set_memory_limit(rff_admm_t h, size_t bytes) {
  if (!h) return RFF_EINVAL;
  h->mem_limit = bytes;
  return RFF_OK;
}

rff_status rff_admm_set_stream(rff_admm_t h, void* cuda_stream) {
  if (!h || !cuda_stream) return RFF_EINVAL;
  h->err.clear();
  cudaStream_t ns = static_cast<cudaStream_t>(cuda_stream);
  if (ns == h->st) return RFF_OK;
  CK(cudaStreamSynchronize(h->st));
  if (h->own_stream) cudaStreamDestroy(h->st);
  h->st = ns;
  h->own_stream = false;
  return RFF_OK;
}

rff_status rff_admm_estimate_bytes(const rff_admm_params* params, int64_t n, int64_t d, size_t* resident,
                                   size_t* peak) {
  std::string why;
  rff_status st = check_params(params, why);
  if (st != RFF_OK) return st;
  if (n < params->R || d < 1 || n > ((int64_t)1 << 31) - 1) return RFF_EINVAL;
  rff_admm_s s;
  s.p = *params;
  compute_geometry(s, n, d);
  const size_t ws = working_set_bytes(s);
  if (resident) *resident = ws;
  if (peak) *peak = ws + setup_bytes(s, 1) + (size_t)n * (d + s.m) * 4 + (size_t)s.nslots * s.dld * 4;
  return RFF_OK;
}

rff_status rff_admm_predict_labels(rff_admm_t h, const float* Xq, int64_t q, int32_t* labels, int is_device_ptr) {
  if (!h) return RFF_EINVAL;
  h->err.clear();
  if (q < 0) return h->fail(RFF_EINVAL, "q < 0");
  if (q == 0) return RFF_OK;
  if (!Xq || !labels) return h->fail(RFF_EINVAL, "NULL pointer");
  auto& s = *h;
  // scores into a stream-ordered temporary (device queries are read in place), then the labels
  const size_t sb = round_up((size_t)q * s.m * 4, 256), lb = (size_t)q * 4;
  char* tmp = nullptr;
  if (cudaMallocAsync((void**)&tmp, sb + lb + (is_device_ptr ? 0 : (size_t)q * s.d * 4), s.st) != cudaSuccess) {
    cudaGetLastError();
    return h->fail(RFF_ENOMEM, "label scratch");
  }
  float* sc = reinterpret_cast<float*>(tmp);
  int32_t* lab = reinterpret_cast<int32_t*>(tmp + sb);
  const float* xq = Xq;
  rff_status r = RFF_OK;
  cudaError_t e = cudaSuccess;
  if (!is_device_ptr) {
    float* xd = reinterpret_cast<float*>(tmp + sb + lb);
    e = cudaMemcpyAsync(xd, Xq, (size_t)q * s.d * 4, cudaMemcpyHostToDevice, s.st);
    xq = xd;
  }
  if (e == cudaSuccess) r = rff_admm_predict(h, xq, q, sc, 1);
  if (e == cudaSuccess && r == RFF_OK) e = launch_argmax_rows(sc, q, (int)s.m, s.m, lab, s.st);
  if (e == cudaSuccess && r == RFF_OK)
    e = cudaMemcpyAsync(labels, lab, lb, is_device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s.st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s.st);
  cudaFreeAsync(tmp, s.st);
  if (r != RFF_OK) return r;
  if (e != cudaSuccess) return h->cuda_fail(e, "predict_labels");
  return RFF_OK;
}

int32_t rff_check_enabled(void) {
#ifdef RFF_CHECK
  return 1;
#else
  return 0;
#endif
}

rff_status rff_check_report(int64_t* out) {
  if (!out) return RFF_EINVAL;
  for (int k = 0; k < 5; ++k) out[k] = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return RFF_ECUDA;
  }
  // the units in the order of their numbers in the report
  cudaError_t (*const units[])(CheckHit*) = {check_collect_elementwise, check_collect_qgemm,
                                             check_collect_regen_simt,  check_collect_tc,
                                             check_collect_sketch,      check_collect_ozaki};
  for (int u = 0; u < 6; ++u) {
    CheckHit hit{};
    if (units[u](&hit) != cudaSuccess) {
      cudaGetLastError();
      return RFF_ECUDA;
    }
    if (hit.count == 0) continue;
    if (out[0] == 0) {
      out[1] = u + 1;
      out[2] = hit.line;
      out[3] = hit.index;
      out[4] = hit.bound;
    }
    out[0] += (int64_t)hit.count;
  }
  return RFF_OK;
}

rff_status rff_selftest_wait_timeout(void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (tc_error_word() != 0) return RFF_ECUDA;   // a failure nobody has collected yet
  if (tc_wait_probe(2000000, st) != cudaSuccess) return RFF_ECUDA;   // ~1 ms at the boost clock
  if (cudaStreamSynchronize(st) != cudaSuccess) return RFF_ECUDA;
  return tc_error_word() != 0 ? RFF_ETIMEOUT : RFF_OK;
}

rff_status rff_admm_release_features(rff_admm_t h, size_t* bytes) {
  if (!h) return RFF_EINVAL;
  h->err.clear();
  if (!h->has_data || !h->factored) return h->fail(RFF_ENOTREADY, "release_features needs a solve first");
  return release_features(h, bytes);
}

rff_status rff_admm_set_block_fraction(rff_admm_t h, double p) {
  if (!h) return RFF_EINVAL;
  h->err.clear();
  if (!(p > 0.0 && p <= 1.0)) return h->fail(RFF_EINVAL, "block fraction must be in (0, 1]");
  const double thr = std::floor(p * 16777216.0);
  if (thr < 1.0) return h->fail(RFF_EINVAL, "block fraction below 2^-24");
  h->bfrac = p;
  h->bthr = (uint32_t)thr;
  h->drop_graph();   // the captured iteration has a different launch sequence
  return RFF_OK;
}

rff_status rff_admm_set_lambdas(rff_admm_t h, const double* lambdas, int32_t m) {
  if (!h) return RFF_EINVAL;
  h->err.clear();
  if (!lambdas) {
    h->lam_col.clear();
  } else {
    if (m != h->p.m) return h->fail(RFF_EINVAL, "need one lambda per output column");
    for (int32_t c = 0; c < m; ++c)
      if (!(lambdas[c] > 0) || !std::isfinite(lambdas[c])) return h->fail(RFF_EINVAL, "lambdas must be > 0");
    h->lam_col.assign(lambdas, lambdas + m);
  }
  return upload_lambdas(h);
}

rff_status rff_admm_enqueue(rff_admm_t h, int32_t iters) {
  if (!h) return RFF_EINVAL;
  h->err.clear();
  if (!h->has_data) return h->fail(RFF_ENOTREADY, "no data: call rff_admm_set_data first");
  if (iters < 0) return h->fail(RFF_EINVAL, "iters must be >= 0");
  if (!h->factored) {
    rff_status r = setup_factors(h);
    if (r != RFF_OK) return r;
  }
  return enqueue_iterations(h, iters, false);
}

rff_status rff_admm_wait(rff_admm_t h) {
  if (!h) return RFF_EINVAL;
  CK(cudaStreamSynchronize(h->st));
  return finish_iterations(h);
}

}  // extern "C"

namespace {
// One iteration of every solve of a sweep as a single executable graph: from a fork on the
// master stream each solve's iteration is captured on its own stream (its kernels form a branch
// of the graph), and the branches join back on the master stream.  The solves in `fused`
// (split precision, Gram form) run their two regeneration passes as two launches for all of
// them together (m1, m2: k_regen_multi, their CTAs side by side in one grid) on the master
// stream, between their other phases, which stay on their own streams:
//   fork -> [pre] -> join -> pass 1 of all -> fork -> [projection] -> join -> pass 2 of all ->
//   fork -> [exchange, averaging] -> join.
// One graph launch then runs one iteration of all solves.
rff_status capture_sweep(rff_admm_t* hs, int32_t n, cudaStream_t master, const std::vector<int>& fused,
                         const TcMulti* m1, const TcMulti* m2, cudaGraphExec_t* out) {
  std::vector<cudaEvent_t> evs;
  auto cleanup = [&]() {
    for (auto e : evs) cudaEventDestroy(e);
  };
  auto new_event = [&](cudaEvent_t* ev) -> cudaError_t {
    cudaError_t e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
    if (e == cudaSuccess) evs.push_back(*ev);
    return e;
  };
  // master -> stream (a fork) or stream -> master (a join)
  auto order = [&](cudaStream_t from, cudaStream_t to) -> cudaError_t {
    cudaEvent_t ev = nullptr;
    cudaError_t e = new_event(&ev);
    if (e == cudaSuccess) e = cudaEventRecord(ev, from);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(to, ev, 0);
    return e;
  };
  std::vector<char> is_fused(n, 0);
  for (int k : fused) is_fused[k] = 1;
  if (cudaStreamBeginCapture(master, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cleanup();
    return RFF_ECUDA;
  }
  rff_status r = RFF_OK;
  cudaError_t e = cudaSuccess;
  // the solves iterated whole on their own streams
  for (int32_t k = 0; k < n && r == RFF_OK && e == cudaSuccess; ++k) {
    if (is_fused[k]) continue;
    rff_admm_t h = hs[k];
    e = order(master, h->st);
    if (e != cudaSuccess) break;
    const int64_t saved = h->launches;
    r = iterate(h, 0);
    h->launches = saved;
    if (e == cudaSuccess) e = order(h->st, master);
  }
  // the fused solves, phase by phase around the shared pass launches
  using Phase = rff_status (*)(rff_admm_t, int);
  const Phase phases[3] = {phase_pre, phase_project, phase_post};
  for (int p = 0; p < 3 && !fused.empty() && r == RFF_OK && e == cudaSuccess; ++p) {
    for (int k : fused) {
      rff_admm_t h = hs[k];
      if ((e = order(master, h->st)) != cudaSuccess) break;
      const int64_t saved = h->launches;
      r = phases[p](h, 0);
      h->launches = saved;
      if (r != RFF_OK || (e = order(h->st, master)) != cudaSuccess) break;
    }
    if (r == RFF_OK && e == cudaSuccess && p < 2) e = tc_multi_launch(p == 0 ? m1 : m2, master);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(master, &g);
  if (r == RFF_OK && (e != cudaSuccess || ee != cudaSuccess)) r = RFF_ECUDA;
  if (r == RFF_OK && cudaGraphInstantiate(out, g, 0) != cudaSuccess) r = RFF_ECUDA;
  if (g) cudaGraphDestroy(g);
  cleanup();
  cudaGetLastError();
  return r;
}

// The solves of a sweep whose passes can share launches: the split precision in the Gram form
// (the passes of k_regen_tc), at least two of them, unless RFF_SWEEP_FUSE=0 keeps every solve's
// passes to itself.
std::vector<int> fusable(rff_admm_t* hs, int32_t n) {
  std::vector<int> f;
  const char* env = getenv("RFF_SWEEP_FUSE");
  if (env && atoi(env) == 0) return f;
  for (int32_t k = 0; k < n && (int)f.size() < 64; ++k) {
    const auto& s = *hs[k];
    if (s.split_path() && !s.cached_z() && !s.outer) f.push_back(k);
  }
  if (f.size() < 2) f.clear();
  return f;
}
}  // namespace

extern "C" {
rff_status rff_sweep_run(rff_admm_t* handles, int32_t n, int32_t iters) {
  if (n < 0 || iters < 0 || (n > 0 && !handles)) return RFF_EINVAL;
  for (int32_t k = 0; k < n; ++k)
    if (!handles[k] || !handles[k]->has_data) return RFF_EINVAL;
  if (n == 0 || iters == 0) return RFF_OK;
  // set-up of every solve first (factors are computed once per handle) ...
  for (int32_t k = 0; k < n; ++k)
    if (!handles[k]->factored) {
      rff_status r = setup_factors(handles[k]);
      if (r != RFF_OK) return r;
    }
  // ... a first, eager iteration of the solves that have none (it also brings back released
  // feature parameters and points the stochastic masks at the right iteration) ...
  int32_t left = iters;
  bool eager = false;
  for (int32_t k = 0; k < n; ++k) eager = eager || handles[k]->iters_done == 0 || handles[k]->profiling ||
                                          handles[k]->features_released;
  rff_status first = RFF_OK;
  if (eager) {
    for (int32_t k = 0; k < n; ++k) {
      rff_status r = enqueue_iterations(handles[k], 1, false);
      if (r != RFF_OK && first == RFF_OK) first = r;
    }
    --left;
  }
  // ... then the rest as one graph launch per iteration for all solves together
  if (left > 0 && first == RFF_OK) {
    bool profiling = false;
    for (int32_t k = 0; k < n; ++k) profiling = profiling || handles[k]->profiling;
    cudaStream_t master = nullptr;
    cudaGraphExec_t gx = nullptr;
    if (profiling || cudaStreamCreateWithFlags(&master, cudaStreamNonBlocking) != cudaSuccess) {
      // per-phase events need eager launches: each solve on its own stream, side by side
      cudaGetLastError();
      for (int32_t k = 0; k < n; ++k) {
        rff_status r = enqueue_iterations(handles[k], left, false);
        if (r != RFF_OK && first == RFF_OK) first = r;
      }
    } else {
      // every solve's pending work is ordered before the graph, and its stochastic masks
      // continue from its own iteration count
      cudaEvent_t ready = nullptr;
      rff_status r = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) == cudaSuccess ? RFF_OK : RFF_ECUDA;
      for (int32_t k = 0; k < n && r == RFF_OK; ++k) {
        rff_admm_t h = handles[k];
        if (h->stochastic()) {
          h->bctr_host = h->iters_done;
          if (cudaMemcpyAsync(h->bctr, &h->bctr_host, sizeof(int64_t), cudaMemcpyHostToDevice, h->st) != cudaSuccess)
            r = RFF_ECUDA;
        }
        if (r == RFF_OK && (cudaEventRecord(ready, h->st) != cudaSuccess ||
                            cudaStreamWaitEvent(master, ready, 0) != cudaSuccess))
          r = RFF_ECUDA;
      }
      if (ready) cudaEventDestroy(ready);
      // the shared pass launches' arguments (written to device memory before the capture)
      const std::vector<int> fused = fusable(handles, n);
      TcMulti *m1 = nullptr, *m2 = nullptr;
      if (r == RFF_OK && !fused.empty()) {
        std::vector<TcView> views;
        std::vector<float*> rp, op;
        std::vector<const __half*> mh, ml;
        std::vector<const unsigned*> ma;
        std::vector<unsigned*> oa;
        for (int k : fused) {
          auto& s = *handles[k];
          views.push_back(iter_view(s));
          rp.push_back(s.Rpart);
          op.push_back(s.Op);
          mh.push_back(s.WThi);
          ml.push_back(s.WTlo);
          ma.push_back(s.amax + AMAX_W);
          oa.push_back(s.amax + AMAX_OP);
        }
        const int nf = (int)fused.size();
        if (tc_multi_create(views.data(), nf, 1, rp.data(), nullptr, nullptr, nullptr, nullptr, &m1) != cudaSuccess ||
            tc_multi_create(views.data(), nf, 2, op.data(), mh.data(), ml.data(), ma.data(), oa.data(), &m2) !=
                cudaSuccess)
          r = RFF_ECUDA;
      }
      if (r == RFF_OK) r = capture_sweep(handles, n, master, fused, m1, m2, &gx);
      for (int32_t it = 0; it < left && r == RFF_OK; ++it)
        if (cudaGraphLaunch(gx, master) != cudaSuccess) r = RFF_ECUDA;
      // the solves' streams wait for the graph before their next work
      cudaEvent_t done = nullptr;
      if (r == RFF_OK && cudaEventCreateWithFlags(&done, cudaEventDisableTiming) == cudaSuccess) {
        cudaEventRecord(done, master);
        for (int32_t k = 0; k < n; ++k) cudaStreamWaitEvent(handles[k]->st, done, 0);
        cudaEventDestroy(done);
      }
      if (r == RFF_OK)
        for (int32_t k = 0; k < n; ++k) {
          handles[k]->iters_done += left;
          handles[k]->launches += (int64_t)left * iter_launches(*handles[k]);
        }
      cudaStreamSynchronize(master);
      if (gx) cudaGraphExecDestroy(gx);
      tc_multi_destroy(m1);
      tc_multi_destroy(m2);
      cudaStreamDestroy(master);
      if (r != RFF_OK && first == RFF_OK) first = r;
    }
  }
  for (int32_t k = 0; k < n; ++k) {
    rff_status r = rff_admm_wait(handles[k]);
    if (r != RFF_OK && first == RFF_OK) first = r;
  }
  return first;
}

rff_status rff_admm_predict(rff_admm_t h, const float* Xq, int64_t q, float* scores, int is_device_ptr) {
  if (!h) return RFF_EINVAL;
  NvtxRange range("rff predict");
  h->err.clear();
  if (!h->has_data || !h->factored) return h->fail(RFF_ENOTREADY, "predict needs a solve first");
  if (q < 0) return h->fail(RFF_EINVAL, "q < 0");
  if (q == 0) return RFF_OK;
  if (!Xq || !scores) return h->fail(RFF_EINVAL, "NULL pointer");
  auto& s = *h;
  if (s.features_released) {   // regenerated for this call only, then given back again
    rff_status r = regenerate_features(h);
    if (r == RFF_OK) r = rff_admm_predict(h, Xq, q, scores, is_device_ptr);
    size_t freed = 0;
    release_features(h, &freed);
    return r;
  }
  const int64_t chunk = std::min<int64_t>(round_up(q, SLOT), 65536);
  const size_t need = (size_t)chunk * s.d * 4 + (size_t)chunk * s.dld * 4 + (size_t)chunk * s.dld * 2 * 2 +
                      (size_t)chunk * s.mpad * 4 + 4096;
  rff_status r = ensure_scratch(h, need);
  if (r != RFF_OK) return r;
  float* stage = static_cast<float*>(s.scratch.p);
  float* xq32 = stage + round_up(chunk * s.d, 64);
  __half* xh = reinterpret_cast<__half*>(xq32 + chunk * s.dld);
  __half* xl = xh + chunk * s.dld;
  float* sc = reinterpret_cast<float*>(xl + chunk * s.dld);
  const cudaMemcpyKind kin = is_device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind kout = is_device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  for (int64_t q0 = 0; q0 < q; q0 += chunk) {
    const int64_t nq = std::min(chunk, q - q0), nqp = round_up(nq, SLOT);
    CK(cudaMemcpyAsync(stage, Xq + q0 * s.d, nq * s.d * 4, kin, s.st));
    CK(cudaMemsetAsync(s.flag, 0, 16, s.st));
    CK(launch_finite_check(stage, nq * s.d, s.p.feature_map == RFF_MAP_LAPLACE ? 2 : 0, s.flag, s.st,
                           reinterpret_cast<unsigned*>(s.flag + 2)));
    int fl[3] = {0, 0, 0};
    CK(cudaMemcpyAsync(fl, s.flag, 12, cudaMemcpyDeviceToHost, s.st));
    CK(cudaStreamSynchronize(s.st));
    if (fl[0] & 1) return h->fail(RFF_EINVAL, "queries contain NaN or Inf");
    if (fl[0] & 4) return h->fail(RFF_EINVAL, "the random Laplace map takes nonnegative queries");
    if ((r = check_query_range(h, fl[2])) != RFF_OK) return r;
    // rows q0..q0+nq into a slot-padded block (rows beyond nq are zero and discarded)
    CK(cudaMemsetAsync(xq32, 0, nqp * s.dld * 4, s.st));
    CK(launch_gather_rows(stage, s.d, s.d, nullptr, nq, xq32, s.dld, s.st));
    if (s.bias_col >= 0) CK(launch_set_column(xq32, s.dld, nqp, s.bias_col, 1.f, s.st));
    if (s.tc_scores()) CK(launch_split_f16(xq32, nqp * s.dld, s.xscale, xh, xl, s.st));
    if ((r = scores_pass(h, xq32, xh, xl, nqp, nullptr, sc)) != RFF_OK) return r;
    CK(cudaMemcpy2DAsync(scores + q0 * s.m, s.m * 4, sc, s.mpad * 4, s.m * 4, nq, kout, s.st));
  }
  CK(cudaStreamSynchronize(s.st));
  return RFF_OK;
}

rff_status rff_admm_get_weights(rff_admm_t h, float* Wout, int is_device_ptr) {
  if (!h) return RFF_EINVAL;
  h->err.clear();
  if (!h->has_data) return h->fail(RFF_ENOTREADY, "no data");
  if (!Wout) return h->fail(RFF_EINVAL, "NULL pointer");
  auto& s = *h;
  rff_status r = ensure_scratch(h, (size_t)s.D * s.m * 4 + 256);
  if (r != RFF_OK) return r;
  float* tmp = static_cast<float*>(s.scratch.p);
  CK(launch_gather_rows(s.Wbar, s.mpad, s.m, s.slot_of_feat, s.D, tmp, s.m, s.st));
  CK(cudaMemcpyAsync(Wout, tmp, (size_t)s.D * s.m * 4, is_device_ptr ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     s.st));
  CK(cudaStreamSynchronize(s.st));
  return RFF_OK;
}

// ---- checkpoint: header + raw slot-layout arrays
namespace {
struct StateHeader {
  char magic[8];
  uint32_t version, pad;
  rff_admm_params p;
  int64_t n, d, m, nslots, fslots;
  int32_t R, C, iters_done, reserved;
};
struct Piece {
  void* ptr;
  size_t bytes;
};
// the iteration's state: O, Obar, nu, O'_ij, the pass-1 operand (V, or on the tensor-core
// path the FP16 split of V^T with the maxima that scale it), W, Wbar, mu, W'_ij, mu'_ij
// (O'_ij and W'_ij carry over to the next iteration for the blocks a stochastic iteration
// leaves out)
std::vector<Piece> state_pieces(rff_admm_s& s) {
  const size_t rowb = (size_t)s.nslots * s.mpad * 4, colb = (size_t)s.fslots * s.mpad * 4;
  std::vector<Piece> v{{s.O, rowb}, {s.Obar, rowb}, {s.nu, rowb}, {s.Op, rowb * s.C}};
  if (s.split_path() && !s.outer) {
    v.push_back({s.VThi, rowb / 2 * s.C});
    v.push_back({s.VTlo, rowb / 2 * s.C});
    v.push_back({s.amax, AMAX_WORDS * 4});
  } else {
    v.push_back({s.V32, rowb * s.C});
  }
  for (Piece pc : std::vector<Piece>{{s.W, colb}, {s.Wbar, colb}, {s.mu, colb}, {s.What, colb * s.R},
                                     {s.muij, colb * s.R}})
    v.push_back(pc);
  return v;
}
}  // namespace

rff_status rff_admm_get_state(rff_admm_t h, void* buf, size_t* bytes) {
  if (!h || !bytes) return RFF_EINVAL;
  h->err.clear();
  if (!h->has_data) return h->fail(RFF_ENOTREADY, "no data");
  auto pieces = state_pieces(*h);
  size_t need = sizeof(StateHeader);
  for (auto& pc : pieces) need += pc.bytes;
  if (!buf) {
    *bytes = need;
    return RFF_OK;
  }
  if (*bytes < need) return h->fail(RFF_EINVAL, "buffer too small");
  StateHeader hd{};
  memcpy(hd.magic, "RFFADMM", 8);
  hd.version = 2;
  hd.p = h->p;
  hd.n = h->n; hd.d = h->d; hd.m = h->m; hd.nslots = h->nslots; hd.fslots = h->fslots;
  hd.R = h->R; hd.C = h->C; hd.iters_done = h->iters_done;
  char* out = static_cast<char*>(buf);
  memcpy(out, &hd, sizeof(hd));
  size_t off = sizeof(hd);
  for (auto& pc : pieces) {
    CK(cudaMemcpyAsync(out + off, pc.ptr, pc.bytes, cudaMemcpyDeviceToHost, h->st));
    off += pc.bytes;
  }
  CK(cudaStreamSynchronize(h->st));
  *bytes = need;
  return RFF_OK;
}

rff_status rff_admm_set_state(rff_admm_t h, const void* buf, size_t bytes) {
  if (!h || !buf) return RFF_EINVAL;
  h->err.clear();
  if (!h->has_data) return h->fail(RFF_ENOTREADY, "no data");
  auto& s = *h;
  auto pieces = state_pieces(s);
  size_t need = sizeof(StateHeader);
  for (auto& pc : pieces) need += pc.bytes;
  if (bytes != need) return h->fail(RFF_EINVAL, "state size mismatch");
  StateHeader hd;
  memcpy(&hd, buf, sizeof(hd));
  if (memcmp(hd.magic, "RFFADMM", 8) != 0 || hd.version != 2) return h->fail(RFF_EINVAL, "not a state buffer");
  if (hd.n != s.n || hd.d != s.d || hd.m != s.m || hd.R != s.R || hd.C != s.C || hd.p.D != s.p.D ||
      hd.p.seed != s.p.seed || hd.p.loss != s.p.loss || hd.p.reg != s.p.reg || hd.p.prec != s.p.prec ||
      hd.p.lambda != s.p.lambda || hd.p.sigma != s.p.sigma || hd.p.rho != s.p.rho ||
      hd.p.rho_scale != s.p.rho_scale || hd.p.feature_map != s.p.feature_map)
    return h->fail(RFF_EINVAL, "state was written for other data, parameters or grid");
  if (!s.factored) {   // the set-up writes scratch into state buffers (the tuning passes): run it first
    rff_status r = setup_factors(h);
    if (r != RFF_OK) return r;
  }
  const char* in = static_cast<const char*>(buf);
  size_t off = sizeof(hd);
  for (auto& pc : pieces) {
    CK(cudaMemcpyAsync(pc.ptr, in + off, pc.bytes, cudaMemcpyHostToDevice, s.st));
    off += pc.bytes;
  }
  CK(cudaStreamSynchronize(s.st));
  s.iters_done = hd.iters_done;
  return RFF_OK;
}

}  // extern "C"

// Scoring into caller-provided scratch (used by the allocation-free entry point in
// noalloc.cu).  Xq and scores are device pointers; scratch holds the slot-padded
// queries, their BF16 split and the padded scores.
namespace rff {
rff_status predict_into_scratch(rff_admm_t h, const float* Xq, int64_t q, float* scores, void* scratch,
                                size_t scratch_bytes) {
  if (!h) return RFF_EINVAL;
  h->err.clear();
  if (!h->has_data || !h->factored) return h->fail(RFF_ENOTREADY, "predict needs a solve first");
  if (h->features_released)
    return h->fail(RFF_ENOTREADY, "the feature parameters were released; regenerating them allocates");
  if (q < 0) return h->fail(RFF_EINVAL, "q < 0");
  if (q == 0) return RFF_OK;
  if (!Xq || !scores || !scratch) return h->fail(RFF_EINVAL, "NULL pointer");
  auto& s = *h;
  const int64_t qp = round_up(q, SLOT);
  const size_t x32 = (size_t)qp * s.dld * 4, xsplit = s.split_path() ? (size_t)qp * s.dld * 2 : 0,
               scb = (size_t)qp * s.mpad * 4;
  const size_t need = round_up(x32, 256) + 2 * round_up(xsplit, 256) + scb;
  if (need > scratch_bytes)
    return h->fail(RFF_EINVAL, "q = " + std::to_string(q) + " needs " + std::to_string(need) +
                                   " bytes of the fixed scratch, which holds " + std::to_string(scratch_bytes) +
                                   ": score the queries in smaller batches");
  char* base = static_cast<char*>(scratch);
  float* xq32 = reinterpret_cast<float*>(base);
  __half* xh = reinterpret_cast<__half*>(base + round_up(x32, 256));
  __half* xl = reinterpret_cast<__half*>(base + round_up(x32, 256) + round_up(xsplit, 256));
  float* sc = reinterpret_cast<float*>(base + round_up(x32, 256) + 2 * round_up(xsplit, 256));
  CK(cudaMemsetAsync(s.flag, 0, 16, s.st));
  CK(launch_finite_check(Xq, q * s.d, s.p.feature_map == RFF_MAP_LAPLACE ? 2 : 0, s.flag, s.st,
                         reinterpret_cast<unsigned*>(s.flag + 2)));
  int fl[3] = {0, 0, 0};
  CK(cudaMemcpyAsync(fl, s.flag, 12, cudaMemcpyDeviceToHost, s.st));
  CK(cudaStreamSynchronize(s.st));
  if (fl[0] & 1) return h->fail(RFF_EINVAL, "queries contain NaN or Inf");
  if (fl[0] & 4) return h->fail(RFF_EINVAL, "the random Laplace map takes nonnegative queries");
  {
    rff_status rr = check_query_range(h, fl[2]);
    if (rr != RFF_OK) return rr;
  }
  // the scratch keeps the previous call's contents: the padding rows are cleared here
  CK(cudaMemsetAsync(xq32, 0, x32, s.st));
  CK(launch_gather_rows(Xq, s.d, s.d, nullptr, q, xq32, s.dld, s.st));
  if (s.bias_col >= 0) CK(launch_set_column(xq32, s.dld, qp, s.bias_col, 1.f, s.st));
  if (s.tc_scores()) CK(launch_split_f16(xq32, qp * s.dld, s.xscale, xh, xl, s.st));
  rff_status r = scores_pass(h, xq32, xh, xl, qp, nullptr, sc);
  if (r != RFF_OK) return r;
  CK(cudaMemcpy2DAsync(scores, s.m * 4, sc, s.mpad * 4, s.m * 4, q, cudaMemcpyDeviceToDevice, s.st));
  CK(cudaStreamSynchronize(s.st));
  return RFF_OK;
}
}  // namespace rff

extern "C" {

// ------------------------------------------------------------------ step-level entry points
rff_status rff_philox4x32_10(const uint32_t* ctr, uint64_t seed, int64_t n, uint32_t* out, void* stream) {
  if (n < 0 || (n > 0 && (!ctr || !out))) return RFF_EINVAL;
  return launch_philox_raw(ctr, seed, n, out, static_cast<cudaStream_t>(stream)) == cudaSuccess ? RFF_OK
                                                                                                : RFF_ECUDA;
}

rff_status rff_rff_params(uint64_t seed, double sigma, int64_t d, int64_t k_lo, int64_t k_hi, float* G, float* b,
                          void* stream) {
  if (d < 1 || k_lo < 0 || k_hi < k_lo || !(sigma > 0) || !G) return RFF_EINVAL;
  return launch_params_rowmajor(seed, sigma, d, k_lo, k_hi - k_lo, G, b, static_cast<cudaStream_t>(stream)) ==
                 cudaSuccess
             ? RFF_OK
             : RFF_ECUDA;
}

rff_status rff_fastfood_params(uint64_t seed, double sigma, int64_t d, int64_t k_lo, int64_t k_hi, float* Vt,
                               float* b, void* stream) {
  if (d < 1 || d > 4096 || k_lo < 0 || k_hi < k_lo || !(sigma > 0) || !Vt || !b) return RFF_EINVAL;
  if (k_hi == k_lo) return RFF_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t nk = k_hi - k_lo;
  const size_t tb = round_up(fastfood_table_bytes(k_hi, fastfood_dim(d)), 256);
  char* base = nullptr;
  if (cudaMallocAsync((void**)&base, tb + (size_t)nk * 4 + 256, st) != cudaSuccess) {
    cudaGetLastError();
    return RFF_ENOMEM;
  }
  int32_t* fos = reinterpret_cast<int32_t*>(base + tb);
  unsigned* mx = reinterpret_cast<unsigned*>(fos + nk);
  std::vector<int32_t> f(nk);
  for (int64_t i = 0; i < nk; ++i) f[i] = (int32_t)(k_lo + i);
  cudaError_t e = cudaMemcpyAsync(fos, f.data(), nk * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_fastfood_params(seed, sigma, d, d, k_hi, nk, fos, Vt, b, mx, base, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);   // f is read by the asynchronous copy
  cudaFreeAsync(base, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return RFF_ECUDA;
  }
  return RFF_OK;
}

rff_status rff_laplace_params(uint64_t seed, double sigma, int64_t d, int64_t k_lo, int64_t k_hi, float* W,
                              void* stream) {
  if (d < 1 || k_lo < 0 || k_hi < k_lo || !(sigma > 0) || !W) return RFF_EINVAL;
  return launch_params_rowmajor(seed, sigma, d, k_lo, k_hi - k_lo, W, nullptr, static_cast<cudaStream_t>(stream),
                                RFF_MAP_LAPLACE) == cudaSuccess
             ? RFF_OK
             : RFF_ECUDA;
}

}  // extern "C"

namespace {
// Z for global features k_lo..k_hi-1 through the solver's own kernels: the random Fourier map
// in FP32 (prec 0) or on the tensor cores (prec 1), or the random Laplace map (map 1, FP32)
rff_status features_impl(const float* X, int64_t n, int64_t d, uint64_t seed, double sigma, int64_t D, int64_t k_lo,
                         int64_t k_hi, int32_t prec, int map, float* Z, void* stream) {
  if (n < 0 || d < 1 || D < 1 || k_lo < 0 || k_hi < k_lo || k_hi > D || !(sigma > 0) || prec < 0 || prec > 1 ||
      (map && prec))
    return RFF_EINVAL;
  if (n == 0 || k_hi == k_lo) return RFF_OK;
  if (!X || !Z) return RFF_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int64_t nf = k_hi - k_lo, dld = round_up(d, 64), np = round_up(n, SLOT), fp = round_up(nf, SLOT);
  const size_t bytes = (size_t)np * dld * 4 + (size_t)fp * dld * 4 + (size_t)fp * 4 + (size_t)np * 4 + (size_t)fp * 4 +
                       (size_t)(np + fp) * dld * 2 * 2 + 64 + 64 + 4096;
  char* base = nullptr;
  if (cudaMallocAsync((void**)&base, bytes, st) != cudaSuccess) {
    cudaGetLastError();
    return RFF_ENOMEM;
  }
  float* X32 = reinterpret_cast<float*>(base);
  float* G32 = X32 + np * dld;
  float* bias = G32 + fp * dld;
  int32_t* rok = reinterpret_cast<int32_t*>(bias + fp);
  int32_t* fok = rok + np;
  __half* Xh = reinterpret_cast<__half*>(fok + fp);
  __half* Xl = Xh + np * dld;
  __half* Gh = Xl + np * dld;
  __half* Gl = Gh + fp * dld;
  int64_t* tabs = reinterpret_cast<int64_t*>(Gl + fp * dld);   // {0, n, 0, nf}
  unsigned* xmaxbits = reinterpret_cast<unsigned*>(tabs + 4);
  std::vector<int32_t> r(np), f(fp);
  const int64_t htab[4] = {0, n, 0, nf};
  for (int64_t i = 0; i < np; ++i) r[i] = i < n ? (int32_t)i : -1;
  for (int64_t i = 0; i < fp; ++i) f[i] = i < nf ? (int32_t)(k_lo + i) : -1;
  cudaError_t e = cudaMemcpyAsync(rok, r.data(), np * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(tabs, htab, sizeof(htab), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(fok, f.data(), fp * 4, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = launch_gather_rows(X, d, d, rok, np, X32, dld, st);
  const int64_t bcol = (prec == RFF_PREC_SPLIT_BF16 && round_up(d + 1, 64) == dld) ? d : -1;
  // the split path scales X and G by powers of two into the FP16 range (largest |x|, |g| <= 2^8)
  float xscale = 1.f;
  const float gscale = g_scale(sigma);
  bool negative = false;
  if (e == cudaSuccess && (prec || map)) {
    unsigned bits[2] = {0, 0};
    int* fflag = reinterpret_cast<int*>(xmaxbits + 1);
    e = cudaMemsetAsync(xmaxbits, 0, 8, st);
    if (e == cudaSuccess) e = launch_finite_check(X, n * d, map ? 2 : 0, fflag, st, xmaxbits);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bits, xmaxbits, 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    float xmax = 0.f;
    memcpy(&xmax, &bits[0], 4);
    xscale = pow2_scale(std::max<double>(xmax, bcol >= 0 ? 1.0 : 0.0));
    negative = map && (bits[1] & 5);
  }
  if (e == cudaSuccess && !negative)
    e = launch_params_slots(seed, sigma, d, dld, fp, fok, G32, prec ? Gh : nullptr, prec ? Gl : nullptr, gscale, bias,
                            bcol, st, map);
  const float scale = (float)(map ? 1.0 / std::sqrt((double)D) : std::sqrt(2.0 / (double)D));
  if (e == cudaSuccess && !negative) {
    if (prec == RFF_PREC_FP32) {
      ZArgs za{X32, dld, G32, dld, (int)dld, bias, scale, rok, fok, 0, n, 0, nf, Z, nf, map};
      e = launch_write_z_simt(za, st);
    } else {
      if (bcol >= 0) e = launch_set_column(X32, dld, np, bcol, 1.f, st);
      if (e == cudaSuccess) e = launch_split_f16(X32, np * dld, xscale, Xh, Xl, st);
      if (e == cudaSuccess) {
        const int64_t zero = 0;
        TcView v{};
        v.Xhi = Xh; v.Xlo = Xl; v.Ghi = Gh; v.Glo = Gl;
        v.bias = bias; v.row_ok = rok; v.feat_ok = fok;
        v.nslots = np; v.fslots = fp; v.dld = dld; v.mpad = 16; v.R = 1; v.C = 1; v.nsplit = 1;
        v.row_slot = &zero; v.row_size = &n; v.col_slot = &zero; v.col_size = &nf;
        v.d_row_slot = tabs; v.d_row_size = tabs + 1; v.d_col_slot = tabs + 2; v.d_col_size = tabs + 3;
        v.scale = scale; v.inv_xg = 1.f / (xscale * gscale); v.bias_in_mma = bcol >= 0 ? 1 : 0; v.st = st;
        e = tc_write_z(v, 0, n, 0, nf, Z, nf);
      }
    }
  }
  // the host vectors above are read by the asynchronous copies: finish before they go
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(base, st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorNotSupported ? RFF_EINVAL : RFF_ECUDA;
  }
  if (negative) return RFF_EINVAL;
  if (prec == RFF_PREC_SPLIT_BF16 && tc_error_word() != 0) return RFF_ETIMEOUT;
  return RFF_OK;
}
}  // namespace

extern "C" {
rff_status rff_features(const float* X, int64_t n, int64_t d, uint64_t seed, double sigma, int64_t D, int64_t k_lo,
                        int64_t k_hi, int32_t prec, float* Z, void* stream) {
  return features_impl(X, n, d, seed, sigma, D, k_lo, k_hi, prec, RFF_MAP_FOURIER, Z, stream);
}

rff_status rff_laplace_features(const float* X, int64_t n, int64_t d, uint64_t seed, double sigma, int64_t D,
                                int64_t k_lo, int64_t k_hi, float* Z, void* stream) {
  return features_impl(X, n, d, seed, sigma, D, k_lo, k_hi, RFF_PREC_FP32, RFF_MAP_LAPLACE, Z, stream);
}

rff_status rff_tensorsketch_features(const float* X, int64_t n, int64_t d, uint64_t seed, double sigma,
                                     double coef0, int32_t degree, int64_t D, int32_t C, float* Z, void* stream) {
  if (!X || !Z || n < 0 || d < 1 || d > (1 << 20) || D < 1 || C < 1 || C > D || C > 65535) return RFF_EINVAL;
  if (degree < 1 || degree > TS_MAX_DEGREE || !(coef0 >= 0) || !std::isfinite(coef0) || !(sigma > 0)) return RFF_EINVAL;
  std::vector<int64_t> start, size;
  partition(D, C, start, size);
  const int64_t smax = size[0];
  if (smax > TS_MAX_BLOCK || tensorsketch_smem_bytes(degree, d, smax) > TS_MAX_SMEM) return RFF_EINVAL;
  if (n == 0) return RFF_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int64_t* dcol = nullptr;
  if (cudaMallocAsync(&dcol, (size_t)C * 16, st) != cudaSuccess) {
    cudaGetLastError();
    return RFF_ENOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(dcol, start.data(), (size_t)C * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dcol + C, size.data(), (size_t)C * 8, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    TsArgs a{};
    a.X = X;
    a.ldx = d;
    a.d = (int)d;
    a.nr = n;
    a.q = degree;
    a.inv_sigma = (float)(1.0 / sigma);
    a.sqrt_c = (float)std::sqrt(coef0);
    a.k0 = (uint32_t)seed;
    a.k1 = (uint32_t)(seed >> 32);
    a.col_slot = dcol;
    a.col_size = dcol + C;
    a.out = Z;
    a.ldo = D;
    a.out_elems = n * D;
    a.D = D;
    e = launch_tensorsketch(a, C, smax, st);
  }
  // the host vectors are read by the copies: pageable memory is staged before they return
  cudaError_t f = cudaFreeAsync(dcol, st);
  if (e == cudaSuccess) e = f;
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorInvalidValue ? RFF_EINVAL : RFF_ECUDA;
  }
  return RFF_OK;
}

rff_status rff_prox_loss(int32_t loss, const float* V, const float* Yv, int64_t n, int32_t m, double t,
                         int32_t newton_iters, float* out, void* stream) {
  if (loss < 0 || loss > 5 || n < 0 || m < 1 || m > 256 || !(t >= 0) || (n > 0 && (!V || !Yv || !out)))
    return RFF_EINVAL;
  if (loss == RFF_LOSS_LOGISTIC && m != 1) return RFF_EINVAL;
  return launch_prox_loss(loss, V, Yv, n, m, m, (float)t, newton_iters > 0 ? newton_iters : 8, out,
                          static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? RFF_OK
             : RFF_ECUDA;
}

rff_status rff_prox_reg(int32_t reg, const float* V, int64_t n, double tau, float* out, void* stream) {
  if (reg < 0 || reg > 1 || n < 0 || !(tau >= 0) || (n > 0 && (!V || !out))) return RFF_EINVAL;
  return launch_prox_reg(reg, V, nullptr, n, (float)tau, out, static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? RFF_OK
             : RFF_ECUDA;
}

rff_status rff_cholesky_f64(double* A, int32_t batch, int32_t s, int32_t* info, void* stream) {
  if (batch < 0 || s < 1 || (batch > 0 && (!A || !info))) return RFF_EINVAL;
  if (batch == 0) return RFF_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const size_t need = factor_scratch_bytes(batch, s);
  void* scr = nullptr;
  if (cudaMallocAsync(&scr, need, st) != cudaSuccess) {
    cudaGetLastError();
    return RFF_ENOMEM;
  }
  std::vector<MatJob> jobs;
  for (int b = 0; b < batch; ++b) jobs.push_back(MatJob{A + (size_t)b * s * s, s, s, nullptr, 0, info + b});
  cudaError_t e = cudaMemsetAsync(info, 0, (size_t)batch * 4, st);
  if (e == cudaSuccess) e = factor_and_invert_f64(jobs, false, scr, st);
  if (e == cudaSuccess) e = launch_zero_strict_upper(A, s, batch, st);
  cudaFreeAsync(scr, st);
  return e == cudaSuccess ? RFF_OK : RFF_ECUDA;
}

}  // extern "C"
