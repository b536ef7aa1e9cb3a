// Internal launcher declarations shared by the translation units of the library.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

namespace rff {

// Arguments of the fused regeneration passes (SIMT and tensor-core versions).
// Row-side arrays are indexed by row slot, feature-side arrays by feature slot.
// TensorSketch features (the polynomial kernel's map): rows [r0, r0 + nr) of X (slot layout,
// ld ldx, first d columns used; row_ok: slot -> row, -1 = padding, or null) for the column
// blocks j = j0 .. j0 + nblocks - 1 (S = col_size[j] features each, at column col_slot[j] - f_base
// of out, scaled by sqrt(S / D)); pad: also write zeros up to the block's slot boundary;
// amax: max |z| (float bits, atomicMax; zero it first), or null; out may be null.
constexpr int TS_MAX_DEGREE = 8;
constexpr int64_t TS_MAX_BLOCK = 8192;          // features per column block
constexpr size_t TS_MAX_SMEM = 200 * 1024;
struct TsArgs {
  const float* X;
  int64_t ldx;
  int d;
  const int32_t* row_ok;
  int64_t r0, nr;
  int q;
  float inv_sigma, sqrt_c;
  uint32_t k0, k1;                              // Philox key
  int j0;                                       // first column block of the launch
  const int64_t* col_slot;                      // device, one per block
  const int64_t* col_size;                      // device
  float* out;
  int64_t ldo, f_base, out_elems;
  int pad;
  int64_t D;
  unsigned* amax;
};
size_t tensorsketch_smem_bytes(int q, int64_t d, int64_t S);
// nblocks column blocks (grid y), smax = the largest of their sizes
cudaError_t launch_tensorsketch(const TsArgs& a, int nblocks, int64_t smax, cudaStream_t st);

// read and clear the bounds-check record of each checked translation unit (zeros in the
// ordinary build)
cudaError_t check_collect_elementwise(CheckHit* h);
cudaError_t check_collect_qgemm(CheckHit* h);
cudaError_t check_collect_regen_simt(CheckHit* h);
cudaError_t check_collect_tc(CheckHit* h);
cudaError_t check_collect_sketch(CheckHit* h);
cudaError_t check_collect_ozaki(CheckHit* h);

struct PassArgs {
  const float* X;        // data rows (slots) x K, float32            (SIMT)
  int64_t ldx;
  const float* Gt;       // feature rows (slots) x K, float32         (SIMT)
  int64_t ldg;
  int K;                 // padded input dimension (multiple of 64)
  const float* bias;     // b per feature slot
  float scale;           // sqrt(2/D)
  const int32_t* row_ok; // row_of_slot table (-1 = padding), or null = all valid
  const int32_t* feat_ok;
  const int64_t* row_slot;  // R entries: first slot of each row block
  const int64_t* row_size;  // R entries: n_i
  int R;
  const int64_t* col_slot;  // C entries
  const int64_t* col_size;  // C entries: s_j
  int C;
  const float* M;           // chain operand (SIMT: rows x m_pad float32)
  int64_t m_block_stride;   // elements between the chain operands of successive blocks
  float* out;
  int64_t out_block_stride; // elements between outputs of successive blocks
  int mpad;
  int nsplit;               // pass 1: row splits per row block
  int per_block;            // pass 2: write per column block (1) or once (0)
  const uint8_t* bmask;     // device, R x C: active blocks of a stochastic iteration, or null
  int map;                  // feature map: 1 random Laplace (exp(-T)); else cos(T + b) (Fourier, Fastfood)
  // extents, tested by the bounds-checked build: rows of X and of Gt, elements of M and of out
  int64_t x_rows, g_rows, m_elems, out_elems;
};

struct ZArgs {
  const float* X;
  int64_t ldx;
  const float* Gt;
  int64_t ldg;
  int K;
  const float* bias;
  float scale;
  const int32_t* row_ok;
  const int32_t* feat_ok;
  int64_t r0, nr, f0, nf;   // row slots [r0, r0+nr), feature slots [f0, f0+nf)
  float* out;
  int64_t ldo;
  int map;                  // as PassArgs::map
};

// philox.cu
cudaError_t launch_philox_raw(const uint32_t* ctr, uint64_t seed, int64_t n, uint32_t* out, cudaStream_t st);
// Fastfood (feature map 2): d' = the smallest power of two >= d (at most 4096)
inline int fastfood_dim(int64_t d) {
  int p = 1;
  while (p < d) p *= 2;
  return p;
}
size_t fastfood_table_bytes(int64_t D, int dp);
// V rows (feature-major, ld columns, zero beyond d) for the features of the slots, b, and
// max |V| into maxbits (float bits, atomicMax; zero it first); tables: fastfood_table_bytes
cudaError_t launch_fastfood_params(uint64_t seed, double sigma, int64_t d, int64_t ld, int64_t D, int64_t nslots,
                                   const int32_t* feat_of_slot, float* Gt, float* bias, unsigned* maxbits,
                                   void* tables, cudaStream_t st);
// hi/lo FP16 split of Gt * gscale (n x ld) with b * gscale in column bias_col (if >= 0)
cudaError_t launch_split_g_bias(const float* Gt, int64_t n, int64_t ld, const float* bias, int64_t bias_col,
                                float gscale, __half* hi, __half* lo, cudaStream_t st);
// Active blocks of a stochastic iteration: mask[b] = 1 iff (w >> 8) < thr, w the first
// word of Philox4x32-10 at counter (b, k, 2, 0) under seed, k = *ctr; then *ctr = k + 1
cudaError_t launch_block_mask(uint64_t seed, uint32_t thr, int nblocks, int64_t* ctr, uint8_t* mask,
                              cudaStream_t st);
// map 0: G (random Fourier) and b; map 1: the random Laplace map's W, b = 0
cudaError_t launch_params_rowmajor(uint64_t seed, double sigma, int64_t d, int64_t k_lo, int64_t nk, float* G,
                                   float* b, cudaStream_t st, int map = 0);
// Ghi/Glo: the FP16 split of G * gscale; bias_col >= 0: they carry b * gscale in that
// column (inputs then carry ones there)
cudaError_t launch_params_slots(uint64_t seed, double sigma, int64_t d, int64_t ld, int64_t nslots,
                                const int32_t* feat_of_slot, float* Gt, __half* Ghi, __half* Glo, float gscale,
                                float* bias, int64_t bias_col, cudaStream_t st, int map = 0);

// regen_simt.cu
cudaError_t launch_pass1_simt(const PassArgs& p, int64_t nfeat_slots, cudaStream_t st);
cudaError_t launch_pass2_simt(const PassArgs& p, int64_t nrow_slots, cudaStream_t st);
cudaError_t launch_write_z_simt(const ZArgs& p, cudaStream_t st);

// dense.cu: batched dense linear algebra (SIMT)
struct GemmDesc {          // D = alpha * op(A) op(B) + beta * Cm, row-major
  const void* A;
  const void* B;
  const void* Cm;
  void* D;
  int M, N, K;
  int64_t lda, ldb, ldc, ldd;
};
// f32 iteration GEMM, NN only, desc array on the device; bmask: descriptor b runs only if
// bmask[b] != 0 (null: all run)
cudaError_t launch_gemm_f32_nn(const GemmDesc* descs_dev, int nbatch, int maxM, int maxN, float alpha, float beta,
                               cudaStream_t st, const uint8_t* bmask = nullptr);
// the same for one product whose descriptor is passed by value (no device copy of it)
cudaError_t launch_gemm_f32_nn_one(const GemmDesc& g, float alpha, float beta, cudaStream_t st);
// f64 with runtime transposes; double_float: FP64 in and out, double-float arithmetic inside
cudaError_t launch_gemm_f64(const GemmDesc* descs_dev, int nbatch, int maxM, int maxN, int transA, int transB,
                            double alpha, double beta, int lower_only, cudaStream_t st, bool double_float = false);
// double-float GEMM whose A and B are float pairs (hi, lo) and whose C and D are FP64
cudaError_t launch_gemm_df_pairs(const GemmDesc* descs_dev, int nbatch, int maxM, int maxN, int transA, int transB,
                                 double alpha, double beta, int lower_only, cudaStream_t st);
// D (float pairs, ld ldd) = A (FP64, ld lda), M x N per descriptor
cudaError_t launch_to_pairs(const GemmDesc* descs_dev, int nbatch, int maxM, int maxN, cudaStream_t st);
// Gram: D(f64) = beta*D + Z^T Z over rows, Z float32 (n x s, ld), FP32 products, FP64 accumulation
cudaError_t launch_gram_f32_to_f64(const float* Z, int64_t ldz, int64_t n, int64_t s, double* H, int64_t ldh,
                                   cudaStream_t st);
struct DiagJob {   // one matrix of a batched factorisation
  double* A;       // matrix base (s x s, leading dimension ld)
  int64_t ld;
  int s;
  double* inv;     // 64 x 64: inverse of the current diagonal factor
  int32_t* info;   // first failing column + 1, or untouched
};
cudaError_t launch_potrf_diag(const DiagJob* jobs_dev, int njobs, int kcol, cudaStream_t st);
cudaError_t launch_add_identity_and_mirror(double* H, int64_t ldh, int64_t s, cudaStream_t st);
cudaError_t launch_zero_strict_upper(double* A, int64_t s, int nbatch, cudaStream_t st);
struct MatJob {    // host description of one matrix to factor (and invert)
  double* A;       // in: SPD matrix; out: lower Cholesky factor
  int64_t ld;
  int s;
  double* Q;       // out: inverse (must hold the identity on entry), or null
  int64_t ldq;
  int32_t* info;   // device int32, zero on entry
};
size_t factor_scratch_bytes(int njobs, int smax);
// blocked Cholesky (and inverse); double_float selects the double-float GEMM for the block
// updates under RFF_FACTOR=df (the 64 x 64 diagonal factorisations stay FP64); oz_bits: the
// leading bits of every update operand the tensor-core updates keep (48 or 40)
cudaError_t factor_and_invert_f64(const std::vector<MatJob>& jobs, bool invert, void* dev_scratch, cudaStream_t st,
                                  bool double_float = false, int oz_bits = 48);
cudaError_t launch_mirror_lower(double* Q, int64_t ld, int64_t s, cudaStream_t st);

// ozaki.cu: the same factorisation with the block updates on the tensor cores (error-free
// slices of the FP64 operands); factor_and_invert_f64 calls it unless RFF_FACTOR=df
size_t oz_factor_scratch_bytes(int njobs, int smax);
cudaError_t factor_and_invert_oz(const std::vector<MatJob>& jobs, bool invert, void* dev_scratch, cudaStream_t st,
                                 int bits);

// elementwise.cu
// dst[p][c] = src[map[p] * lds + c] (c < w), zero for c >= w or map[p] < 0; map null = identity
cudaError_t launch_gather_rows(const float* src, int64_t lds, int64_t w, const int32_t* map, int64_t nrows,
                               float* dst, int64_t ld, cudaStream_t st);
cudaError_t launch_set_column(float* X, int64_t ld, int64_t rows, int64_t col, float v, cudaStream_t st);
// CSR structure check: *flag |= 1 unless indptr[0] = 0, indptr[n] = nnz, indptr non-decreasing
// and every column index of a well-formed row in [0, d) (indices are read only for such rows)
cudaError_t launch_csr_check(const int64_t* indptr, const int32_t* indices, int64_t n, int64_t d, int64_t nnz,
                             int* flag, cudaStream_t st);
// dst[p][c] = sum of the values of row map[p] in column c (CSR; map[p] < 0: zero row), ld >= d
cudaError_t launch_scatter_csr(const int64_t* indptr, const int32_t* indices, const float* values,
                               const int32_t* map, int64_t nrows, float* dst, int64_t ld, cudaStream_t st);
cudaError_t launch_split_bf16(const float* src, int64_t n, __nv_bfloat16* hi, __nv_bfloat16* lo, cudaStream_t st);
// hi/lo FP16 split of src * scale (scale a power of two)
cudaError_t launch_split_f16(const float* src, int64_t n, float scale, __half* hi, __half* lo, cudaStream_t st);
cudaError_t launch_prox_loss(int loss, const float* V, const float* Y, int64_t n, int m, int64_t ld, float t,
                             int newton, float* out, cudaStream_t st);
cudaError_t launch_prox_reg(int reg, const float* V, const float* mu, int64_t n, float tau, float* out,
                            cudaStream_t st, const float* tau_col = nullptr, int ncol = 1);
// words of the device array of maxima (float bits) that scale the FP16 splits
constexpr int AMAX_V = 0, AMAX_W = 1, AMAX_WB = 2, AMAX_FLAG = 3, AMAX_OP = 4, AMAX_O = 5, AMAX_NU = 6,
              AMAX_O_NEXT = 7, AMAX_NU_NEXT = 8, AMAX_OINC = 9, AMAX_WORDS = 16;

struct RowEpiArgs {
  const float* Op;      // C x slots x mpad
  float* O;             // slots x mpad (in: O^k, out: O^{k+1} = prox(Obar - nu))
  float* Obar;
  float* nu;
  const float* Y;
  // U_i = Delta_i/(C+1) + nu_i (Obar_ij + nu_i = O'_ij + U_i), one operand for every column
  // block: into V32 (slots x mpad, FP32) when given, else as the tensor-core operand below
  float* V32;
  // U^T written as its scaled FP16 hi/lo split (mpad x slots), the scale from an upper bound
  // of |U| built from the maxima in amax (float bits): amax[AMAX_OP] =
  // max |O'|, amax[AMAX_O] / amax[AMAX_NU] = max |O|, |nu| of this kernel's inputs; the kernel
  // stores the bound in amax[AMAX_V] and reduces max |O|, |nu| of its outputs into
  // amax[AMAX_O_NEXT], amax[AMAX_NU_NEXT]
  __half* VThi;
  __half* VTlo;
  unsigned* amax;
  const int32_t* row_ok;
  int64_t nslots;
  int C, m, mpad, loss, newton;
  float t_loss;
};
cudaError_t launch_row_epilogue(const RowEpiArgs& a, cudaStream_t st);
// rhs_ij = Wbar_j - mu'_ij (- W'_ij when What is given: the incremental projection) + sum
// of the R partials
cudaError_t launch_rhs(const float* Wbar, const float* muij, const float* Rpart, int nsplit, int R, int64_t nfe,
                       float* rhs, cudaStream_t st, const int32_t* feat_ok = nullptr, int mpad = 0,
                       const float* What = nullptr);
// W' = rhs - sum of the nsplit partials, padding feature slots zero (outer form); with
// bmask (R x C, col_slot: first slot of each of the C column blocks) only active blocks
// W'_ij (+)= rhs_ij - sum of the R partials (accumulate: added to W'_ij, the incremental
// projection); an inactive block of a stochastic iteration keeps its W'_ij
cudaError_t launch_sub_partials(const float* rhs, const float* Rpart, int nsplit, int R, int64_t nfe,
                                const int32_t* feat_ok, int mpad, float* What, cudaStream_t st,
                                const uint8_t* bmask = nullptr, const int64_t* col_slot = nullptr, int C = 1,
                                int accumulate = 0);
// Outer form of the projection (C x slots x mpad blocks, U_i = block 0 of U):
//   e_ij = O'_ij + U_i - u_ij (into u, in place);
cudaError_t launch_outer_residual(float* u, const float* Op, const float* U, int64_t nslots, int mpad, int C,
                                  cudaStream_t st);
//   O'_ij += U_i + y_ij for the active blocks (bmask per row block i, column block j; null: all)
cudaError_t launch_outer_update(float* Op, const float* U, const float* y, int64_t nslots, int mpad, int R, int C,
                                const int64_t* d_row_slot, const uint8_t* bmask, cudaStream_t st);
// dst[c][r] = src[r][c]
cudaError_t launch_transpose_f32(const float* src, int64_t rows, int64_t cols, float* dst, int64_t dld,
                                 cudaStream_t st);
cudaError_t launch_avg_dual(const float* W, const float* What, int R, int64_t nfe, float* Wbar, float* mu,
                            float* muij, cudaStream_t st);
// hi/lo FP16 split of src^T scaled by f16_scale(*amax) (amax non-null) or by scale
cudaError_t launch_transpose_split_f16(const float* src, int64_t rows, int cols, int nbatch, int64_t src_batch_stride,
                                       __half* hi, __half* lo, int64_t dst_ld, int64_t dst_batch_stride, float scale,
                                       const unsigned* amax, cudaStream_t st);
cudaError_t launch_transpose_split(const float* src, int64_t rows, int cols, int nbatch, int64_t src_batch_stride,
                                   __nv_bfloat16* hi, __nv_bfloat16* lo, int64_t dst_ld, int64_t dst_batch_stride,
                                   cudaStream_t st);
cudaError_t launch_sqdiff_partials(const float* a, const float* b, int64_t n, double* partials, int nblocks,
                                   cudaStream_t st);
cudaError_t launch_loss_partials(int loss, const float* Y, const float* S, const int32_t* row_ok, int64_t nslots,
                                 int m, int mpad, double* partials, int nblocks, cudaStream_t st);
cudaError_t launch_reg_partials(int reg, const float* W, int64_t n, double* partials, int nblocks, cudaStream_t st,
                                const float* w = nullptr, int ncol = 1);
cudaError_t launch_convert_f64_f32(const double* src, float* dst, int64_t n, cudaStream_t st);
// flag |= 1 for NaN/Inf; pm1 = 1: |= 2 for a value other than +-1; pm1 = 2: |= 4 for a negative value
cudaError_t launch_finite_check(const float* x, int64_t n, int pm1, int* flag, cudaStream_t st,
                                unsigned* maxbits = nullptr);
cudaError_t launch_set_diag(double* A, int64_t ld, int64_t s, double v, cudaStream_t st);
// H (FP64, ld ldh) += the sum over nchunk partial tiles (FP32, 128 x 256 each, chunk-major)
// of the 128 x 256 tiles listed in tiles (first row, first column); entries at or below the
// diagonal of the s x s matrix only; the chunks (at most 8) are added in order in FP64
cudaError_t launch_gram_reduce(const float* P, int nchunk, int ntiles, const int2* tiles, int64_t s, double* H,
                               int64_t ldh, cudaStream_t st);
// labels of q rows of scores (ld columns, m used): m = 1: +1 if score >= 0 else -1;
// m > 1: the index of the largest score, the lowest index among equal ones
cudaError_t launch_argmax_rows(const float* scores, int64_t q, int m, int64_t ld, int32_t* labels, cudaStream_t st);

}  // namespace rff
