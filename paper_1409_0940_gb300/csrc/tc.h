// Tensor-core (tcgen05) regeneration passes of the split-BF16 path.
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace rff {

// What the tensor-core passes need from a solver handle.  Host arrays (row_slot,
// ...) describe the block grid; device arrays hold the data in slot layout.
struct TcView {
  const __half *Xhi, *Xlo;          // nslots x dld, FP16 split of X * xscale
  const __half *Ghi, *Glo;          // fslots x dld, FP16 split of G * gscale
  const __half *VThi, *VTlo;        // C x mpad x nslots (pass-1 chain operand), FP16 split of V^T
  const unsigned* v_amax;           // max |V| (float bits): the scale of that split
  const float* bias;                // fslots
  const int32_t *row_ok, *feat_ok;  // slot tables, -1 = padding
  int64_t nslots, fslots, dld, mpad;
  int R, C, nsplit;
  const int64_t *row_slot, *row_size, *col_slot, *col_size;  // host
  const int64_t *d_row_slot, *d_row_size, *d_col_slot, *d_col_size;  // device copies
  float scale;
  float inv_xg;                     // 1 / (xscale gscale): the X.G accumulator times this is X G
  int bias_in_mma;                  // 1: b is column d of G and X carries ones there
  int kc;                           // ring K chunk (64 or 32; 0 = library default)
  int zt;                           // 1: Z tile in tensor memory, 0: in shared memory,
                                    // 2: in tensor memory with acc1 double-buffered (m_pad <= 128),
                                    // 3: the wide geometry (N = 256 X.G, Z hi in TMEM and lo in
                                    //    shared memory; m_pad <= 192; one CTA)
  int cg;                           // 2: CTA pairs (tcgen05.mma.cta_group::2, Z in TMEM), else one CTA
  const uint8_t* bmask;             // device, R x C: active blocks of a stochastic iteration, or null
  int v_shared;                     // pass 1: one chained operand for every column block (rows 0..m_pad)
  int64_t row_tiles;                // pass 2: 128-row tiles taken from the first (0 = all of them)
  cudaStream_t st;
};

// Z for row slots [r0, r0+nr) x feature slots [f0, f0+nf) into out (ld ldo), float32.
cudaError_t tc_write_z(const TcView& v, int64_t r0, int64_t nr, int64_t f0, int64_t nf, float* out, int64_t ldo);
// The same window as Z^T split into FP16 hi/lo of scale * Z: hi[f][r], lo[f][r] (ld ldt) for
// f < nf, r < nr; the elements outside the window are left as they are.
cudaError_t tc_write_zt_split(const TcView& v, int64_t r0, int64_t nr, int64_t f0, int64_t nf, float scale,
                              __half* hi, __half* lo, int64_t ldt);
// Pass 1: R-partials [nsplit][R][fslots][mpad] = Z_ij^T V_ij.
cudaError_t tc_pass1(const TcView& v, float* Rpart);
// Pass 2: out[j][slots][mpad] = Z_ij M_i (per_block) or out[slots][mpad] = sum_j Z_ij M (predict);
// M given transposed and split: [R][mpad][fslots] hi/lo FP16 of M scaled by f16_scale(*m_amax),
// m_block_stride elements apart.
cudaError_t tc_pass2(const TcView& v, const __half* Mhi, const __half* Mlo, int64_t m_block_stride,
                     float* out, int per_block, const unsigned* m_amax, unsigned* out_amax = nullptr);
// One launch of pass 1 (which = 1) or pass 2 (which = 2) for n solves (a model-selection
// sweep, n <= 64): per solve its view and the arguments its own tc_pass1 / tc_pass2 call would
// take (outs = Rpart or O'; Mhi, Mlo, m_amax, out_amax for pass 2 only, else null).  The solves'
// arguments go to device memory that the object owns (a synchronous copy: create it outside
// stream capture); every launch then reads them, so the object must outlive the launches.
// Every solve runs the default geometry (K chunk 64, Z tile in TMEM, one CTA per MMA).
struct TcMulti;
cudaError_t tc_multi_create(const TcView* views, int n, int which, float* const* outs, const __half* const* Mhi,
                            const __half* const* Mlo, const unsigned* const* m_amax, unsigned* const* out_amax,
                            TcMulti** out);
cudaError_t tc_multi_launch(const TcMulti* t, cudaStream_t st);
void tc_multi_destroy(TcMulti* t);
// Scores for a query block (nrows slot-padded rows of split X) against M (mpad x fslots hi/lo).
// Error word of the tensor-core kernels (bounded waits that gave up); reads and clears it.
// Synchronises the device.  0 = no error.
int tc_error_word();
cudaError_t tc_predict(const TcView& v, const __half* Xh, const __half* Xl, int64_t nrows,
                       const __half* Mhi, const __half* Mlo, const unsigned* m_amax, float* out);


// Split streaming GEMM on the tensor cores, one CTA per job:
//   out[job.out + r*mpad + c] = out_scale / s_B sum_k A[job.a_row + r][job.a_k0 + k] B[job.b_row + c][job.b_k0 + k]
// for r < 128, c < mpad, k < 32*job.nk, with A and B split into three BF16 terms (six
// products; f16 = 0) or into two scaled FP16 terms (three products; f16 = 1).  s_B is
// f16_scale(*b_amax) when b_amax is given (the scale B's split was written with), else 1;
// amax, when given, receives max |out| (atomicMax of float bits).  A is a_rows x a_cols
// (row-major), B b_rows x b_cols; every job's K range and rows lie inside them.
struct SgJob {
  int32_t a_row, a_k0, b_row, b_k0, nk;
  int32_t blk;   // block i C + j the job belongs to (skipped when bmask[blk] == 0)
  int64_t out;
};
struct SgView {
  const void* A[3];
  int64_t a_rows, a_cols;
  const void* B[3];
  int64_t b_rows, b_cols;
  int na, nb, f16;
  const SgJob* jobs;                   // device
  int njobs, mpad;
  float* out;
  int64_t out_elems;                   // elements of out (every job's 128 x mpad tile lies inside)
  float out_scale;
  const unsigned* b_amax;
  unsigned* amax;
  size_t smem_budget;                  // ring bytes per CTA (0 = the largest; smaller lets 2 CTAs share an SM)
  int two_acc;                         // 1: hi.hi products in their own TMEM accumulator (twice the columns)
  const uint8_t* bmask;                // device, R x C: a job of an inactive block does nothing; or null
  int accumulate;                      // 1: out += the product (amax of the sum)
  int persistent;                      // 1: CTAs that stay resident and take jobs in turn
  int kc;                              // K per ring stage: 32 (0 = default) or 64 (128-byte swizzle; an
                                       // odd nk then reads 32 more K columns, zero in A or past its end)
  cudaStream_t st;
};
cudaError_t split_gemm(const SgView& v);
// Q (s x s, row-major float64) split three ways into rows [qrow, qrow+s) of q1..q3 (ld ldq).
cudaError_t launch_split3_q(const double* Q, int s, int64_t ldq, int64_t qrow, __nv_bfloat16* q1,
                            __nv_bfloat16* q2, __nv_bfloat16* q3, cudaStream_t st);
// rhs_ij = Wbar_j - mu'_ij (- W'_ij when What is given) + sum of the R partials, split three
// ways and transposed to [R][mpad][fslots]; padding feature slots are written as zero.
cudaError_t launch_rhs_split3T(const float* Wbar, const float* muij, const float* Rpart, int nsplit, int R,
                               int64_t fslots, int mpad, const int32_t* feat_ok, __nv_bfloat16* r1,
                               __nv_bfloat16* r2, __nv_bfloat16* r3, cudaStream_t st, const float* What = nullptr);

// helpers shared by the tensor-core kernels
cudaError_t tc_make_map_bf16(CUtensorMap* m, const void* ptr, int64_t cols, int64_t rows, int64_t ld, int box_rows,
                             int kc);
int* tc_error_ptr();
// launch a probe whose bounded wait on a barrier nothing arrives on runs out after `cycles`
cudaError_t tc_wait_probe(long long cycles, cudaStream_t st);

}  // namespace rff
