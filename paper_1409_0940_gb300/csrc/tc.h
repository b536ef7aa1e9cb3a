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
  const __nv_bfloat16 *Xhi, *Xlo;   // nslots x dld
  const __nv_bfloat16 *Ghi, *Glo;   // fslots x dld
  const __nv_bfloat16 *VThi, *VTlo; // C x mpad x nslots (pass-1 chain operand)
  const float* bias;                // fslots
  const int32_t *row_ok, *feat_ok;  // slot tables, -1 = padding
  int64_t nslots, fslots, dld, mpad;
  int R, C, nsplit;
  const int64_t *row_slot, *row_size, *col_slot, *col_size;  // host
  const int64_t *d_row_slot, *d_row_size, *d_col_slot, *d_col_size;  // device copies
  float scale;
  int bias_in_mma;                  // 1: b is column d of G and X carries ones there
  int kc;                           // ring K chunk (64 or 32; 0 = library default)
  cudaStream_t st;
};

// Z for row slots [r0, r0+nr) x feature slots [f0, f0+nf) into out (ld ldo), float32.
cudaError_t tc_write_z(const TcView& v, int64_t r0, int64_t nr, int64_t f0, int64_t nf, float* out, int64_t ldo);
// Pass 1: R-partials [nsplit][R][fslots][mpad] = Z_ij^T V_ij.
cudaError_t tc_pass1(const TcView& v, float* Rpart);
// Pass 2: out[j][slots][mpad] = Z_ij M_i (per_block) or out[slots][mpad] = sum_j Z_ij M (predict);
// M given transposed and split: [R][mpad][fslots] hi/lo, m_block_stride elements apart.
cudaError_t tc_pass2(const TcView& v, const __nv_bfloat16* Mhi, const __nv_bfloat16* Mlo, int64_t m_block_stride,
                     float* out, int per_block);
// Scores for a query block (nrows slot-padded rows of split X) against M (mpad x fslots hi/lo).
// Error word of the tensor-core kernels (bounded waits that gave up); reads and clears it.
// Synchronises the device.  0 = no error.
int tc_error_word();
cudaError_t tc_predict(const TcView& v, const __nv_bfloat16* Xh, const __nv_bfloat16* Xl, int64_t nrows,
                       const __nv_bfloat16* Mhi, const __nv_bfloat16* Mlo, float* out);


// Cached projection of the split path, eq. (gpWij): for every block (i, j)
// out[i*fslots + slot_j + r][c] = sum_k Q_ij[r][k] rhs_ij[k][c], with Q_ij and rhs split
// three ways into BF16 and six tensor-core products accumulated in FP32.  The result
// is also written transposed and split two ways (WThi/WTlo, [R][mpad][fslots]) for pass 2.
struct QgemmView {
  const __nv_bfloat16 *Q1, *Q2, *Q3;   // q_rows x ldq, block b's rows from tab[5b]
  int64_t q_rows, ldq;
  const __nv_bfloat16 *R1, *R2, *R3;   // rhs transposed: [R*mpad][fslots]
  int64_t r_rows, r_cols;
  const int* tab;                      // device, per block: Q row, s_j, i*mpad, slot_j, i*fslots + slot_j
  int nblocks, max_s, mpad;
  float* out;                          // [R*fslots][mpad]
  __nv_bfloat16 *WThi, *WTlo;          // [R*mpad][fslots]
  int64_t fslots;
  cudaStream_t st;
};
cudaError_t tc_qgemm(const QgemmView& v);
// Q (s x s, row-major float64) split three ways into rows [qrow, qrow+s) of q1..q3 (ld ldq).
cudaError_t launch_split3_q(const double* Q, int s, int64_t ldq, int64_t qrow, __nv_bfloat16* q1,
                            __nv_bfloat16* q2, __nv_bfloat16* q3, cudaStream_t st);
// rhs_ij = Wbar_j - mu'_ij + sum of the R partials, split three ways and transposed
// to [R][mpad][fslots]; padding feature slots are written as zero.
cudaError_t launch_rhs_split3T(const float* Wbar, const float* muij, const float* Rpart, int nsplit, int R,
                               int64_t fslots, int mpad, const int32_t* feat_ok, __nv_bfloat16* r1,
                               __nv_bfloat16* r2, __nv_bfloat16* r3, cudaStream_t st);

// helpers shared by the tensor-core kernels
cudaError_t tc_make_map_bf16(CUtensorMap* m, const void* ptr, int64_t cols, int64_t rows, int64_t ld, int box_rows,
                             int kc);
int* tc_error_ptr();

}  // namespace rff
