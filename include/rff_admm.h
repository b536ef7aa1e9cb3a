/*
 * rff_admm.h -- C ABI of a GB300 (sm_103a) solver for kernel machines trained by
 * block-splitting ADMM over an implicit random-Fourier-feature matrix.
 *
 * Method: Sindhwani & Avron, "High-performance Kernel Machines with Implicit
 * Distributed Optimization and Randomization" (arXiv:1409.0940).
 *
 *   minimise  sum_i V(y_i, W^T z(x_i)) + n lambda r(W)               Sec. 1 eq. (basicproblem),
 *                                                                    Sec. 2.2 eq. (problem_linear)
 *   z(x) = sqrt(2/D) cos(G^T x + b),  G ~ N(0, sigma^-2), b ~ U[0, pi)   Sec. 4
 *
 * The feature matrix Z (n x D) is split into R row blocks and C column blocks
 * (Sec. 3, the R x C partition) and is never stored: every iteration regenerates
 * each block Z_ij tile by tile on the GPU (the transform T[X_i, j] of Sec. 3),
 * applies it to a right-hand side (Z_ij^T v and Z_ij w), and solves the graph
 * projection of eq. (gp) with the cached factor of eq. (cache).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * - Every call returns an rff_status; none aborts, traps or leaves the device
 *   unusable.  On failure the handle keeps its previous state and
 *   rff_admm_last_error() describes the failure.
 * - Matrices are row-major, float32, densely packed (leading dimension = number
 *   of columns) unless stated otherwise.
 * - "is_device_ptr" = 1 means the pointer is CUDA device memory readable from the
 *   handle's stream; 0 means ordinary host memory.  The library copies inputs;
 *   the caller keeps ownership of everything it passes in.
 * - All work is issued on the stream given to rff_admm_create (NULL = a stream
 *   the handle creates).  Calls that return host data synchronise that stream.
 * - The handle owns all device memory it allocates; rff_admm_destroy frees it.
 * - A handle is not thread-safe: one host thread at a time.
 */
#ifndef RFF_ADMM_H
#define RFF_ADMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RFF_OK = 0,
  RFF_EINVAL = 1,    /* invalid argument, size, NaN/Inf input, or call out of order */
  RFF_ENOMEM = 2,    /* device memory budget exceeded; checked before allocating    */
  RFF_ECUDA = 3,     /* a CUDA runtime call failed                                  */
  RFF_ETIMEOUT = 4,  /* a device-side bounded wait gave up                          */
  RFF_ENOTREADY = 5, /* no data set, or no solve yet                                */
  RFF_ENUMERIC = 6   /* a factorisation met a non-positive pivot                    */
} rff_status;

/* Losses V(y, o), used only through their proximal operators (Sec. 3 "Modularity"). */
typedef enum {
  RFF_LOSS_SQUARED = 0,    /* |y - o|^2, real targets                                  */
  RFF_LOSS_HINGE = 1,      /* m = 1: max(0, 1 - y o); m > 1: one-vs-rest, +-1 targets   */
  RFF_LOSS_LOGISTIC = 2,   /* m = 1: log(1 + exp(-y o)), y = +-1                       */
  RFF_LOSS_MULTINOMIAL = 3 /* log sum_k exp(o_k) - o_c, c = argmax_k y_k               */
} rff_loss;

/* Regularisers r(W), separable over column blocks (Sec. 3, r = sum_j r_j(W_j)). */
typedef enum {
  RFF_REG_L2SQ = 0, /* |W|_F^2 */
  RFF_REG_L1 = 1    /* sum |W_kl| */
} rff_reg;

/* How Z_ij is regenerated and applied. */
typedef enum {
  RFF_PREC_FP32 = 0,      /* X.G, cos and both chained products in FP32 on the SIMT pipes  */
  RFF_PREC_SPLIT_BF16 = 1 /* X.G as three BF16 tensor-core products (hi.hi + hi.lo + lo.hi),
                             FP32 accumulate in TMEM, FP32 cos, chained products again as
                             three BF16 products of the hi/lo split of both operands       */
} rff_precision;

/* Scaling of rho (the paper never fixes it).  RFF_RHO_SUM: rho is the penalty of the
 * objective sum_i V + n lambda r, so the loss prox step is 1/rho and the regulariser
 * step n lambda / rho.  RFF_RHO_MEAN: rho as in Sec. 3 with l_i carrying 1/n, i.e. loss
 * step 1/(n rho), regulariser step lambda/rho.  The two are one method with
 * rho_mean = rho_sum / n. */
typedef enum { RFF_RHO_SUM = 0, RFF_RHO_MEAN = 1 } rff_rho_scale;

typedef struct {
  int32_t loss;      /* rff_loss                                                     */
  int32_t reg;       /* rff_reg                                                      */
  double lambda;     /* regularisation weight lambda > 0 (Sec. 1)                     */
  double sigma;      /* Gaussian kernel bandwidth, k = exp(-|x-x'|^2 / (2 sigma^2))  */
  double rho;        /* ADMM penalty (Sec. 2.3), see rff_rho_scale                    */
  int64_t D;         /* number of random features s = D >= 1                           */
  int32_t R;         /* row blocks (Sec. 3), 1 <= R <= n                               */
  int32_t C;         /* column blocks (Sec. 3), 1 <= C <= D                            */
  uint64_t seed;     /* Philox4x32-10 key: G and b depend on (seed, global feature)  */
  int32_t prec;      /* rff_precision                                                */
  int32_t m;         /* outputs per example, 1 <= m <= 256                            */
  int32_t rho_scale; /* rff_rho_scale                                                */
  int32_t newton_iters; /* Newton steps of the logistic / multinomial prox (0 = 8) */
} rff_admm_params;

typedef struct {
  int32_t iters_done;   /* total iterations since set_data / set_state                  */
  double primal_res;    /* |(O - Obar, W - Wbar, {W'_ij - Wbar_j})|_F after the last one  */
  double dual_res;      /* rho |(Wbar^k - Wbar^{k-1}, Obar^k - Obar^{k-1})|_F             */
  double objective;     /* sum_i V(y_i, (Z Wbar)_i) + n lambda r(Wbar)                   */
  double ms_setup;      /* Philox, split, Gram and factor time of this call (0 if cached) */
  double ms_iterations; /* device time of the iterations of this call                    */
} rff_admm_stats;

typedef struct rff_admm_s* rff_admm_t;

/* Create a solver handle.  params: see rff_admm_params; copied.  stream: a
 * cudaStream_t or NULL.  *out receives the handle.  Errors: RFF_EINVAL for
 * out-of-range parameters (lambda <= 0, sigma <= 0, rho <= 0, D < 1, R < 1,
 * C < 1, C > D, m outside [1, 256], unknown enums, logistic loss with m != 1,
 * C > 64 with RFF_PREC_SPLIT_BF16),
 * RFF_ECUDA if no device is usable. */
rff_status rff_admm_create(const rff_admm_params* params, void* stream, rff_admm_t* out);

/* Attach the training set (Sec. 3: X_i, Y_i row blocks).  X: n x d, Y: n x m,
 * row-major float32; copied, the caller keeps ownership.  Resets the ADMM state
 * and drops any cached factors.  Errors: RFF_EINVAL for n < R, d < 1, NaN/Inf
 * in X or Y, targets outside {-1, +1} for the hinge and logistic losses;
 * RFF_ENOMEM when the device cannot hold the working set (checked first). */
rff_status rff_admm_set_data(rff_admm_t h, const float* X, const float* Y, int64_t n, int64_t d,
                             int is_device_ptr);

/* Run `iters` further ADMM iterations (the update equations of Sec. 3 around
 * eq. (gp), all variables starting at zero after set_data).  The first call
 * after set_data first draws G and b (Sec. 4), forms each block's Gram matrix
 * I + Z_ij^T Z_ij and caches its inverse from an FP64 Cholesky factorisation
 * (eq. (cache)); later calls reuse the cache.  stats may be NULL; when given,
 * residuals and objective are computed after the last iteration (one extra
 * pass over the data).  Errors: RFF_ENOTREADY without data, RFF_ENUMERIC if a
 * Gram matrix is not positive definite, RFF_ECUDA. */
rff_status rff_admm_solve(rff_admm_t h, int32_t iters, rff_admm_stats* stats);

/* Scores f(x) = Wbar^T z(x) for q query rows (Sec. 2.2, H_{k,l}; prediction in
 * Sec. 5).  Xq: q x d, scores: q x m, both row-major float32, both host or both
 * device as is_device_ptr says.  q = 0 is a no-op.  Errors: RFF_ENOTREADY before
 * the first solve, RFF_EINVAL for NaN/Inf queries. */
rff_status rff_admm_predict(rff_admm_t h, const float* Xq, int64_t q, float* scores, int is_device_ptr);

/* Scores without allocating device memory (the paper has no counterpart: it is an
 * interface for callers that cannot call cudaMalloc when they score -- code being
 * captured into a CUDA graph, where allocation is not a capturable operation, and
 * serving loops whose device memory is owned by another pool or that must not
 * allocate on the request path).  Same result as rff_admm_predict, same kernels.
 * Xq (q x d) and scores (q x m) are row-major float32 DEVICE pointers; the call
 * synchronises the handle's stream before it returns.
 * Scratch: one fixed 32 MiB array in device global memory, defined by the library
 * and held by every GPU that loads it until the process exits.  A call needs
 * q_pad * (4 d_pad + 4 m_pad) bytes on the FP32 path and q_pad * (8 d_pad + 4 m_pad)
 * on the split-BF16 path (q_pad = q rounded up to 128, d_pad = d rounded up to 64,
 * m_pad = m rounded up to 16); larger q returns RFF_EINVAL with the limit in the
 * error text -- score in smaller batches.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * All calls share the array and it keeps the previous call's contents (the call
 * clears what must start at zero): calls that overlap on the GPU -- two handles
 * or threads scoring at the same time -- race on it.
 * Errors: RFF_ENOTREADY before the first solve, RFF_EINVAL for NULL pointers,
 * NaN/Inf queries or q beyond the scratch, RFF_ECUDA. */
rff_status rff_admm_predict_noalloc(rff_admm_t h, const float* Xq, int64_t q, float* scores);

/* Copy the consensus weights Wbar (D x m, row-major, rows in global feature
 * order) to W.  Errors: RFF_ENOTREADY without data. */
rff_status rff_admm_get_weights(rff_admm_t h, float* W, int is_device_ptr);

/* Checkpoint: serialise the full ADMM state (O, Obar, nu, Delta, O'_ij, W, Wbar,
 * mu, W'_ij, mu'_ij, iteration count, parameters) into buf (host memory).  With
 * buf == NULL, *bytes receives the size needed.  Cached factors are not part of
 * the state: they are recomputed from (X, seed).  Errors: RFF_EINVAL if *bytes is
 * too small, RFF_ENOTREADY without data. */
rff_status rff_admm_get_state(rff_admm_t h, void* buf, size_t* bytes);

/* Restore a state written by rff_admm_get_state for the same data, parameters
 * and grid; continuing from it reproduces an uninterrupted run bit for bit.
 * Errors: RFF_EINVAL on a size, version or parameter mismatch. */
rff_status rff_admm_set_state(rff_admm_t h, const void* buf, size_t bytes);

/* Per-phase device timing of the iterations, for performance work.  enable = 1
 * makes rff_admm_solve record CUDA events around each phase of every iteration
 * on the handle's stream (a small overhead) and accumulate their durations;
 * enable = 0 stops it.  Either call resets the counters.  Kernel launches are
 * always counted. */
typedef struct {
  int64_t iters;           /* iterations since the last reset                                */
  int64_t launches;        /* kernels launched by those iterations                           */
  double ms_prox_reg;      /* W <- prox_r(Wbar - mu)                                         */
  double ms_pass1;         /* Z_ij^T V_ij, Z regenerated (fused kernel)                      */
  double ms_project;       /* right-hand side and the products with the cached Q_ij          */
  double ms_pass2;         /* Z_ij W'_ij, Z regenerated (fused kernel)                       */
  double ms_exchange;      /* row exchange, nu update, loss prox, next V_ij                  */
  double ms_average;       /* Wbar, mu, mu'_ij updates                                      */
} rff_admm_profile;

rff_status rff_admm_set_profiling(rff_admm_t h, int enable);
rff_status rff_admm_get_profile(rff_admm_t h, rff_admm_profile* out);

/* Release the handle and all device memory it owns.  NULL is ignored. */
void rff_admm_destroy(rff_admm_t h);

/* Text of the last error on this handle ("" if none).  Valid until the next call. */
const char* rff_admm_last_error(rff_admm_t h);

/* ------------------------------------------------------------------------------
 * Step-level entry points.  Each exposes one stage of the iteration on caller
 * device buffers, so every stage can be checked on its own.  All pointers are
 * CUDA device pointers; all calls are asynchronous on `stream` (NULL = legacy
 * default stream) and return RFF_EINVAL for bad sizes, RFF_ECUDA on launch
 * failure.
 * ------------------------------------------------------------------------------ */

/* Philox4x32-10 (Salmon et al., SC'11) on n counters: ctr n x 4 uint32, out n x 4
 * uint32, key = (seed mod 2^32, seed >> 32).  The generator that keeps omega
 * implicit (Sec. 4, last paragraph on the transform's memory). */
rff_status rff_philox4x32_10(const uint32_t* ctr, uint64_t seed, int64_t n, uint32_t* out, void* stream);

/* Random Fourier feature parameters for global features [k_lo, k_hi) (Sec. 4):
 * G (d x (k_hi - k_lo), row-major) with G[r,k] = float32(N_rk / sigma) and
 * b (k_hi - k_lo) with b[k] = float32(pi u_k), where N and u come from counter
 * (k, r/4, 0, 0) through Box-Muller and counter (k, 0, 1, 0) respectively,
 * each uniform u = ((w >> 8) + 0.5) 2^-24. */
rff_status rff_rff_params(uint64_t seed, double sigma, int64_t d, int64_t k_lo, int64_t k_hi, float* G,
                          float* b, void* stream);

/* The transform T[X, j] of Sec. 3 for a feature range: Z = sqrt(2/D) cos(X G + b)
 * for features [k_lo, k_hi) of a D-feature map.  X: n x d, Z: n x (k_hi - k_lo).
 * prec selects the arithmetic of the SIMT (RFF_PREC_FP32) or tensor-core
 * (RFF_PREC_SPLIT_BF16) regeneration kernels. */
rff_status rff_features(const float* X, int64_t n, int64_t d, uint64_t seed, double sigma, int64_t D,
                        int64_t k_lo, int64_t k_hi, int32_t prec, float* Z, void* stream);

/* Row-wise loss prox (Sec. 2.3 definition; Sec. 3 step O <- prox_{(1/rho) l}):
 * out_i = argmin_o 1/2 |o - v_i|^2 + t V(y_i, o).  V, Y, out: n x m.  out may
 * alias V.  newton_iters applies to the logistic and multinomial losses. */
rff_status rff_prox_loss(int32_t loss, const float* V, const float* Y, int64_t n, int32_t m, double t,
                         int32_t newton_iters, float* out, void* stream);

/* Entry-wise regulariser prox: out = argmin_w 1/2 |w - v|^2 + tau r(w).  n values. */
rff_status rff_prox_reg(int32_t reg, const float* V, int64_t n, double tau, float* out, void* stream);

/* Batched Cholesky factorisation in FP64 of `batch` SPD matrices (eq. (cache)):
 * A: batch x s x s row-major float64, overwritten by the lower factor L (upper
 * triangle zeroed).  info (device, batch int32): 0, or k+1 for a non-positive
 * pivot at column k. */
rff_status rff_cholesky_f64(double* A, int32_t batch, int32_t s, int32_t* info, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* RFF_ADMM_H */
