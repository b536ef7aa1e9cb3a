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
  RFF_ENUMERIC = 6,  /* a factorisation met a non-positive pivot                    */
  RFF_ECANCELLED = 7 /* a serving request cancelled before it started               */
} rff_status;

/* Losses V(y, o), used only through their proximal operators (Sec. 3 "Modularity"). */
typedef enum {
  RFF_LOSS_SQUARED = 0,    /* |y - o|^2, real targets                                  */
  RFF_LOSS_HINGE = 1,      /* m = 1: max(0, 1 - y o); m > 1: one-vs-rest, +-1 targets   */
  RFF_LOSS_LOGISTIC = 2,   /* log(1 + exp(-y o)) per output column, y = +-1            */
  RFF_LOSS_MULTINOMIAL = 3, /* log sum_k exp(o_k) - o_c, c = argmax_k y_k              */
  RFF_LOSS_L1 = 4,          /* |y - o|_1, real targets                                  */
  RFF_LOSS_CRAMMER_SINGER = 5 /* multiclass hinge max_k (Delta_k + o_k - o_c),          */
                              /* Delta_k = 1 - [k = c], c = argmax_k y_k                */
} rff_loss;

/* Regularisers r(W), separable over column blocks (Sec. 3, r = sum_j r_j(W_j)). */
typedef enum {
  RFF_REG_L2SQ = 0, /* |W|_F^2 */
  RFF_REG_L1 = 1    /* sum |W_kl| */
} rff_reg;

/* How Z_ij is regenerated and applied. */
typedef enum {
  RFF_PREC_FP32 = 0,      /* X.G, cos and both chained products in FP32 on the SIMT pipes  */
  RFF_PREC_SPLIT_BF16 = 1, /* the split tensor-core path: X.G as three FP16 products
                             (hi.hi + hi.lo + lo.hi) of the hi/lo splits of X and G, each
                             scaled by a power of two into |.| <= 2^8 (22 significant bits
                             per operand), FP32 accumulate in TMEM, FP32 cos; the chained
                             products as three FP16 products of hi/lo splits of 2^7 cos and
                             of V, W' (scaled from their maxima); the projection with Q and
                             its right-hand side as three BF16 terms (six products, the
                             dominant ones in an accumulator of their own).  Queries beyond
                             2^15 / (X scale), at least 128 times the largest training |x|,
                             are refused (RFF_EINVAL)                                    */
  RFF_PREC_CACHED_Z = 2   /* Z materialised once (set-up, FP32 on the SIMT pipes) and kept
                             in device memory as a scaled FP16 hi/lo pair, with a
                             transposed copy: n_slots x D_slots x 8 bytes.  Each iteration
                             streams it through the same three-product chained GEMMs
                             instead of regenerating it; the comparison mode of the paper's
                             memory trade-off (Sec. 3: Z is not stored), for data sets
                             whose Z fits in device memory                                 */
} rff_precision;

/* Scaling of rho (the paper never fixes it).  RFF_RHO_SUM: rho is the penalty of the
 * objective sum_i V + n lambda r, so the loss prox step is 1/rho and the regulariser
 * step n lambda / rho.  RFF_RHO_MEAN: rho as in Sec. 3 with l_i carrying 1/n, i.e. loss
 * step 1/(n rho), regulariser step lambda/rho.  The two are one method with
 * rho_mean = rho_sum / n. */
typedef enum { RFF_RHO_SUM = 0, RFF_RHO_MEAN = 1 } rff_rho_scale;

/* The feature map z(.) behind the operator T[X_i, j] (Sec. 4: the solver treats it as a
 * black box; the paper lists random Fourier features and, among others, random Laplace
 * features).  Both are drawn from the same Philox stream of standard normals g:
 *   RFF_MAP_FOURIER  z(x) = sqrt(2/D) cos(G^T x + b), G = g / sigma, b ~ U[0, pi):
 *                    the Gaussian kernel exp(-|x - x'|^2 / (2 sigma^2))
 *   RFF_MAP_LAPLACE  z(x) = exp(-W^T x) / sqrt(D), W = 1 / (2 sigma^2 g^2) (Levy): the
 *                    exponential semigroup kernel exp(-sum_r sqrt(x_r + x'_r) / sigma) on
 *                    nonnegative inputs (histograms); FP32 and cached-Z precisions only
 *   RFF_MAP_FASTFOOD z(x) = sqrt(2/D) cos(V x + b) with the Fastfood matrix (Le, Sarlos and
 *                    Smola 2013): per block of d' = 2^p >= d features
 *                    V = S H diag(g) P H diag(B) / (sigma sqrt(d')), H Walsh-Hadamard, B signs,
 *                    P a permutation, S chi(d') row lengths over |g|; every row of V is
 *                    N(0, I / sigma^2), so the Gaussian kernel again; d <= 4096
 *   RFF_MAP_TENSORSKETCH  TensorSketch (Pham and Pagh 2013) of the polynomial kernel
 *                    (<x, x'> / sigma^2 + coef0)^degree: with x~ = (x / sigma, sqrt(coef0)),
 *                    column block j (s_j features) is its own sketch, the circular
 *                    convolution of `degree` CountSketches of x~ of length s_j, scaled by
 *                    sqrt(s_j / D) (Sec. 4 assembles maps that need their whole vector from
 *                    independent per-block maps), so Z depends on the column partition.
 *                    Hashes and signs: Philox counter (j, p (d + 1) + i, 7, 0), h = (w0 s_j)
 *                    >> 32, sign -1 iff the top bit of w1 is set.  Cached-Z precision only (Z
 *                    is formed once); degree 1..8, s_j <= 8192 */
typedef enum {
  RFF_MAP_FOURIER = 0,
  RFF_MAP_LAPLACE = 1,
  RFF_MAP_FASTFOOD = 2,
  RFF_MAP_TENSORSKETCH = 3
} rff_feature_map;

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
  int32_t feature_map;  /* rff_feature_map (0: random Fourier features)              */
  int32_t degree;       /* TensorSketch: polynomial degree (1..8); other maps ignore it */
  double coef0;         /* TensorSketch: the kernel's offset >= 0; other maps ignore it */
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
 * C < 1, C > D, m outside [1, 256], unknown enums, C > 64 with
 * RFF_PREC_SPLIT_BF16),
 * RFF_ECUDA if no device is usable. */
rff_status rff_admm_create(const rff_admm_params* params, void* stream, rff_admm_t* out);

/* Attach the training set (Sec. 3: X_i, Y_i row blocks).  X: n x d, Y: n x m,
 * row-major float32; copied, the caller keeps ownership.  Resets the ADMM state
 * and drops any cached factors.  Errors: RFF_EINVAL for n < R, d < 1, NaN/Inf
 * in X or Y, targets outside {-1, +1} for the hinge and logistic losses;
 * RFF_ENOMEM when the device cannot hold the working set (checked first). */
rff_status rff_admm_set_data(rff_admm_t h, const float* X, const float* Y, int64_t n, int64_t d,
                             int is_device_ptr);

/* As rff_admm_set_data with X in compressed sparse row form (Sec. 4: sparse inputs enter
 * only through T): indptr (n + 1, int64, indptr[0] = 0, non-decreasing, indptr[n] = nnz),
 * indices (nnz column indices in [0, d), int32), values (nnz float32).  Repeated columns
 * of a row add up.  The rows are expanded into the dense slot layout on the device (the
 * tensor cores take dense tiles: at the paper's 20 %-dense MNIST rows the dense product
 * is the faster one), so only the sparse arrays cross from the host.  The same arrays
 * go host -> device (is_device_ptr = 0) or stay on the device (1).  Errors: those of
 * rff_admm_set_data, and RFF_EINVAL for a malformed structure. */
rff_status rff_admm_set_data_csr(rff_admm_t h, const int64_t* indptr, const int32_t* indices, const float* values,
                                 int64_t nnz, const float* Y, int64_t n, int64_t d, int is_device_ptr);

/* Run `iters` further ADMM iterations (the update equations of Sec. 3 around
 * eq. (gp), all variables starting at zero after set_data).  The first call
 * after set_data first draws G and b (Sec. 4), forms each block's Gram matrix
 * I + Z_ij^T Z_ij and caches its inverse from an FP64 Cholesky factorisation
 * (eq. (cache)); later calls reuse the cache.  stats may be NULL; when given,
 * residuals and objective are computed after the last iteration (one extra
 * pass over the data).  Errors: RFF_ENOTREADY without data, RFF_ENUMERIC if a
 * Gram matrix is not positive definite, RFF_ECUDA. */
rff_status rff_admm_solve(rff_admm_t h, int32_t iters, rff_admm_stats* stats);

/* Device-memory budget of a handle (0 = whatever the device has free).  set_data
 * refuses a working set beyond it (RFF_ENOMEM, before allocating) and the set-up
 * sizes its factorisation batches to stay within it.  The GPU analogue of the
 * memory model of Sec. 3 (eq. (mem)). */
rff_status rff_admm_set_memory_limit(rff_admm_t h, size_t bytes);

/* Moves the handle's work to another CUDA stream (for instance one of higher
 * priority for scoring a solved model while other solves run).  Waits for the work
 * already on the current stream; a stream the library created is destroyed, the
 * new one stays the caller's.  Results do not depend on the stream. */
rff_status rff_admm_set_stream(rff_admm_t h, void* cuda_stream);

/* Device bytes a solve of n x d data with these parameters holds while it iterates
 * (*resident: data, state, cached factors) and at its peak during set-up with the
 * smallest factorisation batch (*peak); either pointer may be NULL.  No device work. */
rff_status rff_admm_estimate_bytes(const rff_admm_params* params, int64_t n, int64_t d, size_t* resident,
                                   size_t* peak);

/* One lambda per output column (the columns are then independent solves that
 * share X, sigma, D, the grid and therefore Z and its cached factor -- the lambda
 * axis of a model-selection sweep costs one regeneration of Z for all lambdas).
 * lambdas: m values > 0, copied; NULL restores params.lambda for every column.
 * Separable losses only give independent columns (squared, hinge, logistic).
 * Errors: RFF_EINVAL for a wrong count or a non-positive value. */
rff_status rff_admm_set_lambdas(rff_admm_t h, const double* lambdas, int32_t m);

/* Give back the device copies of the feature parameters (G, or the Laplace W, or the
 * Fastfood V, and their FP16 split): Sec. 4 keeps omega implicit as the state of the
 * generator, regenerated on demand.  A resident model then holds no d x D parameters
 * (2 d_pad D_slots x 2 B on the split path, 4 d_pad D_slots B on the FP32 path); each later
 * rff_admm_predict draws them again for that call (a few hundred microseconds at
 * d = 440, D = 16384) and gives them back, and rff_admm_solve keeps them resident again.
 * The draw is bit-identical, so scores and iterates do not change.  *bytes (may be NULL)
 * receives the bytes freed.  rff_admm_predict_noalloc refuses a released model
 * (RFF_ENOTREADY).  Errors: RFF_ENOTREADY before the first solve. */
rff_status rff_admm_release_features(rff_admm_t h, size_t* bytes);

/* Stochastic block subsets (proposed in Sec. 5 and the conclusion): from the next
 * iteration on, each block (i, j) takes part in the graph projection of an iteration
 * with probability p, independently; the others keep their W'_ij and O'_ij for that
 * iteration while every prox, the exchange, the averaging and every dual (mu_ij too)
 * update as usual.  Block b = i C + j is active in iteration k (counted from the
 * start of the solve, across calls and checkpoints) iff (w >> 8) < floor(p 2^24), w the
 * first word of Philox4x32-10 at counter (b, k, 2, 0) under params.seed.  p = 1 (the
 * default) is the deterministic method.  The iteration time of the passes and the
 * projection falls with the number of active blocks.
 * Errors: RFF_EINVAL unless 2^-24 <= p <= 1. */
rff_status rff_admm_set_block_fraction(rff_admm_t h, double p);

/* Queue `iters` iterations on the handle's stream and return without waiting
 * (set-up, when still needed, runs first and synchronously).  rff_admm_wait
 * blocks until they finished and reports a device-side failure. */
rff_status rff_admm_enqueue(rff_admm_t h, int32_t iters);
rff_status rff_admm_wait(rff_admm_t h);

/* Model-selection sweep: runs `iters` iterations of every handle (each created
 * with its own stream, typically one per sigma with its lambdas as columns), all
 * queued before any is waited for, so the solves overlap on the device.  Each
 * iteration after a handle's first runs as one CUDA-graph launch. */
rff_status rff_sweep_run(rff_admm_t* handles, int32_t n, int32_t iters);

/* Scores f(x) = Wbar^T z(x) for q query rows (Sec. 2.2, H_{k,l}; prediction in
 * Sec. 5).  Xq: q x d, scores: q x m, both row-major float32, both host or both
 * device as is_device_ptr says.  q = 0 is a no-op.  Errors: RFF_ENOTREADY before
 * the first solve, RFF_EINVAL for NaN/Inf queries. */
rff_status rff_admm_predict(rff_admm_t h, const float* Xq, int64_t q, float* scores, int is_device_ptr);

/* Class labels of q query rows (test accuracy, Sec. 5): m = 1: +1 where the score is >= 0,
 * else -1; m > 1: the index of the largest score (the lowest index among equal scores).
 * labels: q int32, host (is_device_ptr = 0, Xq host too) or device (1).  Errors: those of
 * rff_admm_predict. */
rff_status rff_admm_predict_labels(rff_admm_t h, const float* Xq, int64_t q, int32_t* labels, int is_device_ptr);

/* Scores without allocating device memory (the paper has no counterpart: it is an
 * interface for callers that cannot call cudaMalloc when they score -- a serving loop
 * whose device memory is handed out entirely by another allocator's pool, so that a
 * cudaMalloc of its own would fail or fragment that pool, or one that must not take the
 * device-wide synchronisation an allocation or a free can cost in the middle of a
 * request).  Same result as rff_admm_predict with device pointers, bit for bit: the
 * same kernels on the same padded layout.  Xq (q x d) and scores (q x m) are row-major
 * float32 DEVICE pointers.  The call synchronises the handle's stream twice (after the
 * finite-value check of the queries and before it returns).
 * Scratch: one fixed 32 MiB array in device global memory, defined by the library and
 * held by every GPU that loads it until the process exits.  With q_pad = q rounded up to
 * 128, d_pad = d rounded up to 64, m_pad = m rounded up to 16 and up() rounding up to a
 * multiple of 256 bytes, a call needs up(4 q_pad d_pad) + 4 q_pad m_pad bytes on the
 * FP32 path and up(4 q_pad d_pad) + 2 up(2 q_pad d_pad) + 4 q_pad m_pad bytes on the
 * split path (the queries in FP32, their FP16 hi/lo split, the padded scores); a larger
 * q returns RFF_EINVAL with the limit in the error text -- score in smaller batches.
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress,
 * once per device, that device current).
 * All calls share the array and it keeps the previous call's contents (the call clears
 * what must start at zero): calls that overlap on the GPU -- two handles or threads
 * scoring at the same time -- race on it.
 * Errors: RFF_ENOTREADY before the first solve or after rff_admm_release_features,
 * RFF_EINVAL for NULL pointers, NaN/Inf queries or q beyond the scratch, RFF_ECUDA. */
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
 * and grid; continuing from it reproduces an uninterrupted run bit for bit (with a
 * block fraction, when the same fraction is set).  Runs the set-up (factors) first
 * if no solve has yet.  Errors: RFF_EINVAL on a size, version or parameter mismatch. */
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
  int32_t tc_kchunk;       /* K chunk of the tensor-core ring chosen by the autotuner (0: FP32) */
  int32_t nsplit;          /* row splits of pass 1 chosen by the autotuner                   */
  int32_t tc_z_tmem;       /* geometry of the tensor-core passes (chosen by the autotuner;
                              the environment variable RFF_TC_GEOMETRY="kc,zt" or
                              "kc,zt,cg" fixes it instead): 0 the Z tile in shared memory,
                              1 in tensor memory, 2 in tensor memory with two X.G
                              accumulators (m_pad <= 128), 3 X.G products 256 features wide
                              (m_pad <= 192)                                               */
  int32_t tc_cta_pair;     /* 1: the tensor-core passes run as CTA pairs (clusters of two
                              CTAs sharing each M = 256 MMA), 0: one CTA per MMA            */
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

/* The random Laplace map's parameters W (d x (k_hi - k_lo), row-major, device) for
 * global features k_lo..k_hi-1, from the same counters as rff_rff_params' G. */
rff_status rff_laplace_params(uint64_t seed, double sigma, int64_t d, int64_t k_lo, int64_t k_hi, float* W,
                              void* stream);

/* Z = exp(-X W) / sqrt(D) for global features k_lo..k_hi-1 (FP32), X n x d nonnegative,
 * Z n x (k_hi - k_lo); device pointers.  Errors: RFF_EINVAL for a negative or non-finite x. */
rff_status rff_laplace_features(const float* X, int64_t n, int64_t d, uint64_t seed, double sigma, int64_t D,
                                int64_t k_lo, int64_t k_hi, float* Z, void* stream);

/* TensorSketch features (RFF_MAP_TENSORSKETCH) of the rows of X (n x d, device, row-major)
 * for D features in C column blocks partitioned as the solver does (the leading D mod C
 * blocks one larger): Z (n x D, device, row-major), block j in its columns, scaled by
 * sqrt(s_j / D).  Errors: RFF_EINVAL for a degree outside 1..8, coef0 < 0, blocks over 8192
 * features or a shared-memory footprint (degree, d, block size) the kernel cannot hold. */
rff_status rff_tensorsketch_features(const float* X, int64_t n, int64_t d, uint64_t seed, double sigma,
                                     double coef0, int32_t degree, int64_t D, int32_t C, float* Z, void* stream);

/* The Fastfood map's projection for global features k_lo..k_hi-1: Vt ((k_hi - k_lo) x d,
 * row-major: row r is V's row k_lo + r) and b (k_hi - k_lo), device pointers; D sets the
 * block structure only through d' (features are grouped in blocks of d').  d <= 4096. */
rff_status rff_fastfood_params(uint64_t seed, double sigma, int64_t d, int64_t k_lo, int64_t k_hi, float* Vt,
                               float* b, void* stream);

/* Failure-path self test: launches a one-thread probe that waits, through the tensor-core
 * passes' bounded wait, on an mbarrier nothing arrives on.  The wait gives up after about a
 * millisecond, sets the device error word and returns, so the call returns RFF_ETIMEOUT (the
 * status a timed-out pass reports) and clears the word; the context stays usable.  RFF_OK
 * would mean the bound did not fire. */
rff_status rff_selftest_wait_timeout(void* stream);

/* Bounds-checked build.  The library is also built with device-side bounds checks
 * (librff_admm_check.so, compiled with -DRFF_CHECK): the kernels of the iteration and of
 * scoring test, at their global accesses, that every element index lies inside the layout
 * the operation defines (the regeneration passes' X, G, chained-operand and output tiles, the
 * tensor-core epilogues' output rows, the exchange's row tiles, the sparse scatter's column
 * indices, the TensorSketch output rows, the factorisation's operand slices) and that every
 * TMA box starts on a 16-byte boundary; a failed test skips the access and is counted.  rff_check_enabled() is 1 in that build and 0 in the ordinary one.
 * rff_check_report synchronises the device and reads and clears the counts into out[5]:
 *   out[0]  failed tests since the last report (0 in the ordinary build),
 *   out[1]  source unit of the first failure: 1 elementwise.cu, 2 qgemm.cu, 3 regen_simt.cu,
 *           4 tc.cu, 5 sketch.cu, 6 ozaki.cu,
 *   out[2]  its source line, out[3] the index tested, out[4] the bound it broke.
 * A skipped TMA copy leaves its barrier incomplete: the bounded wait on it gives up and the
 * pass returns RFF_ETIMEOUT.  Returns RFF_ECUDA if the device reports an error. */
int32_t rff_check_enabled(void);
rff_status rff_check_report(int64_t* out);

/* Measured FMA throughput of this GPU's SIMT pipes in TFLOP/s (2 flop per FMA): FP32 and
 * FP64, each from one timed launch of independent multiply-add chains (about 20 ms), the
 * roofline denominators of the FP32 path and the set-up kernels.  Runs on stream. */
rff_status rff_measure_fma_peaks(double* fp32_tflops, double* fp64_tflops, void* stream);

/* Batched Cholesky factorisation of `batch` SPD matrices (eq. (cache)), FP64 in and out:
 * A: batch x s x s row-major float64, overwritten by the lower factor L (upper
 * triangle zeroed).  info (device, batch int32): 0, or k+1 for a non-positive
 * pivot at column k.  The 64 x 64 diagonal blocks are factored in FP64; the block
 * updates run on the tensor cores as exact products of 8-bit slices of the FP64 operands'
 * 48 leading bits (each update within about 2^-45 of max|A_r| max|B_c| K), so the factor
 * agrees with an FP64 factorisation to about 1e-13 relative (3.8e-14 measured against
 * numpy's at orders up to 2048). */
rff_status rff_cholesky_f64(double* A, int32_t batch, int32_t s, int32_t* info, void* stream);

/* ------------------------------------------------------------------------------
 * Serving: solve and scoring requests of different sizes, admitted by a device-
 * memory budget and run side by side (one CUDA stream per active request); solved
 * models stay resident for scoring until released.  The paper has no serving
 * layer; admission uses the memory accounting of rff_admm_estimate_bytes (the GPU
 * analogue of eq. (mem), Sec. 3).  Thread-safe: any host thread may submit, poll
 * or release.
 * ------------------------------------------------------------------------------ */
typedef struct rff_server_s* rff_server_t;

enum { RFF_REQ_SOLVE = 0, RFF_REQ_SCORE = 1 };

typedef struct {
  int64_t id;         /* request id returned by the submit call                          */
  int32_t kind;       /* RFF_REQ_SOLVE or RFF_REQ_SCORE                                  */
  int32_t status;     /* rff_status of the request                                        */
  double queue_ms;    /* submit -> start (waiting for a worker and for device memory)     */
  double run_ms;      /* start -> done                                                    */
  double latency_ms;  /* submit -> done                                                   */
} rff_completion;

/* budget_bytes: device memory the server may hand out (0 = 90% of what is free);
 * max_active: requests that may run at once (worker threads, 1..256). */
rff_status rff_server_create(size_t budget_bytes, int32_t max_active, rff_server_t* out);

/* Queue a solve of (X, Y) (host, n x d and n x m, copied) for `iters` iterations.
 * *request_id doubles as the model id for scoring.  RFF_ENOMEM when the solve's
 * peak memory exceeds the whole budget (it could never be admitted). */
rff_status rff_server_submit_solve(rff_server_t srv, const rff_admm_params* params, const float* X, const float* Y,
                                   int64_t n, int64_t d, int32_t iters, int64_t* request_id);

/* Queue scores of q rows Xq (host, copied) against a model; `scores` (host, q x m)
 * is written before the completion is posted and must stay valid until then.
 * A model whose solve is still queued or running is waited for. */
rff_status rff_server_submit_score(rff_server_t srv, int64_t model, const float* Xq, int64_t q, float* scores,
                                   int64_t* request_id);

/* Up to `max` completions, oldest first; waits up to wait_ms for the first one. */
rff_status rff_server_poll(rff_server_t srv, rff_completion* out, int32_t max, int32_t* count, int32_t wait_ms);

/* Weights of a solved model (host, D x m), as rff_admm_get_weights. */
rff_status rff_server_get_weights(rff_server_t srv, int64_t model, float* W);

/* Cancel a request that has not started: it leaves the queue and completes at once with
 * status RFF_ECANCELLED (a score waiting for a cancelled solve then fails with RFF_EINVAL).
 * Returns RFF_ENOTREADY for a request that is running or done, RFF_EINVAL for an unknown id. */
rff_status rff_server_cancel(rff_server_t srv, int64_t request_id);

/* Drop a solved (or failed) model and give its memory back to the budget. */
rff_status rff_server_release(rff_server_t srv, int64_t model);

/* Bytes currently reserved and the budget. */
rff_status rff_server_memory(rff_server_t srv, size_t* used, size_t* budget);

/* Stop the workers (running requests finish first) and free every model. */
void rff_server_destroy(rff_server_t srv);

#ifdef __cplusplus
}
#endif

#endif /* RFF_ADMM_H */
