/*
 * mvn.h -- C ABI of the GB300 (sm_103a) library for Separation-of-Variables (SOV) estimation
 * of multivariate normal probabilities and the confidence-region loop built on it.
 *
 * Paper: "Parallel Approximations for High-Dimensional Multivariate Normal Probability
 * Computation in Confidence Region Detection Applications" (arXiv 2405.14892).
 *
 * Conventions (all entry points):
 *   - Array arguments are DEVICE pointers (e.g. torch.Tensor.data_ptr() of a CUDA tensor) unless
 *     a comment says "host".  Scalars are host values.  Matrices are column-major with leading
 *     dimension `ld` (in elements, ld >= n), FP64.
 *   - The caller owns every input and output buffer.  The context owns its workspace, which
 *     grows on demand (cudaMalloc) and is kept until mvn_destroy; after a first call of a given
 *     size, later calls of that size allocate nothing.
 *   - Work is enqueued on the context's stream and is asynchronous unless stated otherwise.
 *     The returned status reports host-side validation and launch errors.  Errors found on
 *     the device (a non-positive pivot, a numeric failure, a wait that timed out) are written to
 *     a device status word; mvn_sync waits for the stream and returns it.
 *   - No exception or exit crosses the ABI.  A context is not thread-safe; separate contexts
 *     are independent.
 *   - A NULL context, graph or TLR handle is rejected before any CUDA call: the entry point
 *     returns MVN_ERR_ARG (mvn_last_error(NULL) returns "null context", mvn_launch_count(NULL)
 *     returns -1, mvn_graph_kernels(NULL) returns 0, and mvn_graph_destroy(NULL) is a no-op
 *     that returns MVN_OK).
 */
#ifndef MVN_H
#define MVN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mvn_ctx mvn_ctx;
typedef struct mvn_tlr mvn_tlr;

typedef enum {
    MVN_OK = 0,
    MVN_ERR_ARG = 1,             /* invalid argument (size, pointer, NaN limit, a > b ...)      */
    MVN_ERR_NOT_PD = 2,          /* matrix not positive definite (see `info`)                   */
    MVN_ERR_CUDA = 3,            /* CUDA runtime error (message in mvn_last_error)              */
    MVN_ERR_OOM = 4,             /* workspace allocation failed                                 */
    MVN_ERR_TIMEOUT = 5,         /* a bounded device-side wait expired                          */
    MVN_ERR_NUMERIC = 6,         /* every path has weight 0 (P-hat = 0, log P-hat = -inf)       */
    MVN_ERR_NOT_IMPLEMENTED = 7
} mvn_status;

/* Arithmetic of the compute path.
 *   MVN_FP64       : every step in FP64 (the plain FP64 GPU path).
 *   MVN_MIXED      : Cholesky updates exact from BF16 digit slices on the tcgen05 tensor cores
 *                    with a double-float panel (see mvn_cholesky); SOV limit-update GEMM on the
 *                    tcgen05 tensor cores with each operand split into two FP16 slices (3 MMAs
 *                    per K step, FP32 accumulation in TMEM drained to FP32 registers every
 *                    128 K), limits and transformed variables in FP32, the running log-weight in
 *                    FP64, deep tails of Phi and Phi^-1 in FP64.
 *   MVN_MIXED_SIMT : as MVN_MIXED for the sweep, with the limit-update GEMM in FP32 on the CUDA
 *                    cores; the Cholesky as MVN_FP64. */
typedef enum { MVN_FP64 = 0, MVN_MIXED = 1, MVN_MIXED_SIMT = 2 } mvn_prec;

/* Randomly shifted rank-1 (Richtmyer) lattice rule that replaces the uniforms R of Alg. 2:
 *   w_{q,j,i} = frac(j * alpha_i + Delta_{q,i}) in 64-bit fixed point, j = 1..n_points,
 *   alpha_i = floor(sqrt(p_i) 2^64) mod 2^64 (p_i the i-th prime, p_0 = 2),
 *   Delta_{q,i} = SplitMix64(seed, counter q*2^32 + i), q = 0..n_shifts-1.
 * Path p = q * n_points + (j - 1).  The estimate is P-hat = mean over all paths of exp(logw_p);
 * err = err_k * sd_q(P-hat_q) / sqrt(n_shifts). */
typedef struct {
    int64_t n_points; /* points per shift (>= 1)                                     */
    int32_t n_shifts; /* number of random shifts M (>= 1; >= 2 for an error estimate) */
    int32_t reserved;
    uint64_t seed;    /* key of the shift generator                                  */
    double err_k;     /* error multiplier (3 = three standard errors)                */
} mvn_qmc;

/* ------------------------------------------------------------------ context */

/* Create a context on CUDA device `device`, enqueuing on `cuda_stream` (a cudaStream_t; NULL =
 * the legacy default stream).  *out receives the context.  Errors: MVN_ERR_ARG, MVN_ERR_CUDA. */
mvn_status mvn_create(mvn_ctx** out, int device, void* cuda_stream);
mvn_status mvn_destroy(mvn_ctx* ctx);
/* Switch the stream later calls enqueue on. */
mvn_status mvn_set_stream(mvn_ctx* ctx, void* cuda_stream);
/* Message of the last error on this context (never NULL; "" if none). */
const char* mvn_last_error(const mvn_ctx* ctx);
/* Wait for the stream; return (and clear) the device status word.  If info != NULL (host),
 * *info receives the LAPACK-style failing column of the last failed factorisation, else 0. */
mvn_status mvn_sync(mvn_ctx* ctx, int* info);
/* Number of kernels this context has launched since creation (host counter). */
int64_t mvn_launch_count(const mvn_ctx* ctx);
/* Per-kernel timing: with enable != 0, CUDA events are recorded on the context's stream around
 * every launch of the main kernels (k_oz_update, k_oz_potrf, k_oz_trsm, k_syrk,
 * k_sov_tc, k_sov_simt_f64, k_sov_simt_f32, and in mvn_sov_grad k_sov_grad_fwd_f64/_f32,
 * k_sov_rev_f64/_f32, k_grad_L_f64/_f32); the call waits for the stream and clears earlier
 * records. */
mvn_status mvn_timing(mvn_ctx* ctx, int enable);
/* Total device time (ms, host) and number of launches (host) of kernel `name` recorded since
 * the last mvn_timing call; waits for the stream. */
mvn_status mvn_kernel_time(mvn_ctx* ctx, const char* name, double* total_ms, int64_t* launches);

/* ------------------------------------------------------------------ covariance (Eq. 6) */

/* Matern covariance of Eq. 6 for nu in {0.5, 1.5, 2.5} (closed forms of the Bessel K_nu):
 *   Sigma_ij = C(||s_i - s_j||; sigma2, range, nu) + nugget * [i == j].
 * coords: n x 2 row-major FP64 (x_i, y_i).  Sigma: n x n column-major (ld); only the lower
 * triangle (i >= j) is written.  Errors: MVN_ERR_ARG (nu not supported, n < 0, ld < n). */
mvn_status mvn_matern(mvn_ctx* ctx, int n, const double* coords, double sigma2, double range,
                      double nu, double nugget, double* Sigma, int64_t ld);

/* Contraction of a lower-triangle gradient with the Matern parameter derivatives:
 *   out[0] = sum_{i>=j} Sbar_ij dSigma_ij/dsigma2,  out[1] = sum_{i>=j} Sbar_ij dSigma_ij/drange,
 * for nu in {0.5, 1.5}.  Sbar: n x n column-major (ld), lower triangle read.  out: device
 * double[2].  Deterministic (fixed reduction order). */
mvn_status mvn_matern_grad(mvn_ctx* ctx, int n, const double* coords, double sigma2,
                           double range, double nu, const double* Sbar, int64_t ld,
                           double* out);

/* ------------------------------------------------------------------ Cholesky (Alg. 1, "dpotrf") */

/* In-place lower Cholesky factorisation A = L L^T (Alg. 1 "dpotrf"), tile algorithm.  Only the
 * lower triangle of A is read and written.
 * tile: the paper's tile size (a parameter of its CPU task runtime), accepted for the interface
 * and not used: on this GPU the panel width is fixed at 64 (the width of the tensor-core digit
 * tiles and of the FP64 register-blocked kernels), and what the autotuner chooses instead is the
 * split-K size of the update's work items (mvn_autotune); any value >= 0 is accepted.
 * prec: MVN_FP64 / MVN_MIXED_SIMT: right-looking over 64-wide panels, every update in FP64.
 *   MVN_MIXED: left-looking over 64-wide panels; the trailing updates run on the tcgen05 tensor
 *   cores on exact BF16 digit slices of the rows of L (6 balanced digits of 7 bits of each entry
 *   after a per-row power-of-two scaling, 42 bits in all; digit products summed exactly in FP32
 *   over 256-wide K groups and then in 64-bit integers, so every product carries ~42 bits and
 *   the result does not depend on the order of the split-K partial sums).  The diagonal block
 *   (POTRF and its inverse) and the panel solve run in double-float (FP32 pair, ~48 bits)
 *   arithmetic, reading and writing FP64.  The SOV estimate needs a factor well beyond FP32
 *   accuracy (an FP32 factor moves log P by ~1e-2 at n = 16,384); the measured backward error
 *   ||L L^T - A|| / ||A|| is ~1e-11 at n = 700 and below 5e-10 at n = 16,384 (against ~1e-16 for
 *   MVN_FP64), and log P at n = 16,384 moves by ~3e-5.  The Schur complements' diagonal must
 *   lie in FP32's normal range (about 1e-37 .. 1e38).
 * info (host, optional): if non-NULL the call waits for completion and *info = 0 or the 1-based
 * index of the first non-positive pivot (LAPACK convention), returning MVN_ERR_NOT_PD in that
 * case.  If NULL the call is asynchronous and a failure is reported by mvn_sync. */
mvn_status mvn_cholesky(mvn_ctx* ctx, int n, double* A, int64_t ld, int tile, mvn_prec prec,
                        int* info);

/* Cholesky factorisation with the univariate variable reordering (Gibson, Glasbey and Elston
 * 1994; Genz and Bretz 2009, Sec. 4.1.3).  Not in the paper: a variance-reducing variant of the
 * SOV estimator of Eq. 2 that changes the order of integration, not the probability.  Step i
 * places next the remaining variable with the smallest conditional interval probability
 * Phi(b'_j) - Phi(a'_j), a'_j = (a_j - s_j)/sqrt(d_j), b'_j = (b_j - s_j)/sqrt(d_j), where d_j is
 * its conditional variance given the variables placed so far and s_j = sum_k L_jk y_k with y_k
 * the truncated-normal means E[Z | a'_k < Z < b'_k] of those variables (an interval probability
 * that underflows takes the finite limit as y); ties go to the variable earliest in the current
 * order.
 *   A      : on entry Sigma (n x n, column-major, ld; lower triangle read); on exit the lower
 *            factor L of Sigma[perm, perm] (strict upper part untouched).  FP64 throughout.
 *   a, b   : device n-vectors of the limits (inputs).
 *   perm   : device int32[n]; perm[i] = original index of the i-th variable.
 *   a_perm, b_perm: device n-vectors, a[perm] and b[perm] (inputs of mvn_sov with this L).
 *   info   : as in mvn_cholesky (the 1-based step at which no remaining conditional variance is
 *            positive).
 * Workspace: ~2 n doubles.  Asynchronous unless info is given. */
mvn_status mvn_cholesky_reorder(mvn_ctx* ctx, int n, double* A, int64_t ld, const double* a,
                                const double* b, int32_t* perm, double* a_perm, double* b_perm,
                                int* info);

/* Reverse mode of mvn_cholesky (blocked form of the column algorithm's adjoint; Murray 2016).
 * L: the factor (lower, ld).  Lbar: on entry dF/dL (lower triangle, ld); on exit dF/dA for the
 * lower-triangle entries A_ij (i >= j) read by the factorisation (strict upper part untouched). */
mvn_status mvn_cholesky_grad(mvn_ctx* ctx, int n, const double* L, int64_t ld, double* Lbar);

/* ------------------------------------------------------------------ SOV (Eqs. 2-3, Algs. 2-3) */

/* P(a <= X <= b), X ~ N(0, L L^T), by the blocked SOV sweep on the shifted lattice rule.
 * a, b: device n-vectors (a_i = -INFINITY / b_i = +INFINITY allowed; a_i <= b_i, no NaN).
 * L: lower Cholesky factor, n x n column-major (ld), FP64 (only the lower triangle is read).
 * out3: device double[3] = {log P-hat, P-hat, err}.
 * path_logw: optional device double[n_points * n_shifts], the per-path log-weights.
 * Errors: MVN_ERR_ARG; MVN_ERR_NUMERIC (via mvn_sync) if every path has weight 0. */
mvn_status mvn_sov(mvn_ctx* ctx, int n, const double* a, const double* b, const double* L,
                   int64_t ld, const mvn_qmc* qmc, mvn_prec prec, double* out3,
                   double* path_logw);

/* One shard of mvn_sov: the global paths [p0, p1) of the lattice rule (0 <= p0 <= p1 <=
 * n_points * n_shifts), for splitting one problem over several GPUs.  The paths are independent
 * QMC samples (Sec. IV-C; Alg. 2's tasks over the sample tiles), so every GPU sweeps its own range
 * with the same factor and limits, and the shards' per-shift pairs are combined afterwards
 * (mvn_sov_combine) after an exchange of 2 * n_shifts doubles per shard.
 *   partial: device double[2 * n_shifts]; for each shift q, partial[2q] = max of the log-weights
 *            of the shard's paths of shift q, partial[2q+1] = sum of exp(logw - that max); a
 *            shift with no path in the range gets (-inf, 0).
 *   path_logw: optional device double[p1 - p0], the shard's per-path log-weights (local index
 *            p - p0), identical to mvn_sov's for the same paths.
 * Other arguments and errors as in mvn_sov (precisions included).  Asynchronous. */
mvn_status mvn_sov_partial(mvn_ctx* ctx, int n, const double* a, const double* b,
                           const double* L, int64_t ld, const mvn_qmc* qmc, mvn_prec prec,
                           int64_t p0, int64_t p1, double* partial, double* path_logw);

/* Combine the pairs of nparts shards (device, partials[r * 2 * n_shifts + ...] as written by
 * mvn_sov_partial; disjoint path ranges that together cover the rule) into out3 = {log P-hat,
 * P-hat, err} (device double[3]): per shift, m = max over shards and s = sum of s_r exp(m_r - m)
 * in shard order, then log P_q = m + log s - log n_points and Alg. 2's mean over the shifts as
 * in mvn_sov.  One shard covering all paths reproduces mvn_sov's out3 bit for bit; a split
 * inside a shift agrees to rounding (~1e-16 relative).  MVN_ERR_NUMERIC via mvn_sync if every
 * weight is 0.  Asynchronous. */
mvn_status mvn_sov_combine(mvn_ctx* ctx, int nparts, const mvn_qmc* qmc, const double* partials,
                           double* out3);

/* SOV estimate and its gradient (reverse mode of the per-path recurrence; not in the paper):
 *   dlogp_da, dlogp_db: device n-vectors of d log P-hat / d a_i, d b_i (either may be NULL);
 *   dlogp_dL: optional device n x n (ld) lower-triangle d log P-hat / d L_ik.
 * The reverse sweep recomputes each block's elementwise terms from the stored transformed
 * variables instead of storing them.
 * prec = MVN_FP64: every step in FP64; out3 equals mvn_sov's MVN_FP64 estimate.
 * prec = MVN_MIXED or MVN_MIXED_SIMT: the forward sweep forms the limit shifts in FP32 and keeps
 *   the transformed variables in FP32, with the elementwise step of Eq. 2 in FP64 (out3 is this
 *   sweep's estimate); the reverse sweep forms the limit shifts and the sums over later
 *   dimensions in FP32 and the elementwise derivative terms in FP64; dlogp_dL sums FP32 products
 *   within each 128-path tile and the tiles in FP64.  Workspace per 128 paths: 2 * n * 128 * 8 bytes (FP64) or
 *   * 4 bytes (mixed).
 * dlogp_dL uses the leading dimension ld of L; its strict upper part is not written.  out3 as
 * in mvn_sov.
 * Memory: the transformed variables y and the reverse sums of a 128-path tile take
 * 2 * n * 128 * (8 or 4) bytes; when all tiles together exceed the context's limit
 * (mvn_grad_set_ylimit, default 8 GiB), the tiles run in batches under that limit: a first
 * forward sweep over all paths gives the log-weights (hence every path's weight in log P-hat),
 * then each batch recomputes its forward sweep and runs its reverse sweep.  out3, dlogp_da and
 * dlogp_db are then bit-identical to the unbatched call; dlogp_dL agrees to rounding (its
 * off-diagonal sums are added batch by batch). */
mvn_status mvn_sov_grad(mvn_ctx* ctx, int n, const double* a, const double* b,
                        const double* L, int64_t ld, const mvn_qmc* qmc, mvn_prec prec,
                        double* out3, double* dlogp_da, double* dlogp_db, double* dlogp_dL);

/* Limit (bytes) of the y and reverse-sum buffers of mvn_sov_grad on this context; 0 restores
 * the default (8 GiB).  Smaller limits trade memory for one more forward sweep (see above). */
mvn_status mvn_grad_set_ylimit(mvn_ctx* ctx, int64_t bytes);

/* nprob independent problems in one launch (Alg. 1's loop of PMVN calls):
 * problem p has dimension dims[p] (host array) and limits a[off_p .. off_p + dims[p]),
 * b[...] with off_p = limit_offsets[p] (host array); its factor is the leading
 * dims[p] x dims[p] block of L_shared (ld).  out3: device double[nprob * 3].
 * Work items (problem, 128-path tile) are scheduled longest-first by a persistent kernel. */
mvn_status mvn_sov_batched(mvn_ctx* ctx, int nprob, const int* dims,
                           const int64_t* limit_offsets, const double* a, const double* b,
                           const double* L_shared, int64_t ld, const mvn_qmc* qmc,
                           mvn_prec prec, double* out3);

/* FP64 SOV estimate that allocates nothing (the paper has no counterpart; this is a service for
 * callers that cannot allocate device memory at call time -- code under a caching allocator
 * that must not see foreign cudaMalloc calls, a real-time loop where an allocation's implicit
 * synchronisation is not allowed, or an embedding that only hands over device buffers and
 * cannot create a context with its own workspace).  Same arithmetic as mvn_sov with MVN_FP64,
 * without a context:
 *   - work is enqueued on `cuda_stream` (a cudaStream_t, NULL = legacy default stream) of the
 *     current device;
 *   - all scratch lives in one fixed file-scope device array of about 10.2 MiB that every GPU
 *     which loads the library holds until the process exits;
 *   - limits: n <= 256, n_points * n_shifts <= 262144, n_shifts <= 64; larger sizes return
 *     MVN_ERR_ARG before any work is enqueued;
 *   - the first call on each device looks up the array's device address (cudaGetSymbolAddress);
 *     make that first call before any stream capture on that device.  A device reset
 *     (cudaDeviceReset) or a new primary context invalidates that address: the first call in the
 *     new context looks it up again (so it too should come before any capture);
 *   - every call shares the one array: calls that overlap on the GPU (other streams, other host
 *     threads) race and give wrong results -- serialise them;
 *   - no device-side argument check: limits with a_i > b_i or NaN give NaN results; every path
 *     with weight 0 gives out3 = {-inf, 0, 0}.
 * a, b, L, ld, qmc, out3 (device double[3]) and path_logw (optional device
 * double[n_points * n_shifts]) as in mvn_sov.  Returns MVN_OK, MVN_ERR_ARG or MVN_ERR_CUDA. */
mvn_status mvn_sov_fp64_noalloc(int n, const double* a, const double* b, const double* L,
                                int64_t ld, const mvn_qmc* qmc, double* out3, double* path_logw,
                                void* cuda_stream);

/* ------------------------------------------------------------------ posterior field (Sec. V-B) */

/* Posterior of a Gaussian field x ~ N(mu, Sigma) given noisy observations y = A x + e,
 * e ~ N(0, noise_var I), of the sites obs[0..n_obs) (A = the n_obs x n indicator matrix):
 *   Sigma_post = (Sigma^-1 + A^T A / noise_var)^-1                  (Eq. 7)
 *   mu_post    = mu + Sigma_post A^T (y - A mu) / noise_var           (Eq. 8)
 * computed without inverting Sigma, as the Schur complement that n_obs steps of the FP64 tile
 * Cholesky leave in the bordered matrix [K, .; Sigma[:, obs], Sigma; (y - mu[obs])^T, 0] with
 * K = Sigma[obs, obs] + noise_var I (the same matrices by the Woodbury identity).  The outputs
 * feed mvn_excursion (Alg. 1: Sigma_post as the covariance, mu_post in the limits).
 *   n        : number of sites; n = 0 does nothing.
 *   mu       : device double[n], prior mean; NULL = zero mean.
 *   Sigma    : device n x n, column-major, leading dimension ld >= n; lower triangle read.
 *   obs      : device int32[n_obs], site indices in [0, n); a site may appear more than once
 *              (repeated observations); n_obs = 0 gives the prior back.
 *   y        : device double[n_obs], the observations.
 *   noise_var: host, > 0 and finite.
 *   prec     : MVN_FP64 (or MVN_MIXED_SIMT): the FP64 tile Cholesky's first n_obs steps.
 *              MVN_MIXED: the same Schur complement from the tensor-core factorisation of
 *              mvn_cholesky (MVN_MIXED) run for the first n_obs columns, padded to a multiple of
 *              64 with independent unit-variance variables: the n_obs columns in double-float,
 *              then each trailing column updated once by all of them with exact 42-bit digit
 *              products and the update subtracted in FP64 (relative error ~1e-11 against ~1e-15
 *              for FP64; measured in the tests).
 *   mu_post  : device double[n] (output; may be mu itself).
 *   Sigma_post: device n x n, leading dimension ld_post >= n; lower triangle written, strict
 *              upper part untouched; may be Sigma itself (ld_post == ld).
 *   info     : host, optional.  If given, the call waits for the stream and returns the device
 *              status (MVN_ERR_NOT_PD with *info = the failing column of K; MVN_ERR_ARG with
 *              *info = the 1-based position of an index outside [0, n) in obs).
 * Workspace: (n_obs + n + 1)^2 doubles (grown on demand; MVN_MIXED also the digits of the n_obs
 * columns, ~48 (n_obs + n) n_obs bytes).  Asynchronous unless info is given.
 * Errors: MVN_ERR_ARG (sizes, pointers, noise_var), MVN_ERR_OOM, MVN_ERR_CUDA. */
mvn_status mvn_posterior(mvn_ctx* ctx, int n, const double* mu, const double* Sigma, int64_t ld,
                         int n_obs, const int32_t* obs, const double* y, double noise_var,
                         mvn_prec prec, double* mu_post, double* Sigma_post, int64_t ld_post,
                         int* info);

/* ------------------------------------------------------------------ confidence region (Alg. 1) */

/* Positive confidence region of level 1-alpha above threshold u for X ~ N(mu, Sigma):
 *   marginal[i] = P(X_i > u);  order = indices sorted by descending marginal (ties by index);
 *   L = chol(Sigma[order, order]);  F[t] = P-hat(X_{order[0..k_t)} > u) for the prefix
 *   lengths k_t = prefix_dims[t] (host array, NULL = all 1..n, then nprob = n);
 *   region[i] = 1 for i in order[0..K), K = the largest listed k_t with F[t] >= 1-alpha.
 * The prefix problems share the lattice, so every F[t] comes from one sweep over n dimensions.
 * prec: the factorisation of Sigma[order, order] and the sweep as in mvn_cholesky and mvn_sov
 * (MVN_MIXED: tensor-core Cholesky and sweep; MVN_MIXED_SIMT: FP64 Cholesky, FP32 sweep).
 * mu (n), Sigma (n x n, ld, lower triangle read) are inputs; order (int32, n), marginal (n),
 * F (nprob), region (uint8, n) are outputs.  Workspace holds the permuted factor (n x n).
 * tile: as in mvn_cholesky (accepted, not used). */
mvn_status mvn_excursion(mvn_ctx* ctx, int n, const double* mu, const double* Sigma,
                         int64_t ld, double u, double one_minus_alpha, int nprob,
                         const int* prefix_dims, const mvn_qmc* qmc, mvn_prec prec, int tile,
                         int32_t* order, double* marginal, double* F, uint8_t* region);

/* The confidence-region pipeline of mvn_excursion (marginals, order, permuted Cholesky, the
 * prefix sweep, estimates, region) captured once into a CUDA graph and replayed with one launch
 * (Alg. 1 run repeatedly on fields of one shape, e.g. successive posterior updates).
 * Arguments as in mvn_excursion.  The call runs the pipeline once eagerly (outputs valid after
 * it returns; a non-positive pivot fails the call with MVN_ERR_NOT_PD), then captures the same
 * work on a private stream.  The graph owns a private workspace, lattice table and status word,
 * so calls on ctx between launches cannot disturb it; it allocates them here (the workspace of
 * mvn_excursion for this size, plus the three index tables).
 * Every launch reads mu and Sigma from the device buffers given here (their contents may change
 * between launches) and writes order, marginal, F and region given here; these buffers must
 * outlive the graph.  Launches of one graph must not overlap (launch it on one stream).
 * Synchronous.  Errors: as mvn_excursion; MVN_ERR_CUDA if capture or instantiation fails. */
typedef struct mvn_graph mvn_graph;
mvn_status mvn_excursion_graph(mvn_ctx* ctx, int n, const double* mu, const double* Sigma,
                               int64_t ld, double u, double one_minus_alpha, int nprob,
                               const int* prefix_dims, const mvn_qmc* qmc, mvn_prec prec,
                               int32_t* order, double* marginal, double* F, uint8_t* region,
                               mvn_graph** out);
/* Enqueue one replay of the graph on the stream of the context it was created with. */
mvn_status mvn_graph_launch(mvn_graph* g);
/* Wait for that stream; return (and clear) the graph's device status word (info as in
 * mvn_sync). */
mvn_status mvn_graph_sync(mvn_graph* g, int* info);
/* Number of kernels one launch of the graph runs. */
int64_t mvn_graph_kernels(const mvn_graph* g);
/* Wait for the creating context's stream, then free the graph and everything it owns. */
mvn_status mvn_graph_destroy(mvn_graph* g);

/* ------------------------------------------------------------------ tile low-rank (Sec. III-E) */

/* Compress the lower triangle of Sigma (n x n, ld) into tile low-rank form with square tiles
 * of size `tile`: diagonal tiles dense, each off-diagonal tile Sigma_ij ~= U_ij V_ij^T with the
 * smallest rank k such that the (k+1)-th singular value is <= acc, capped at max_rank.
 * *out receives the new object (owned by the library until mvn_tlr_free).
 * max_rank_hit (host, optional): number of tiles whose rank was capped.  Synchronous. */
mvn_status mvn_tlr_compress(mvn_ctx* ctx, int n, const double* Sigma, int64_t ld, int tile,
                            double acc, int max_rank, mvn_tlr** out, int* max_rank_hit);
/* Tile low-rank Cholesky in place (dense diagonal POTRF, TRSM on the V factors, low-rank
 * updates recompressed at the object's accuracy).  info as in mvn_cholesky. */
mvn_status mvn_tlr_cholesky(mvn_ctx* ctx, mvn_tlr* tlr, int* info);
/* Expand to a dense lower matrix L (n x n, ld, FP64; strict upper part untouched). */
mvn_status mvn_tlr_to_dense(mvn_ctx* ctx, const mvn_tlr* tlr, double* L, int64_t ld);
/* ranks (host int array of length nt*(nt-1)/2, nt = ceil(n/tile)), tile (i,j), i > j, in
 * column order: (1,0),(2,0),...,(nt-1,0),(2,1),... */
mvn_status mvn_tlr_ranks(const mvn_tlr* tlr, int* ranks);
/* The SOV estimate of mvn_sov with the factor in tile low-rank form (after mvn_tlr_cholesky):
 * the limit shifts of block row r are sum_{c<r} U_rc (V_rc^T y_c) with the compressed off-diagonal
 * tiles (2 m k multiply-adds per path and tile of rank k instead of m^2), the diagonal tiles dense
 * (Alg. 2 step (c) on the TLR factor of Sec. III-E; the paper expands the factor instead).
 * a, b, qmc, out3, path_logw as in mvn_sov; the dimension is the object's n.
 * prec = MVN_FP64: FP64 shifts and step; MVN_MIXED or MVN_MIXED_SIMT: FP32 shifts and y on the CUDA
 * cores with the FP32 step of MVN_MIXED_SIMT (FP64 in the deep tails).  Workspace per resident CTA:
 * (n rounded up to tiles + tile) x 128 words.  Asynchronous; errors as mvn_sov, MVN_ERR_ARG for an
 * object that is not factored. */
mvn_status mvn_sov_tlr(mvn_ctx* ctx, const mvn_tlr* tlr, const double* a, const double* b,
                       const mvn_qmc* qmc, mvn_prec prec, double* out3, double* path_logw);
mvn_status mvn_tlr_free(mvn_tlr* tlr);

/* ------------------------------------------------------------------ autotuner (launch shapes) */

/* Launch shapes of the hot kernels (not in the paper, whose tile size is a parameter of its CPU
 * runtime).  No choice changes a result bit: the MVN_MIXED Cholesky update sums exact integers
 * in any order, and the sweeps compute every path on its own whatever the grid.
 *   chol_bulk_p, chol_tail_p: K sub-chunks (32 columns each) per work item (one CTA) of the bulk
 *     and the tail update of a block column in the MVN_MIXED Cholesky (defaults 16 and 2);
 *   sweep_ctas_per_sm: persistent grid of the sweep, CTAs per SM (tensor-core sweep 1..2,
 *     CUDA-core sweeps 1..3; default 2);
 *   from_cache: 1 if mvn_autotune took the entry from its cache file, else 0. */
typedef struct {
    int32_t chol_bulk_p;
    int32_t chol_tail_p;
    int32_t sweep_ctas_per_sm;
    int32_t from_cache;
} mvn_tune_result;

/* Pick the launch shapes for problems of dimension n with n_paths lattice paths at precision
 * prec: time every candidate on a synthetic problem of that size on the context's device (an
 * exponential covariance on a regular grid, b = 0.5; the Cholesky at order n, the sweep on the
 * same number of 128-path tiles over min(n, 2048) dimensions), keep the fastest in the context
 * (used by later calls whose n and path-tile count fall in the same power-of-two buckets) and,
 * if cache_path (host string) is not NULL, append it there as one JSON line keyed by device
 * name, SM count, precision and the two buckets.  A matching line already in cache_path is used
 * without timing.  Synchronous; allocates ~2 n^2 * 8 bytes while it runs; *out (host) receives
 * the choice.  Errors: MVN_ERR_ARG (n outside 1..65536), MVN_ERR_OOM, MVN_ERR_CUDA. */
mvn_status mvn_autotune(mvn_ctx* ctx, int n, int64_t n_paths, mvn_prec prec,
                        const char* cache_path, mvn_tune_result* out);
/* Set the launch shapes for (n, n_paths, prec) by hand (host struct; from_cache ignored). */
mvn_status mvn_tune_set(mvn_ctx* ctx, int n, int64_t n_paths, mvn_prec prec,
                        const mvn_tune_result* params);

/* ------------------------------------------------------------------ lattice tables (testing) */

/* Copy the lattice generators alpha_0..alpha_{n-1} (u64, see mvn_qmc) to the device buffer out.
 * Synchronous on first use (the table is computed on the device and cached in the context). */
mvn_status mvn_lattice_alpha(mvn_ctx* ctx, int n, uint64_t* out);
/* Write the shifts Delta_{q,i} = SplitMix64(seed, q*2^32 + i) to out[q*n + i] (device, M x n). */
mvn_status mvn_lattice_shifts(mvn_ctx* ctx, uint64_t seed, int M, int n, uint64_t* out);

/* Self-test of the tensor-core limit-update GEMM used by MVN_MIXED (Alg. 2 step (c)):
 * S (128 x 128, row-major FP32) = Y (128 x K, row-major FP64) * L (128 x K, row-major FP64)^T,
 * computed through the same per-row scaling, FP16 two-slice split, swizzled tiles, bulk-copy
 * pipeline, tcgen05 MMAs and TMEM drains as the sweep's far GEMM.  1 <= K <= 65536; the call
 * uses workspace of ~(K + 256)^2 * 8 bytes.  Asynchronous; errors via mvn_sync. */
mvn_status mvn_tc_selftest(mvn_ctx* ctx, int K, const double* Y, const double* L, float* S);

/* The elementwise step of Eq. 2 (Alg. 3's inner step) as the sweeps of precision prec run it,
 * on `count` independent inputs: a' = (a - s) / lii, b' = (b - s) / lii with the lattice point
 * w = ((W >> 11) + 1/2) 2^-53 of the 64-bit integer W; writes y (the transformed variable) and
 * delta (the factor Phi(b') - Phi(a'), 0 when it underflows).  MVN_FP64: the FP64 step of the
 * FP64 sweep; MVN_MIXED_SIMT: the FP32 step of the CUDA-core mixed sweep (s and lii rounded to
 * FP32); MVN_MIXED: the FP32-only step of the tensor-core sweep (likewise).  All arrays are
 * device arrays of `count` entries (W: uint64).  Asynchronous; errors: MVN_ERR_ARG. */
mvn_status mvn_sov_step_test(mvn_ctx* ctx, mvn_prec prec, int64_t count, const double* a,
                             const double* b, const double* s, const double* lii,
                             const uint64_t* W, double* y, double* delta);

/* Self-test of the bounded device-side waits: a kernel waits on an mbarrier that nothing
 * completes, gives up after budget_cycles (1e3 .. 4e9 SM clock cycles) and raises
 * MVN_ERR_TIMEOUT in the status word (read by mvn_sync); the context stays usable. */
mvn_status mvn_wait_selftest(mvn_ctx* ctx, int64_t budget_cycles);

#ifdef __cplusplus
}
#endif
#endif /* MVN_H */
