// mvn_posterior.cu -- posterior of a Gaussian field observed with noise at some of its sites
// (Sec. V-B, Eqs. 7-8), the input of the confidence-region loop (Alg. 1).
//
// Eqs. 7-8 are written with the inverse of the n x n prior covariance.  Here nothing is inverted:
// with K = Sigma[obs, obs] + noise_var I = L_K L_K^T and T = L_K^-1 Sigma[obs, :],
//   Sigma_post = Sigma - T^T T,   mu_post = mu + T^T L_K^-1 (y - mu[obs])
// (the same matrices, by the Woodbury identity).  Both are Schur complements, and the first n_obs
// steps of the tile Cholesky leave them in the trailing block of the bordered matrix of order
// N = n_obs + n + 1 (lower triangle)
//   [ K                 .               .  ]
//   [ Sigma[:, obs]     Sigma           .  ]
//   [ (y - mu[obs])^T   0 ... 0         0  ]
// in the rows and columns n_obs .. n_obs+n-1 (Sigma_post) and in the last row (-(mu_post - mu)).
// FP64: the right-looking FP64 tile Cholesky (POTRF/TRSM/SYRK of mvn_chol.cu).  MVN_MIXED: the
// tensor-core factorisation's partial mode (mvn_chol_oz.cu): the n_obs columns (padded to a
// multiple of 64 with independent unit-variance variables) factorised in double-float with
// exact-digit updates, then every trailing column updated once by all of them on the tensor
// cores (42-bit digit products, summed exactly) and the update subtracted in FP64.
#include <math.h>

#include "mvn_internal.cuh"

mvn_status chol_f64_partial(mvn_ctx* ctx, int n, double* A, int64_t ld, int ncols);
mvn_status chol_oz_partial(mvn_ctx* ctx, int n, double* A, int64_t ld, int ncols, char* ws);
size_t chol_oz_partial_ws_bytes(int n, int ncols);

// Sigma(p, q) from the lower triangle of the symmetric prior
__device__ __forceinline__ double sym_lower(const double* __restrict__ S, int64_t ld, int p, int q) {
    return p >= q ? S[p + (int64_t)q * ld] : S[q + (int64_t)p * ld];
}

// Lower triangle of the bordered matrix W (order N = kp + n + 1, column-major, leading
// dimension ldw): thread r of column c writes W(r, c) for r >= c.  Rows and columns
// n_obs .. kp-1 are unit-variance variables independent of everything (kp = n_obs, or n_obs
// rounded up to the 64-column panels of the tensor-core factorisation); they leave every Schur
// complement unchanged.  An observation index outside [0, n) raises MVN_ERR_ARG (info =
// 1-based position in obs) and is read as nothing.  W(N-1, N-1) is set by k_post_corner.
__global__ void k_post_border(int n, int n_obs, int kp, const double* __restrict__ mu,
                              const double* __restrict__ S, int64_t ld,
                              const int* __restrict__ obs, const double* __restrict__ y,
                              double noise_var, double* __restrict__ W, int64_t ldw,
                              int* status) {
    const int64_t N = (int64_t)kp + n + 1;
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t c = blockIdx.y; c < N; c += gridDim.y) {
        if (r < c || r >= N) continue;
        double v = 0.0;
        if (c < n_obs) {
            const int oc = obs[c];
            const bool okc = oc >= 0 && oc < n;
            if (!okc) {
                if (r == c) dev_raise(status, MVN_ERR_ARG, (int)c + 1);
            } else if (r < n_obs) {                       // K = Sigma[obs, obs] + noise_var I
                const int orr = obs[r];
                if (orr >= 0 && orr < n) v = sym_lower(S, ld, orr, oc);
                if (r == c) v += noise_var;
            } else if (r < kp) {                           // padding variables
                v = 0.0;
            } else if (r < N - 1) {                        // Sigma[:, obs]
                v = sym_lower(S, ld, (int)(r - kp), oc);
            } else {                                       // border row: y - mu[obs]
                v = y[c] - (mu ? mu[oc] : 0.0);
            }
        } else if (c < kp) {                               // padding: identity
            v = (r == c) ? 1.0 : 0.0;
        } else if (r < N - 1) {                            // Sigma itself (r >= c >= kp)
            v = S[(r - kp) + (c - kp) * ld];
        }
        W[r + c * ldw] = v;
    }
}

// W(N-1, N-1) = 1 + sum_k (y_k - mu[obs_k])^2 / noise_var: the border row's part of the factor is
// L_K^-1 (y - mu[obs]), whose squared norm is at most ||y - mu[obs]||^2 / noise_var (K's
// eigenvalues are >= noise_var), so the corner bounds it like a variance bounds its row; the
// tensor-core factorisation scales the row's digits by it.  The corner takes no other part.
__global__ void k_post_corner(int n, int n_obs, const double* __restrict__ mu,
                              const int* __restrict__ obs, const double* __restrict__ y,
                              double noise_var, double* __restrict__ corner) {
    __shared__ double red[256];
    double s = 0.0;
    for (int k = threadIdx.x; k < n_obs; k += 256) {
        const int o = obs[k];
        const double d = y[k] - ((mu && o >= 0 && o < n) ? mu[o] : 0.0);
        s += d * d;
    }
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *corner = 1.0 + red[0] / noise_var;
}

// Sigma_post (lower) and mu_post from the trailing block and the border row of W.
__global__ void k_post_extract(int n, int kp, const double* __restrict__ W, int64_t ldw,
                               const double* __restrict__ mu, double* __restrict__ mu_post,
                               double* __restrict__ Sp, int64_t ldp) {
    const int64_t N = (int64_t)kp + n + 1;
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t j = blockIdx.y; j < n; j += gridDim.y) {
        if (i < j || i >= n) continue;
        Sp[i + j * ldp] = W[(kp + i) + (kp + j) * ldw];
        if (i == j) mu_post[j] = (mu ? mu[j] : 0.0) - W[(N - 1) + (kp + j) * ldw];
    }
}

extern "C" mvn_status mvn_posterior(mvn_ctx* ctx, int n, const double* mu, const double* Sigma,
                                    int64_t ld, int n_obs, const int32_t* obs, const double* y,
                                    double noise_var, mvn_prec prec, double* mu_post,
                                    double* Sigma_post, int64_t ld_post, int* info) {
    if (!ctx) return MVN_ERR_ARG;
    if (n < 0 || n_obs < 0 || (int64_t)n + n_obs + 65 > (1 << 20) || ld < (n > 0 ? n : 1) ||
        ld_post < (n > 0 ? n : 1))
        return mvn_fail(ctx, MVN_ERR_ARG, "mvn_posterior: invalid size or leading dimension");
    if (n > 0 && (!Sigma || !mu_post || !Sigma_post))
        return mvn_fail(ctx, MVN_ERR_ARG, "mvn_posterior: null matrix or output");
    if (n_obs > 0 && (!obs || !y))
        return mvn_fail(ctx, MVN_ERR_ARG, "mvn_posterior: null observations");
    if (!(noise_var > 0.0) || !isfinite(noise_var))
        return mvn_fail(ctx, MVN_ERR_ARG, "mvn_posterior: noise variance must be positive");
    if (prec != MVN_FP64 && prec != MVN_MIXED && prec != MVN_MIXED_SIMT)
        return mvn_fail(ctx, MVN_ERR_ARG, "unknown precision");
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    if (info) *info = 0;
    if (n > 0) {
        const bool tc = (prec == MVN_MIXED) && n_obs > 0;
        const int kp = tc ? (n_obs + 63) / 64 * 64 : n_obs;
        const int64_t N = (int64_t)kp + n + 1;
        const size_t wbytes = ws_round(sizeof(double) * (size_t)N * (size_t)N);
        MVN_TRY(ws_reserve(ctx, wbytes + (tc ? chol_oz_partial_ws_bytes((int)N, kp) : 0) + 1024));
        double* W = (double*)ctx->ws;
        const unsigned gy = (unsigned)(N < 65535 ? N : 65535);
        k_post_border<<<dim3((unsigned)((N + 255) / 256), gy), 256, 0, ctx->stream>>>(
            n, n_obs, kp, mu, Sigma, ld, obs, y, noise_var, W, N, ctx->d_status);
        MVN_LAUNCHED(ctx);
        k_post_corner<<<1, 256, 0, ctx->stream>>>(n, n_obs, mu, obs, y, noise_var,
                                                   W + (N - 1) + (N - 1) * N);
        MVN_LAUNCHED(ctx);
        if (tc) {
            MVN_TRY(chol_oz_partial(ctx, (int)N, W, N, kp, (char*)ctx->ws + wbytes));
        } else if (n_obs > 0) {
            MVN_TRY(chol_f64_partial(ctx, (int)N, W, N, n_obs));
        }
        const unsigned gx = (unsigned)((n + 255) / 256), gj = (unsigned)(n < 65535 ? n : 65535);
        k_post_extract<<<dim3(gx, gj), 256, 0, ctx->stream>>>(n, kp, W, N, mu, mu_post,
                                                               Sigma_post, ld_post);
        MVN_LAUNCHED(ctx);
    }
    if (info) return mvn_sync(ctx, info);
    return MVN_OK;
}
