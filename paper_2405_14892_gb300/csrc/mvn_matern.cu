// mvn_matern.cu -- Matern covariance generation (Eq. 6) and its parameter-gradient contraction.
#include "mvn_internal.cuh"

// C(h)/sigma2 for nu in {1/2, 3/2, 5/2} (closed forms of Eq. 6's Bessel K_nu):
//   nu=1/2: e^-x;  nu=3/2: (1+x) e^-x;  nu=5/2: (1 + x + x^2/3) e^-x,  x = h / range.
__device__ __forceinline__ double matern_unit(double x, int nu2) {
    double e = exp(-x);
    if (nu2 == 1) return e;
    if (nu2 == 3) return (1.0 + x) * e;
    return (1.0 + x + x * x * (1.0 / 3.0)) * e;
}

// One block: 256 rows x 8 columns of the lower triangle, column-major writes.
__global__ void k_matern(int n, const double* __restrict__ xy, double sigma2, double inv_range,
                         int nu2, double nugget, double* __restrict__ S, int64_t ld) {
    const int i = blockIdx.x * 256 + threadIdx.x;
    const int j0 = blockIdx.y * 8;
    if (i >= n || i < j0) return;
    const double xi = xy[2 * i], yi = xy[2 * i + 1];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        int j = j0 + c;
        if (j > i || j >= n) break;
        double dx = xi - xy[2 * j], dy = yi - xy[2 * j + 1];
        double h = sqrt(dx * dx + dy * dy);
        double v = sigma2 * matern_unit(h * inv_range, nu2);
        if (i == j) v = sigma2 + nugget;
        S[i + (int64_t)j * ld] = v;
    }
}

extern "C" mvn_status mvn_matern(mvn_ctx* ctx, int n, const double* coords, double sigma2,
                                 double range, double nu, double nugget, double* Sigma,
                                 int64_t ld) {
    if (!ctx) return MVN_ERR_ARG;
    int nu2 = (int)(2.0 * nu + 0.5);
    if (n < 0 || ld < (n > 0 ? n : 1) || !(range > 0.0) || !(sigma2 > 0.0) ||
        (nu2 != 1 && nu2 != 3 && nu2 != 5) || fabs(2.0 * nu - nu2) > 1e-12 ||
        (n > 0 && (!coords || !Sigma)))
        return mvn_fail(ctx, MVN_ERR_ARG, "mvn_matern: invalid argument (nu must be 0.5, 1.5 or 2.5)");
    if (n == 0) return MVN_OK;
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    dim3 grid((n + 255) / 256, (n + 7) / 8);
    k_matern<<<grid, 256, 0, ctx->stream>>>(n, coords, sigma2, 1.0 / range, nu2, nugget, Sigma,
                                            ld);
    MVN_LAUNCHED(ctx);
    return MVN_OK;
}

// Per-block partial sums of Sbar_ij * dSigma_ij/dsigma2 and * dSigma_ij/drange (lower triangle).
//   nu=1/2: dC/dsigma2 = e^-x,        dC/da = sigma2 x e^-x / a
//   nu=3/2: dC/dsigma2 = (1+x) e^-x,  dC/da = sigma2 x^2 e^-x / a
__global__ void k_matern_grad_part(int n, const double* __restrict__ xy, double sigma2,
                                   double range, int nu2, const double* __restrict__ Sb,
                                   int64_t ld, double* __restrict__ part) {
    __shared__ double r0[256], r1[256];
    const int t = threadIdx.x;
    const int j = blockIdx.x;  // one column per block
    double s0 = 0.0, s1 = 0.0;
    const double xj = xy[2 * j], yj = xy[2 * j + 1];
    for (int i = j + t; i < n; i += 256) {
        double g = Sb[i + (int64_t)j * ld];
        double dx = xy[2 * i] - xj, dy = xy[2 * i + 1] - yj;
        double x = sqrt(dx * dx + dy * dy) / range;
        double e = exp(-x);
        double base = (nu2 == 1) ? e : (1.0 + x) * e;
        double da = (nu2 == 1) ? sigma2 * x * e / range : sigma2 * x * x * e / range;
        s0 += g * base;
        s1 += g * da;
    }
    r0[t] = s0;
    r1[t] = s1;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w) {
            r0[t] += r0[t + w];
            r1[t] += r1[t + w];
        }
        __syncthreads();
    }
    if (t == 0) {
        part[2 * j] = r0[0];
        part[2 * j + 1] = r1[0];
    }
}

__global__ void k_sum_pairs(int m, const double* __restrict__ part, double* __restrict__ out) {
    __shared__ double r0[256], r1[256];
    const int t = threadIdx.x;
    double s0 = 0.0, s1 = 0.0;
    for (int k = t; k < m; k += 256) {
        s0 += part[2 * k];
        s1 += part[2 * k + 1];
    }
    r0[t] = s0;
    r1[t] = s1;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w) {
            r0[t] += r0[t + w];
            r1[t] += r1[t + w];
        }
        __syncthreads();
    }
    if (t == 0) {
        out[0] = r0[0];
        out[1] = r1[0];
    }
}

extern "C" mvn_status mvn_matern_grad(mvn_ctx* ctx, int n, const double* coords, double sigma2,
                                      double range, double nu, const double* Sbar, int64_t ld,
                                      double* out) {
    if (!ctx) return MVN_ERR_ARG;
    int nu2 = (int)(2.0 * nu + 0.5);
    if (n < 0 || ld < (n > 0 ? n : 1) || !(range > 0.0) || (nu2 != 1 && nu2 != 3) ||
        fabs(2.0 * nu - nu2) > 1e-12 || !out || (n > 0 && (!coords || !Sbar)))
        return mvn_fail(ctx, MVN_ERR_ARG, "mvn_matern_grad: invalid argument (nu must be 0.5 or 1.5)");
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    if (n == 0) {
        MVN_CUDA(ctx, cudaMemsetAsync(out, 0, 2 * sizeof(double), ctx->stream));
        return MVN_OK;
    }
    MVN_TRY(ws_reserve(ctx, sizeof(double) * 2 * (size_t)n));
    double* part = (double*)ctx->ws;
    k_matern_grad_part<<<n, 256, 0, ctx->stream>>>(n, coords, sigma2, range, nu2, Sbar, ld, part);
    MVN_LAUNCHED(ctx);
    k_sum_pairs<<<1, 256, 0, ctx->stream>>>(n, part, out);
    MVN_LAUNCHED(ctx);
    return MVN_OK;
}
