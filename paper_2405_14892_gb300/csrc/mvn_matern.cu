// mvn_matern.cu -- Matern covariance generation (Eq. 6) and its parameter-gradient contraction.
#include "mvn_internal.cuh"

// C(h)/sigma2 for nu in {1/2, 3/2, 5/2} (closed forms of Eq. 6's Bessel K_nu):
//   nu=1/2: e^-x;  nu=3/2: (1+x) e^-x;  nu=5/2: (1 + x + x^2/3) e^-x,  x = h / range.
// ---------------------------------------------------------------- double-float arithmetic
// GB300's FP64 pipe runs at ~1/64 of FP32, so the distance's square root and the exponential run
// in double-float (FP32 pairs, Dekker 1971; ~48 bits): the squared distance is formed in FP64
// (exact differences), everything after it in pairs.
struct MF {
    float hi, lo;
};
__device__ __forceinline__ MF mf_norm(float h, float l) {
    const float s = h + l;
    return MF{s, l - (s - h)};
}
__device__ __forceinline__ MF mf_from(double x) {
    const float h = __double2float_rn(x);
    return MF{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double mf_to(MF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ MF mf_mul(MF a, MF b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return mf_norm(p, e);
}
__device__ __forceinline__ MF mf_add(MF a, MF b) {
    const float s = a.hi + b.hi;
    const float bp = s - a.hi;
    const float e = (a.hi - (s - bp)) + (b.hi - bp);
    return mf_norm(s, e + a.lo + b.lo);
}
__device__ __forceinline__ MF mf_sqrt(MF d) {  // sqrtf, then one Newton correction
    if (!(d.hi > 0.0f)) return MF{0.0f, 0.0f};
    const float s0 = sqrtf(d.hi);
    const float p = s0 * s0;
    const float pe = fmaf(s0, s0, -p);
    const float diff = ((d.hi - p) - pe) + d.lo;
    return mf_norm(s0, diff * (0.5f / s0));
}
// e^-x = 2^-k e^-r for x >= 0: Cody-Waite reduction x = k ln 2 + r, |r| <= ln 2 / 2, with
// ln 2 = c1 + c2 + c3 (c1 with a short mantissa; each k c_i formed exactly as a pair), then
// e^-r = (e^u)^8 with u = -r / 8 (|u| < 0.044) from the Taylor polynomial of degree 7 (truncation
// below 4e-16 relative; three squarings multiply the relative error by 8).  Returns the pair
// e^-r; the caller applies 2^-k in FP64 (no FP32 underflow).
__device__ __forceinline__ MF mf_exp_neg_red(MF x, int& k) {
    const float kf = rintf(x.hi * 1.44269504f);  // x / ln 2
    k = (int)kf;
    const float c1 = 0.693145751953125f;
    const float c2 = 1.428606765330187e-06f;
    const float c3 = 5.497923148104107e-14f;
    MF r = x;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const float c = (i == 0) ? c1 : ((i == 1) ? c2 : c3);
        const float p = kf * c;
        r = mf_add(r, MF{-p, -fmaf(kf, c, -p)});
    }
    const MF u{-r.hi * 0.125f, -r.lo * 0.125f};
    MF q{1.0f, 0.0f};  // Horner: q = 1 + (u / m) q, m = 7 .. 1
#pragma unroll
    for (int m = 7; m >= 1; --m) {
        const float fm = (float)m;
        const float uh = u.hi / fm;
        const float ul = (fmaf(-uh, fm, u.hi) + u.lo) / fm;  // u / m as a pair
        q = mf_add(MF{1.0f, 0.0f}, mf_mul(q, MF{uh, ul}));
    }
    q = mf_mul(q, q);
    q = mf_mul(q, q);
    return mf_mul(q, q);
}

// Exact difference of two double-float numbers as a pair (two-sum of the high parts, then the
// low parts added).
__device__ __forceinline__ MF mf_sub(MF a, MF b) { return mf_add(a, MF{-b.hi, -b.lo}); }

// Coordinates as double-float pairs (x_hi, x_lo, y_hi, y_lo): the site differences are then formed
// on the FP32 pipe; a pair keeps 48 bits of each coordinate (|x| <= 1 here: 4e-15 absolute).
__global__ void k_coords_df(int n, const double* __restrict__ xy, float4* __restrict__ cp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const MF x = mf_from(xy[2 * i]), y = mf_from(xy[2 * i + 1]);
    cp[i] = make_float4(x.hi, x.lo, y.hi, y.lo);
}

// One block per lower 128 x 128 tile (ti >= tj, linear index over the triangle): thread t owns
// row i = 128 ti + t and walks the tile's 128 columns (column-major writes, coalesced over the
// rows).  Everything up to the final value runs in FP32 pairs; the FP64 pipe (~1/64 of FP32 on
// this GPU) only forms the output double (two conversions and one add) and, where e^-x would
// leave FP32's range, applies 2^-k.
__global__ void __launch_bounds__(128) k_matern(int n, const float4* __restrict__ cp,
                                                double sigma2, double inv_range, int nu2,
                                                double nugget, double* __restrict__ S,
                                                int64_t ld) {
    __shared__ float4 cj[128];
    const int x = blockIdx.x;
    int ti = (int)((sqrt(8.0 * x + 1.0) - 1.0) * 0.5);
    while ((ti + 1) * (ti + 2) / 2 <= x) ++ti;
    while (ti * (ti + 1) / 2 > x) --ti;
    const int tj = x - ti * (ti + 1) / 2;
    const int t = threadIdx.x;
    const int j0 = tj * 128;
    if (j0 + t < n) cj[t] = cp[j0 + t];
    __syncthreads();
    const int i = ti * 128 + t;
    if (i >= n) return;
    const float4 ci = cp[i];
    const MF xi{ci.x, ci.y}, yi{ci.z, ci.w};
    const MF sg = mf_from(sigma2), ir = mf_from(inv_range);
    const int jn = min(128, min(n - j0, i - j0 + 1));
    for (int c = 0; c < jn; ++c) {
        const int j = j0 + c;
        double out;
        if (i == j) {
            out = sigma2 + nugget;
        } else {
            const float4 cc = cj[c];
            const MF dx = mf_sub(xi, MF{cc.x, cc.y}), dy = mf_sub(yi, MF{cc.z, cc.w});
            const MF xx = mf_mul(mf_sqrt(mf_add(mf_mul(dx, dx), mf_mul(dy, dy))), ir);
            out = 0.0;
            if (xx.hi < 700.0f) {
                int k;
                const MF e = mf_exp_neg_red(xx, k);
                MF poly{1.0f, 0.0f};
                if (nu2 >= 3) poly = mf_add(poly, xx);
                if (nu2 == 5)
                    poly = mf_add(poly, mf_mul(mf_mul(xx, xx),
                                               MF{0.3333333432674408f, -9.934107758624577e-09f}));
                MF v = mf_mul(sg, mf_mul(poly, e));
                if (k <= 60 && fabsf(v.hi) >= 0x1p-40f) {  // 2^-k in FP32: both parts stay normal
                    const float sc = __int_as_float((127 - k) << 23);
                    out = (double)(v.hi * sc) + (double)(v.lo * sc);
                } else {
                    out = mf_to(v) * __longlong_as_double((long long)(1023 - k) << 52);
                }
            }
        }
        S[i + (int64_t)j * ld] = out;
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
    MVN_TRY(ws_reserve(ctx, sizeof(float4) * (size_t)n + 1024));
    float4* cp = (float4*)ctx->ws;
    k_coords_df<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, coords, cp);
    MVN_LAUNCHED(ctx);
    const int64_t T = (n + 127) / 128;
    k_matern<<<(unsigned)(T * (T + 1) / 2), 128, 0, ctx->stream>>>(n, cp, sigma2, 1.0 / range,
                                                                  nu2, nugget, Sigma, ld);
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
