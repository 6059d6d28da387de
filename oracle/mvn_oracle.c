/*
 * mvn_oracle.c -- plain FP64 CPU oracle for the SOV estimator of MVN probabilities.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct reference that the
 * GPU library is checked against.  Only the tests, the smoke check and the bench's CPU
 * baseline leg may load it.  It shares no code, header or table with the CUDA library.
 *
 * What it follows (paper: Cao/Abdulah et al., "Parallel approximations for high-dimensional
 * multivariate normal probability computation in confidence region detection applications"):
 *   - Phi, Q, Phi^-1 ........ Sec. III-B, Eq. 2 (the univariate normal CDF and its inverse).
 *                              Phi^-1 is Wichura's AS241 (PPND16, Applied Statistics 1988),
 *                              written here from the published rational approximations.
 *   - Cholesky .............. Alg. 1 step "L <- dpotrf(Sigma)": plain column (left-looking)
 *                              unblocked factorisation, Sigma = L L^T, lower.
 *   - SOV per-path weights .. Eq. 2 / Eq. 3 and Alg. 3 (the QMC tile kernel), one path at a
 *                              time, dimensions in order, with the log of the running product.
 *   - SOV adjoint ........... reverse-mode differentiation of the same per-path recurrence
 *                              (not in the paper; plain chain rule of Eq. 2).
 *   - Cholesky adjoint ...... reverse of the same column Cholesky loop (Murray 2016, arXiv
 *                              1602.07527, unblocked reverse mode), written from the forward loop.
 *   - lattice shifts ......... SplitMix64 (Steele, Lea, Flood 2014) output function applied
 *                              to a counter; the point rule is the rank-1 Richtmyer lattice.
 *
 * Readings of the paper used here (the paper is ambiguous at these places):
 *   - Eq. 3 prints (b'_i - a'_i); the factor is read as Phi(b'_i) - Phi(a'_i) (consistent with
 *     Eq. 2 and Alg. 3).
 *   - Alg. 3's Y update omits "Phi(a') +"; Eq. 2's form y = Phi^-1(Phi(a') + w (Phi(b')-Phi(a')))
 *     is used.  The running product starts at 1 (log-weight 0).
 *   - The uniforms R(i,j) of Alg. 2 are replaced by randomly shifted rank-1 lattice points
 *     w = frac(j * alpha_i + Delta_{q,i}) in 64-bit fixed point.
 *   - Tail-stable difference: for a' > 0 both tails are taken from the upper side,
 *     Delta = Q(a') - Q(b') and y = -Phi^-1(Q(a') - w Delta); otherwise
 *     Delta = Phi(b') - Phi(a') and y = Phi^-1(Phi(a') + w Delta).
 *   - If Delta underflows to 0 the path weight is 0 (log-weight -inf) and y is set to the
 *     finite limit (a' if a' > 0, else b') so no NaN is produced.
 *   - An argument of Phi^-1 rounded to exactly 0 or 1 is moved to the nearest interior double.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_SQRT1_2 0.70710678118654752440
#define ORC_INV_SQRT_2PI 0.39894228040143267794

/* ---------------------------------------------------------------- univariate normal */

/* Phi(x) = P(Z <= x) = erfc(-x / sqrt 2) / 2   (Table I: "Phi(x)") */
double orc_Phi(double x) { return 0.5 * erfc(-x * ORC_SQRT1_2); }

/* Q(x) = P(Z > x) = 1 - Phi(x), evaluated without cancellation in the upper tail. */
double orc_Q(double x) { return 0.5 * erfc(x * ORC_SQRT1_2); }

/* standard normal density */
double orc_phi(double x) { return ORC_INV_SQRT_2PI * exp(-0.5 * x * x); }

/* Phi^-1(p): Wichura's algorithm AS241 (PPND16), about 1e-16 relative accuracy.
 * Central region |p - 1/2| <= 0.425: rational function of r = 0.180625 - q^2;
 * tails: rational function of r = sqrt(-log(min(p, 1-p))), split at r = 5. */
double orc_Phinv(double p) {
    if (!(p > 0.0)) return (p == 0.0) ? -INFINITY : NAN;
    if (!(p < 1.0)) return (p == 1.0) ? INFINITY : NAN;
    double q = p - 0.5;
    if (fabs(q) <= 0.425) {
        double r = 0.180625 - q * q;
        double num = (((((((2.5090809287301226727e+3 * r + 3.3430575583588128105e+4) * r +
                           6.7265770927008700853e+4) * r + 4.5921953931549871457e+4) * r +
                         1.3731693765509461125e+4) * r + 1.9715909503065514427e+3) * r +
                       1.3314166789178437745e+2) * r + 3.3871328727963666080e+0);
        double den = (((((((5.2264952788528545610e+3 * r + 2.8729085735721942674e+4) * r +
                           3.9307895800092710610e+4) * r + 2.1213794301586595867e+4) * r +
                         5.3941960214247511077e+3) * r + 6.8718700749205790830e+2) * r +
                       4.2313330701600911252e+1) * r + 1.0);
        return q * num / den;
    }
    double r = (q < 0.0) ? p : 1.0 - p;
    r = sqrt(-log(r));
    double val;
    if (r <= 5.0) {
        r -= 1.6;
        double num = (((((((7.74545014278341407640e-4 * r + 2.27238449892691845833e-2) * r +
                           2.41780725177450611770e-1) * r + 1.27045825245236838258e+0) * r +
                         3.64784832476320460504e+0) * r + 5.76949722146069140550e+0) * r +
                       4.63033784615654529590e+0) * r + 1.42343711074968357734e+0);
        double den = (((((((1.05075007164441684324e-9 * r + 5.47593808499534494600e-4) * r +
                           1.51986665636164571966e-2) * r + 1.48103976427480074590e-1) * r +
                         6.89767334985100004550e-1) * r + 1.67638483018380384940e+0) * r +
                       2.05319162663775882187e+0) * r + 1.0);
        val = num / den;
    } else {
        r -= 5.0;
        double num = (((((((2.01033439929228813265e-7 * r + 2.71155556874348757815e-5) * r +
                           1.24266094738807843860e-3) * r + 2.65321895265761230930e-2) * r +
                         2.96560571828504891230e-1) * r + 1.78482653991729133580e+0) * r +
                       5.46378491116411436990e+0) * r + 6.65790464350110377720e+0);
        double den = (((((((2.04426310338993978564e-15 * r + 1.42151175831644588870e-7) * r +
                           1.84631831751005468180e-5) * r + 7.86869131145613259100e-4) * r +
                         1.48753612908506148525e-2) * r + 1.36929880922735805310e-1) * r +
                       5.99832206555887937690e-1) * r + 1.0);
        val = num / den;
    }
    return (q < 0.0) ? -val : val;
}

void orc_Phi_vec(int64_t n, const double* x, double* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = orc_Phi(x[i]);
}
void orc_Q_vec(int64_t n, const double* x, double* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = orc_Q(x[i]);
}
void orc_Phinv_vec(int64_t n, const double* p, double* out) {
    for (int64_t i = 0; i < n; ++i) out[i] = orc_Phinv(p[i]);
}

/* ---------------------------------------------------------------- lattice shifts */

/* SplitMix64 output for counter c under key `seed`:
 *   x = seed + (c + 1) * 0x9E3779B97F4A7C15 (mod 2^64), then the SplitMix64 finaliser.
 * The shift for shift index q and dimension i uses c = q * 2^32 + i. */
uint64_t orc_splitmix64(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* Delta[q * n + i] for q < M, i < n */
void orc_shifts(uint64_t seed, int M, int n, uint64_t* out) {
    for (int q = 0; q < M; ++q)
        for (int i = 0; i < n; ++i)
            out[(int64_t)q * n + i] = orc_splitmix64(seed, ((uint64_t)q << 32) | (uint64_t)i);
}

/* w = ((W >> 11) + 1/2) 2^-53 with W = j * alpha + Delta (mod 2^64); j = 1..N_s */
static double orc_point(uint64_t j, uint64_t alpha, uint64_t delta) {
    uint64_t W = j * alpha + delta;
    return ((double)(W >> 11) + 0.5) * 0x1p-53;
}

void orc_points(int64_t count, const uint64_t* j, const uint64_t* alpha, const uint64_t* delta,
                double* out) {
    for (int64_t t = 0; t < count; ++t) out[t] = orc_point(j[t], alpha[t], delta[t]);
}

/* ---------------------------------------------------------------- Cholesky */

/* In-place lower Cholesky of the column-major n x n matrix A (leading dimension ld).
 * Column j: L_jj = sqrt(A_jj - sum_{k<j} L_jk^2); L_ij = (A_ij - sum_{k<j} L_ik L_jk) / L_jj.
 * Only the lower triangle is read and written.  Returns 0, or the 1-based index of the first
 * column whose pivot is not positive (LAPACK convention).
 * The entries L_ij of one column (i > j) are independent of each other; with OpenMP they are
 * shared among threads, each computed by the same loop in the same order as serially, so the
 * result does not depend on the thread count. */
int orc_cholesky(int n, double* A, int64_t ld) {
    for (int j = 0; j < n; ++j) {
        double d = A[j + (int64_t)j * ld];
        for (int k = 0; k < j; ++k) {
            double l = A[j + (int64_t)k * ld];
            d -= l * l;
        }
        if (!(d > 0.0)) return j + 1;
        double ljj = sqrt(d);
        A[j + (int64_t)j * ld] = ljj;
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if ((int64_t)(n - j) * j > 200000)
#endif
        for (int i = j + 1; i < n; ++i) {
            double s = A[i + (int64_t)j * ld];
            for (int k = 0; k < j; ++k) s -= A[i + (int64_t)k * ld] * A[j + (int64_t)k * ld];
            A[i + (int64_t)j * ld] = s / ljj;
        }
    }
    return 0;
}

/* Reverse mode of orc_cholesky.  On entry Lbar holds dF/dL (lower triangle); on exit it
 * holds dF/dA for the lower-triangle entries A_ij (i >= j) that the factorisation reads.
 * Derived by running the column loop above backwards (j = n-1 .. 0; in each column the
 * off-diagonal entries first, then the pivot). */
void orc_cholesky_grad(int n, const double* L, int64_t ld, double* Lbar) {
#define LL(i, k) L[(i) + (int64_t)(k) * ld]
#define LB(i, k) Lbar[(i) + (int64_t)(k) * ld]
    for (int j = n - 1; j >= 0; --j) {
        double ljj = LL(j, j);
        for (int i = n - 1; i > j; --i) {
            /* forward: L_ij = (A_ij - sum_{k<j} L_ik L_jk) / L_jj */
            double g = LB(i, j) / ljj; /* d/d(numerator) */
            for (int k = 0; k < j; ++k) {
                LB(i, k) -= g * LL(j, k);
                LB(j, k) -= g * LL(i, k);
            }
            LB(j, j) -= g * LL(i, j);
            LB(i, j) = g; /* = dF/dA_ij */
        }
        /* forward: L_jj = sqrt(A_jj - sum_{k<j} L_jk^2) */
        double g = LB(j, j) / (2.0 * ljj); /* d/d(radicand) */
        for (int k = 0; k < j; ++k) LB(j, k) -= 2.0 * g * LL(j, k);
        LB(j, j) = g;
    }
#undef LL
#undef LB
}

/* ---------------------------------------------------------------- SOV, one path */

/* The argument of Phi^-1 in Eq. 2 lies strictly inside (0,1) for w in (0,1); rounding can push
 * it to exactly 0 or 1 (probability ~2^-53 per step), which would make y infinite.  Such a
 * value is moved to the nearest interior double. */
static double orc_interior(double p) {
    if (p <= 0.0) return 4.9406564584124654e-324;
    if (p >= 1.0) return 0.99999999999999988898; /* 1 - 2^-53 */
    return p;
}

/* One dimension of Eq. 2 with the tail-stable branches, given the standardised limits a', b'
 * and the path's uniform w: returns Delta = Phi(b') - Phi(a') and writes y.
 *   a' > 0 : Delta = Q(a') - Q(b'),    y = -Phi^-1(Q(a') - w Delta)
 *   else   : Delta = Phi(b') - Phi(a'), y =  Phi^-1(Phi(a') + w Delta)
 * Delta = 0 (underflow) gives y = the finite limit (a' if a' > 0, else b'). */
static double orc_step(double ap, double bp, double w, double* y) {
    double delta;
    if (ap > 0.0) {
        double qa = orc_Q(ap), qb = orc_Q(bp);
        delta = qa - qb;
        *y = (delta > 0.0) ? -orc_Phinv(orc_interior(qa - w * delta)) : ap;
    } else {
        double pa = orc_Phi(ap), pb = orc_Phi(bp);
        delta = pb - pa;
        *y = (delta > 0.0) ? orc_Phinv(orc_interior(pa + w * delta)) : bp;
    }
    return delta;
}

/* The step above on `count` independent inputs, each given as the limits a, b, the limit shift
 * s, the diagonal entry L_ii and the lattice integer W (w = ((W >> 11) + 1/2) 2^-53):
 * a' = (a - s) / L_ii, b' = (b - s) / L_ii; writes y and Delta. */
void orc_sov_step_vec(int64_t count, const double* a, const double* b, const double* s,
                      const double* lii, const uint64_t* W, double* y, double* delta) {
    for (int64_t t = 0; t < count; ++t) {
        double w = ((double)(W[t] >> 11) + 0.5) * 0x1p-53;
        delta[t] = orc_step((a[t] - s[t]) / lii[t], (b[t] - s[t]) / lii[t], w, &y[t]);
    }
}

/* One SOV path (Eq. 2, Alg. 3): returns the log-weight sum_i log(Phi(b'_i) - Phi(a'_i)).
 * w[i] are the path's uniforms, y[i] receives the transformed variables; ap_out, bp_out and
 * d_out (optional) receive a'_i, b'_i and Delta_i.
 * If kprefix != NULL, logw_prefix[t] receives the log-weight after kprefix[t] dimensions. */
static double orc_sov_one(int n, const double* a, const double* b, const double* L, int64_t ld,
                          const double* w, double* y, double* ap_out, double* bp_out,
                          double* d_out, int nprefix, const int* kprefix, double* logw_prefix) {
    double logw = 0.0;
    int t = 0;
    for (int i = 0; i < n; ++i) {
        while (t < nprefix && kprefix[t] == i) logw_prefix[t++] = logw;
        double s = 0.0;
        for (int k = 0; k < i; ++k) s += L[i + (int64_t)k * ld] * y[k];
        double lii = L[i + (int64_t)i * ld];
        double ap = (a[i] - s) / lii; /* -inf stays -inf */
        double bp = (b[i] - s) / lii;
        double delta = orc_step(ap, bp, w[i], &y[i]);
        logw += (delta > 0.0) ? log(delta) : -INFINITY;
        if (ap_out) ap_out[i] = ap;
        if (bp_out) bp_out[i] = bp;
        if (d_out) d_out[i] = delta;
    }
    while (t < nprefix && kprefix[t] == n) logw_prefix[t++] = logw;
    return logw;
}

/* Per-path log-weights for paths p in [p0, p1) of the shifted lattice rule with M shifts and
 * Ns points per shift (path p = q * Ns + (j - 1), j = 1..Ns).
 *   alpha[i]      : lattice generator of dimension i (u64 fixed point)
 *   delta[q*n+i]  : random shift of shift q, dimension i (u64 fixed point)
 *   logw[p - p0]  : output log-weights
 *   Y (optional)  : Y[(p - p0) * n + i] receives y_i of the path
 *   D (optional)  : D[(p - p0) * n + i] receives the factor Delta_i of the path
 *   kprefix/nprefix (optional): sorted prefix lengths; logw_prefix[(p-p0)*nprefix + t]. */
void orc_sov_paths(int n, const double* a, const double* b, const double* L, int64_t ld,
                   int64_t Ns, const uint64_t* alpha, const uint64_t* delta, int64_t p0,
                   int64_t p1, double* logw, double* Y, double* D, int nprefix,
                   const int* kprefix, double* logw_prefix, int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
#endif
    {
        double* w = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        double* y = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
        for (int64_t p = p0; p < p1; ++p) {
            int64_t q = p / Ns;
            uint64_t j = (uint64_t)(p - q * Ns) + 1u;
            for (int i = 0; i < n; ++i) w[i] = orc_point(j, alpha[i], delta[q * n + i]);
            double* lp = logw_prefix ? logw_prefix + (p - p0) * nprefix : NULL;
            logw[p - p0] = orc_sov_one(n, a, b, L, ld, w, y, NULL, NULL,
                                       D ? D + (p - p0) * n : NULL, lp ? nprefix : 0, kprefix,
                                       lp);
            if (Y) memcpy(Y + (p - p0) * n, y, sizeof(double) * (size_t)n);
        }
        free(w);
        free(y);
    }
}

/* ---------------------------------------------------------------- SOV adjoint */

/* Reverse mode of orc_sov_one for one path, weighted by `weight`:
 * accumulates weight * d(logw)/da into ga, d/db into gb and d/dL into gL (lower, ld).
 * Chain rule of Eq. 2 (per dimension i, reverse order):
 *   ybar_i   = sum_{j>i} sbar_j L_ji
 *   a'bar_i  = dlog(Delta_i)/da'_i + ybar_i dy_i/da'_i    (likewise b')
 *   abar_i   = a'bar_i / L_ii,  bbar_i = b'bar_i / L_ii
 *   sbar_i   = -(a'bar_i + b'bar_i) / L_ii
 *   Lbar_ii  = -(a'bar_i a'_i + b'bar_i b'_i) / L_ii
 *   Lbar_ik += sbar_i y_k, ybar_k += sbar_i L_ik  (k < i)
 * with dlog(Delta)/da' = -phi(a')/Delta, dlog(Delta)/db' = phi(b')/Delta,
 * dy/da' = (1 - w) phi(a') / phi(y), dy/db' = w phi(b') / phi(y); terms of an infinite limit
 * are zero.  A path with weight 0 (Delta underflow) contributes nothing. */
static void orc_sov_grad_one(int n, const double* a, const double* b, const double* L,
                             int64_t ld, const double* w, const double* y, const double* ap,
                             const double* bp, double weight, double* ybar, double* ga,
                             double* gb, double* gL) {
    for (int i = 0; i < n; ++i) ybar[i] = 0.0;
    for (int i = n - 1; i >= 0; --i) {
        double lii = L[i + (int64_t)i * ld];
        double delta = (ap[i] > 0.0) ? orc_Q(ap[i]) - orc_Q(bp[i]) : orc_Phi(bp[i]) - orc_Phi(ap[i]);
        double phia = isinf(ap[i]) ? 0.0 : orc_phi(ap[i]);
        double phib = isinf(bp[i]) ? 0.0 : orc_phi(bp[i]);
        double phiy = orc_phi(y[i]);
        double apbar = -phia / delta + ybar[i] * (1.0 - w[i]) * phia / phiy;
        double bpbar = phib / delta + ybar[i] * w[i] * phib / phiy;
        double sbar = -(apbar + bpbar) / lii;
        ga[i] += weight * apbar / lii;
        gb[i] += weight * bpbar / lii;
        double lbar_ii = 0.0;
        if (phia != 0.0) lbar_ii -= apbar * ap[i];
        if (phib != 0.0) lbar_ii -= bpbar * bp[i];
        if (gL) gL[i + (int64_t)i * ld] += weight * lbar_ii / lii;
        for (int k = 0; k < i; ++k) {
            if (gL) gL[i + (int64_t)k * ld] += weight * sbar * y[k];
            ybar[k] += sbar * L[i + (int64_t)k * ld];
        }
    }
}

/* Gradient of log P-hat = log(mean_p exp(logw_p)) over all M*Ns paths:
 *   d log P-hat = sum_p softmax(logw)_p d logw_p.
 * weights[p] = softmax weights (computed by the caller from a forward pass).
 * ga, gb (n) and gL (n x n lower, ld; may be NULL) are accumulated (caller zeroes them).
 * Serial over paths so that the sums are accumulated in a fixed order. */
void orc_sov_grad(int n, const double* a, const double* b, const double* L, int64_t ld,
                  int64_t Ns, int64_t Ntot, const uint64_t* alpha, const uint64_t* delta,
                  const double* weights, double* ga, double* gb, double* gL) {
    double* w = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* y = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* ap = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* bp = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double* ybar = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int64_t p = 0; p < Ntot; ++p) {
        if (!(weights[p] > 0.0)) continue;
        int64_t q = p / Ns;
        uint64_t j = (uint64_t)(p - q * Ns) + 1u;
        for (int i = 0; i < n; ++i) w[i] = orc_point(j, alpha[i], delta[q * n + i]);
        orc_sov_one(n, a, b, L, ld, w, y, ap, bp, NULL, 0, NULL, NULL);
        orc_sov_grad_one(n, a, b, L, ld, w, y, ap, bp, weights[p], ybar, ga, gb, gL);
    }
    free(w);
    free(y);
    free(ap);
    free(bp);
    free(ybar);
}

/* ---------------------------------------------------------------- variable reordering */

/* Cholesky factorisation with the univariate variable reordering of Gibson, Glasbey and Elston
 * (1994), as given by Genz and Bretz (2009, Sec. 4.1.3): a variant of the SOV estimator of
 * Eq. 2 that is not in the paper (the integrand is unchanged in expectation, its variance drops).
 * Step i chooses, among the variables not yet placed, the one whose conditional interval
 * probability Phi(b'_j) - Phi(a'_j) is smallest, where a'_j = (a_j - s_j)/sqrt(d_j),
 * b'_j = (b_j - s_j)/sqrt(d_j), d_j = Sigma_jj - sum_{k<i} L_jk^2 (conditional variance) and
 * s_j = sum_{k<i} L_jk y_k with y_k = E[Z | a'_k < Z < b'_k] of the variables already placed
 * (the truncated-normal mean (phi(a') - phi(b')) / (Phi(b') - Phi(a'))); ties go to the
 * variable placed earliest in the current order.  The chosen variable is swapped into place i and
 * column i of the factor of the permuted matrix is formed.
 *   S    : full symmetric n x n column-major (ld), overwritten (permuted, unspecified)
 *   L    : n x n column-major (ld), receives the lower factor of Sigma[perm, perm]
 *   a, b : overwritten by a[perm], b[perm];  perm[i] = original index of the i-th variable
 * Returns 0, or the 1-based step whose chosen conditional variance is not positive. */
static double orc_interval_prob(double ap, double bp) {
    return (ap > 0.0) ? orc_Q(ap) - orc_Q(bp) : orc_Phi(bp) - orc_Phi(ap);
}

int orc_cholesky_reorder(int n, double* S, double* L, int64_t ld, double* a, double* b,
                         int* perm) {
#define SS(i, j) S[(i) + (int64_t)(j) * ld]
#define LL(i, j) L[(i) + (int64_t)(j) * ld]
    double* y = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) perm[i] = i;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) LL(i, j) = 0.0;
    for (int i = 0; i < n; ++i) {
        int best = -1;
        double best_p = 0.0;
        for (int j = i; j < n; ++j) {
            double d = SS(j, j), s = 0.0;
            for (int k = 0; k < i; ++k) {
                d -= LL(j, k) * LL(j, k);
                s += LL(j, k) * y[k];
            }
            if (!(d > 0.0)) continue;
            double sd = sqrt(d);
            double pj = orc_interval_prob((a[j] - s) / sd, (b[j] - s) / sd);
            if (best < 0 || pj < best_p) {
                best = j;
                best_p = pj;
            }
        }
        if (best < 0) {
            free(y);
            return i + 1;
        }
        if (best != i) { /* swap variables i and best */
            int p = best, tq;
            double t;
            for (int k = 0; k < n; ++k) { t = SS(i, k); SS(i, k) = SS(p, k); SS(p, k) = t; }
            for (int k = 0; k < n; ++k) { t = SS(k, i); SS(k, i) = SS(k, p); SS(k, p) = t; }
            for (int k = 0; k < i; ++k) { t = LL(i, k); LL(i, k) = LL(p, k); LL(p, k) = t; }
            t = a[i]; a[i] = a[p]; a[p] = t;
            t = b[i]; b[i] = b[p]; b[p] = t;
            tq = perm[i]; perm[i] = perm[p]; perm[p] = tq;
        }
        /* column i of the factor of the permuted matrix (the column loop of orc_cholesky) */
        double d = SS(i, i), s = 0.0;
        for (int k = 0; k < i; ++k) {
            d -= LL(i, k) * LL(i, k);
            s += LL(i, k) * y[k];
        }
        double lii = sqrt(d);
        LL(i, i) = lii;
        for (int j = i + 1; j < n; ++j) {
            double v = SS(j, i);
            for (int k = 0; k < i; ++k) v -= LL(j, k) * LL(i, k);
            LL(j, i) = v / lii;
        }
        /* the truncated-normal mean of the placed variable; an interval probability that
         * underflows takes the finite limit (the reading used for Delta = 0 in Eq. 2) */
        double ap = (a[i] - s) / lii, bp = (b[i] - s) / lii;
        double den = orc_interval_prob(ap, bp);
        double pa = isinf(ap) ? 0.0 : orc_phi(ap), pb = isinf(bp) ? 0.0 : orc_phi(bp);
        y[i] = (den > 0.0) ? (pa - pb) / den : ((ap > 0.0) ? ap : bp);
    }
    free(y);
    return 0;
#undef SS
#undef LL
}
