// mvn_sov_step.cuh -- one dimension of the SOV recurrence (Eq. 2) in FP64 and in FP32, and the
// running product of the per-dimension probabilities (Eq. 3) kept as mantissa * 2^exponent.
#pragma once
#include <math.h>
#include <stdint.h>

// ---------------------------------------------------------------- FP64 elementwise step

__device__ __forceinline__ double Phi_d(double x) { return 0.5 * erfc(-x * 0.70710678118654752440); }
__device__ __forceinline__ double Q_d(double x) { return 0.5 * erfc(x * 0.70710678118654752440); }
// keep the argument of Phi^-1 strictly inside (0,1) (rounding can reach 0 or 1 exactly)
__device__ __forceinline__ double interior_d(double p) {
    return p <= 0.0 ? 4.9406564584124654e-324 : (p >= 1.0 ? 0.99999999999999988898 : p);
}

// One dimension of Eq. 2 in FP64 with the tail-stable branches:
//   a' > 0 : Delta = Q(a') - Q(b'),   y = -Phi^-1(Q(a') - w Delta)
//   else   : Delta = Phi(b') - Phi(a'), y =  Phi^-1(Phi(a') + w Delta)
// Delta == 0 gives y = the finite limit.  Returns y, writes Delta.
__device__ __forceinline__ double sov_step_f64(double ai, double bi, double s, double lii,
                                               double w, double& delta) {
    const double ap = (ai - s) / lii, bp = (bi - s) / lii;
    double y;
    if (ap > 0.0) {
        const double qa = Q_d(ap);
        const double qb = (bp == INFINITY) ? 0.0 : Q_d(bp);
        delta = qa - qb;
        y = (delta > 0.0) ? -normcdfinv(interior_d(qa - w * delta)) : ap;
    } else {
        const double pa = (ap == -INFINITY) ? 0.0 : Phi_d(ap);
        const double pb = (bp == INFINITY) ? 1.0 : Phi_d(bp);
        delta = pb - pa;
        y = (delta > 0.0) ? normcdfinv(interior_d(pa + w * delta)) : bp;
    }
    return y;
}

// Running product of the Delta factors as prod * 2^ex (log only at the end / at prefixes).
struct LogProd {
    double prod = 1.0;
    int ex = 0;
    __device__ __forceinline__ void mul(double d) {
        if (d < 0x1p-400) {
            if (!(d > 0.0)) {
                prod = 0.0;
                return;
            }
            int e;
            d = frexp(d, &e);
            ex += e;
        }
        prod *= d;
        if (prod < 0x1p-400 && prod > 0.0) {
            int e;
            prod = frexp(prod, &e);
            ex += e;
        }
    }
    __device__ __forceinline__ double log_value() const {
        return prod > 0.0 ? log(prod) + (double)ex * 0.69314718055994530942 : -INFINITY;
    }
};

// Out-of-line FP64 step for the rare fallbacks of the FP32 step (keeps the unrolled sweep small).
static __device__ __noinline__ float sov_step_f64_slow(double ai, double bi, double s, double lii,
                                                double w, double* delta) {
    return (float)sov_step_f64(ai, bi, s, lii, w, *delta);
}

// ---------------------------------------------------------------- FP32 elementwise step (mixed)
// Phi, Q and Phi^-1 in FP32 (CUDA erfcf / normcdfinvf) away from the deep tails.  Both tails of
// y are taken from the side where the probability is small: with p = Phi(a') + w Delta,
// 1 - p = Q(a') - w Delta is formed from Q and 1 - w (exact in FP64 for w >= 1/2) instead of by
// subtraction, and y = -Phi^-1(1 - p) when p > 1/2.  The deep tails (where FP32 would underflow)
// and two-sided finite intervals (where Phi(b') - Phi(a') cancels) use the FP64 step.
__device__ __forceinline__ float phinv_two_sided_f32(float p, float q) {
    // y = Phi^-1(p) with q = 1 - p given accurately
    return (p <= 0.5f) ? normcdfinvf(p) : -normcdfinvf(q);
}

__device__ __forceinline__ float sov_step_f32(double ai, double bi, float s, float lii, double w,
                                              double& delta) {
    const bool ainf = (ai == -INFINITY), binf = (bi == INFINITY);
    const float wf = (float)w, wcf = (float)(1.0 - w);
    if (ainf && binf) {
        delta = 1.0;
        return phinv_two_sided_f32(wf, wcf);
    }
    if (ainf) {  // Delta = Phi(b'),  p = w Phi(b'),  1 - p = (1 - w) + w Q(b')
        const float bp = ((float)bi - s) / lii;
        if (bp > -9.0f) {
            float pb, qb;
            if (bp < 0.0f) {
                pb = 0.5f * erfcf(-bp * 0.70710678f);
                qb = 1.0f - pb;
                delta = (double)pb;
            } else {
                qb = 0.5f * erfcf(bp * 0.70710678f);
                pb = 1.0f - qb;
                delta = 1.0 - (double)qb;
            }
            const float p = wf * pb, q = wcf + wf * qb;
            if (fminf(p, q) > 1e-30f) return phinv_two_sided_f32(p, q);
        }
        return sov_step_f64_slow(ai, bi, (double)s, (double)lii, w, &delta);
    }
    if (binf) {  // Delta = Q(a'),  p = Phi(a') + w Q(a'),  1 - p = (1 - w) Q(a')
        const float ap = ((float)ai - s) / lii;
        if (ap < 9.0f) {
            float pa, qa;
            if (ap > 0.0f) {
                qa = 0.5f * erfcf(ap * 0.70710678f);
                pa = 1.0f - qa;
                delta = (double)qa;
            } else {
                pa = 0.5f * erfcf(-ap * 0.70710678f);
                qa = 1.0f - pa;
                delta = 1.0 - (double)pa;
            }
            const float p = pa + wf * qa, q = wcf * qa;
            if (fminf(p, q) > 1e-30f) return phinv_two_sided_f32(p, q);
        }
        return sov_step_f64_slow(ai, bi, (double)s, (double)lii, w, &delta);
    }
    return sov_step_f64_slow(ai, bi, (double)s, (double)lii, w, &delta);
}

