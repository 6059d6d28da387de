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
    // w is ((W >> 11) + 1/2) 2^-53 rounded to FP64, which is 1 for the top lattice integers:
    // 1 - w then takes its unrounded value 2^-54 (never 0, so Phi^-1 stays finite)
    const float wf = (float)w, wcf = (float)fmax(1.0 - w, 0x1p-54);
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


// ---------------------------------------------------------------- FP32-only step (mixed sweeps)
// The common path of the mixed sweeps uses no FP64 instruction (GB300's FP64 rate is ~1/64 of
// FP32): the lattice point comes from its 64-bit fixed-point value by integer-to-float
// conversion, w = (2m + 1) 2^-54 and 1 - w = (2^54 - 2m - 1) 2^-54 with m = W >> 11 (both
// never 0), and the factor Delta is returned as an unevaluated FP32 pair dh + dl (so that
// 1 - Q(b') keeps Q(b') even when it is below FP32's resolution of 1) times 2^dex.  Deep tails
// and two-sided intervals fall back to the FP64 step.

// The float nearest to an integer 1 <= x < 2^55 (ties to even), from integer operations only:
// the 64-bit integer-to-float conversion is a long-latency instruction on this GPU, and the
// lattice point sits on the sweep's serial chain.  With e the position of the leading one, the
// 24 leading bits are kept and rounded by the bits shifted out (round half to even).
__device__ __forceinline__ float u55_to_f32_rn(uint64_t x) {
    const int e = 63 - __clzll((long long)x);
    uint32_t mant;
    if (e <= 23) {
        mant = (uint32_t)x << (23 - e);  // exact
    } else {
        const int sh = e - 23;  // 1 .. 31
        mant = (uint32_t)(x >> sh);
        const uint64_t rem = x & ((1ull << sh) - 1ull), half = 1ull << (sh - 1);
        mant += (rem > half || (rem == half && (mant & 1u))) ? 1u : 0u;
    }
    // mant lies in [2^23, 2^24]; a rounding carry to 2^24 moves into the exponent field
    return __uint_as_float(((uint32_t)(e + 127) << 23) + (mant - (1u << 23)));
}

__device__ __forceinline__ void lattice_wf(uint64_t j, uint64_t alpha, uint64_t delta, float& w,
                                           float& wc, uint64_t& m) {
    const uint64_t W = j * alpha + delta;
    m = W >> 11;
    w = u55_to_f32_rn(2u * m + 1u) * 0x1p-54f;
    wc = u55_to_f32_rn((1ull << 54) - 2u * m - 1u) * 0x1p-54f;
}

static __device__ __noinline__ float sov_step_slow_pair(double ai, double bi, float s, float lii,
                                                 uint64_t m, float* dh, float* dl, int* dex) {
    double delta;
    const double w = ((double)m + 0.5) * 0x1p-53;
    const float y = (float)sov_step_f64(ai, bi, (double)s, (double)lii, w, delta);
    if (!(delta > 0.0)) {
        *dh = 0.0f;
        *dl = 0.0f;
        *dex = 0;
    } else {
        int e;
        const double mm = frexp(delta, &e);
        *dh = (float)mm;
        *dl = (float)(mm - (double)*dh);
        *dex = e;
    }
    return y;
}

// One dimension of Eq. 2 in FP32 (see above).  af/bf: the limits as floats; ai/bi: as doubles
// (used only by the fallback); ainf/binf: the limits are infinite.  Written without per-path
// branches on the common path (the paths of a warp take different tails): one erfcf of |x| gives
// both tails, one normcdfinvf of the smaller of p and 1 - p gives y, and the shift is scaled by
// 1 / L_ii, which does not depend on it.
// The same with rl = 1 / lii given (computed once per dimension ahead of the sweep).
__device__ __forceinline__ float sov_step_f32r(float af, float bf, double ai, double bi, bool ainf,
                                               bool binf, float s, float lii, float rl, float w,
                                               float wc, uint64_t m, float& dh, float& dl,
                                               int& dex) {
    dex = 0;
    dl = 0.0f;
    if (ainf && binf) {
        dh = 1.0f;
        return phinv_two_sided_f32(w, wc);
    }
    if (ainf) {  // Delta = Phi(b'),  p = w Phi(b'),  1 - p = (1 - w) + w Q(b')
        const float bp = (bf - s) * rl;
        if (bp > -9.0f) {
            const float e = 0.5f * erfcf(fabsf(bp) * 0.70710678f);  // the smaller tail
            const bool neg = bp < 0.0f;
            const float pb = neg ? e : 1.0f - e;
            const float qb = neg ? 1.0f - e : e;
            dh = pb;
            dl = neg ? 0.0f : -(qb + (pb - 1.0f));  // exact: pb - 1 is exact (Sterbenz)
            const float p = w * pb, q = wc + w * qb;
            if (fminf(p, q) > 1e-30f) {
                const bool lo = p <= 0.5f;
                const float y0 = normcdfinvf(lo ? p : q);
                return lo ? y0 : -y0;
            }
        }
        return sov_step_slow_pair(ai, bi, s, lii, m, &dh, &dl, &dex);
    }
    if (binf) {  // Delta = Q(a'),  p = Phi(a') + w Q(a'),  1 - p = (1 - w) Q(a')
        const float ap = (af - s) * rl;
        if (ap < 9.0f) {
            const float e = 0.5f * erfcf(fabsf(ap) * 0.70710678f);
            const bool pos = ap > 0.0f;
            const float qa = pos ? e : 1.0f - e;
            const float pa = pos ? 1.0f - e : e;
            dh = qa;
            dl = pos ? 0.0f : -(pa + (qa - 1.0f));
            const float p = pa + w * qa, q = wc * qa;
            if (fminf(p, q) > 1e-30f) {
                const bool lo = p <= 0.5f;
                const float y0 = normcdfinvf(lo ? p : q);
                return lo ? y0 : -y0;
            }
        }
        return sov_step_slow_pair(ai, bi, s, lii, m, &dh, &dl, &dex);
    }
    return sov_step_slow_pair(ai, bi, s, lii, m, &dh, &dl, &dex);
}

__device__ __forceinline__ float sov_step_f32p(float af, float bf, double ai, double bi, bool ainf,
                                               bool binf, float s, float lii, float w, float wc,
                                               uint64_t m, float& dh, float& dl, int& dex) {
    return sov_step_f32r(af, bf, ai, bi, ainf, binf, s, lii, 1.0f / lii, w, wc, m, dh, dl, dex);
}

// Running product of the factors as (ph + pl) 2^ex in FP32 pairs: each factor costs an exact
// product (FMA error term) and a few FP32 operations; relative error ~2^-47 per factor.
struct DFProd {
    float ph = 1.0f, pl = 0.0f;
    int ex = 0;
    __device__ __forceinline__ void mul(float dh, float dl, int dex) {
        const float nh = ph * dh;
        const float e = fmaf(ph, dh, -nh);
        const float nl = fmaf(ph, dl, fmaf(pl, dh, e));
        ph = nh + nl;
        pl = nl - (ph - nh);
        ex += dex;
        if (ph < 0x1p-64f) {
            if (!(ph > 0.0f)) {
                ph = 0.0f;
                pl = 0.0f;
            } else {
                ph *= 0x1p64f;
                pl *= 0x1p64f;
                ex -= 64;
            }
        }
    }
    __device__ __forceinline__ double log_value() const {
        const double p = (double)ph + (double)pl;
        return p > 0.0 ? log(p) + (double)ex * 0.69314718055994530942 : -INFINITY;
    }
};
