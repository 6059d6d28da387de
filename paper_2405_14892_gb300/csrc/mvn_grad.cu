// mvn_grad.cu -- adjoints (not in the paper; the chain rule of its Eq. 2 and of Alg. 1's
// factorisation): d log P-hat / d(a, b, L) by a reverse blocked SOV sweep, the reverse mode of the
// Cholesky factorisation (blocked form of the column algorithm's adjoint, Murray 2016), and the
// FP64 GEMMs they need.
//
// log P-hat = log(mean_p exp(logw_p)), so d log P-hat = sum_p w_p d logw_p with w = softmax(logw).
// Per path, the reverse of Eq. 2 in dimension order n-1 .. 0 (a' = (a - s)/L_ii, likewise b'):
//   ybar_i  = sum_{j>i} sbar_j L_ji
//   a'bar   = -phi(a')/Delta + ybar_i (1 - w_i) phi(a')/phi(y_i)   (0 for an infinite limit)
//   b'bar   =  phi(b')/Delta + ybar_i w_i phi(b')/phi(y_i)
//   sbar_i  = -(a'bar + b'bar)/L_ii;  da_i = a'bar/L_ii;  db_i = b'bar/L_ii
//   dL_ii   = -(a'bar a' + b'bar b')/L_ii;  dL_ik = sbar_i y_k (k < i)
// The forward sweep keeps every path tile's y values; the reverse sweep recomputes each block's
// limit shifts from them (one left-looking GEMM per block), forms ybar from the stored sbar of the
// later dimensions, and stores sbar.  dL (strict lower) = sum_p w_p sbar_p y_p^T is one GEMM over
// the path axis.  Every reduction over paths runs in a fixed order (deterministic).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "mvn_internal.cuh"
#include "mvn_sov_simt.cuh"

mvn_status chol_f64_launch(mvn_ctx* ctx, int n, double* A, int64_t ld);
mvn_status sov_reduce_launch_opt(mvn_ctx* ctx, const double* logw, int64_t Ns, int M,
                                 double err_k, double* out3, int nprob, int64_t prob_stride,
                                 bool raise_numeric);

#define RV_B 16
__device__ __forceinline__ double phi_d(double x) {
    return 0.39894228040143267794 * exp(-0.5 * x * x);
}

// ---------------------------------------------------------------- path weights

// lse[0] = log sum_p exp(logw_p) (one block, fixed order)
__global__ void k_lse_all(const double* __restrict__ logw, int64_t N, double* __restrict__ lse) {
    __shared__ double red[512];
    const int t = threadIdx.x;
    double m = -INFINITY;
    for (int64_t k = t; k < N; k += 512) m = fmax(m, logw[k]);
    red[t] = m;
    __syncthreads();
    for (int w = 256; w > 0; w >>= 1) {
        if (t < w) red[t] = fmax(red[t], red[t + w]);
        __syncthreads();
    }
    m = red[0];
    __syncthreads();
    double s = 0.0;
    if (m > -INFINITY)
        for (int64_t k = t; k < N; k += 512) s += exp(logw[k] - m);
    red[t] = s;
    __syncthreads();
    for (int w = 256; w > 0; w >>= 1) {
        if (t < w) red[t] += red[t + w];
        __syncthreads();
    }
    if (t == 0) lse[0] = (m > -INFINITY) ? m + log(red[0]) : -INFINITY;
}

__global__ void k_weights(const double* __restrict__ logw, int64_t N,
                          const double* __restrict__ lse, double* __restrict__ omega) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= N) return;
    const double l = lse[0];
    omega[p] = (l > -INFINITY) ? exp(logw[p] - l) : 0.0;
}

// ---------------------------------------------------------------- reverse sweep

// T = type of the stored y and sbar and of the two per-block sums over dimensions (double: the
// FP64 adjoint; float: the mixed adjoint).  The elementwise derivative terms are FP64 for both.
#define RV_PATHS 32                 // paths per reverse work item (a quarter of a 128-path tile)
#define RV_SUB 4                    // threads per path
#define RV_THREADS (RV_PATHS * RV_SUB)
#define RV_ITEMS_PER_TILE (SOV_P / RV_PATHS)

// One 16-dimension step of the limit-shift sums acc[c] = sum_{k < r0} L(r0 + v_c, k) y_k of a
// path (v_c = sub + 4 c), shared by the forward and the reverse sweep of the adjoint so that both
// form bit-identical limits.  FP64: one FMA chain in dimension order (mid stays zero).  FP32:
// each 16-dimension block is summed into its own partial, the partials of a 128-dimension group
// into mid, and mid into acc at the end of every group (the caller adds the last mid): the chain
// of FP32 additions grows with 16 + 8 + r0 / 128 terms instead of r0 (one FP32 chain biases
// log P by ~1e-6 per dimension on strongly correlated fields).
template <typename T, int NV>
__device__ __forceinline__ void limit_sum_step(const T (&Lk)[RV_B][RV_B], const T* __restrict__ Yt,
                                               int k0, int pc, int sub, T (&acc)[NV],
                                               T (&mid)[NV]) {
    constexpr bool kF32 = sizeof(T) == 4;
    T part_[NV];
#pragma unroll
    for (int c = 0; c < NV; ++c) part_[c] = kF32 ? (T)0 : acc[c];
#pragma unroll 4
    for (int kk = 0; kk < RV_B; ++kk) {
        const T yk = Yt[(int64_t)(k0 + kk) * SOV_P + pc];
#pragma unroll
        for (int c = 0; c < NV; ++c) part_[c] = fma(Lk[kk][sub + RV_SUB * c], yk, part_[c]);
    }
    if (kF32) {
#pragma unroll
        for (int c = 0; c < NV; ++c) mid[c] += part_[c];
        if (((k0 / RV_B) & 7) == 7) {
#pragma unroll
            for (int c = 0; c < NV; ++c) {
                acc[c] += mid[c];
                mid[c] = (T)0;
            }
        }
    } else {
#pragma unroll
        for (int c = 0; c < NV; ++c) acc[c] = part_[c];
    }
}

template <typename T>
struct RevSmem {
    T Lk[RV_B][RV_B];             // GEMM operand tile
    T Ld[RV_B][RV_B + 1];         // diagonal block L(r0+v, r0+u)
    T acc[RV_B][RV_PATHS];        // limit shifts from earlier blocks, per (dim, path)
    T yb[RV_B][RV_PATHS];         // ybar from later dimensions, per (dim, path)
    // per (dim, path) terms of the reverse step that do not depend on ybar
    double ca[RV_B][RV_PATHS];    // -phi(a') / Delta
    double cya[RV_B][RV_PATHS];   // (1 - w) phi(a') / phi(y)
    double cb[RV_B][RV_PATHS];    // phi(b') / Delta
    double cyb[RV_B][RV_PATHS];   // w phi(b') / phi(y)
    double ta[RV_B][RV_PATHS];    // a' (0 where phi(a') = 0)
    double tb[RV_B][RV_PATHS];    // b' (0 where phi(b') = 0)
    double a[RV_B], b[RV_B];
    uint64_t alpha[RV_B];
};

// One work item = 32 paths (quarter h of 128-path tile `tile`), dimension blocks in reverse order.
// Y and Sbar of the tile live at Yt/St[k * 128 + path]; the item's paths are 32 h .. 32 h + 31.
// 128 threads, thread (sub = t / 32, pl = t % 32) works for path pl on the block's dimensions
// v = sub, sub + 4, ..:
//   (a), (b) the sums over earlier dimensions (limit shift) and later dimensions (ybar), each v
//            summed by one thread in dimension order;
//   (d)      a', b' from the stored y and the elementwise terms of the reverse step (Phi, phi of
//            Eq. 2), which do not depend on ybar;
// then warp 0 runs the reverse chain of the block for its 32 paths (ybar of dimension u < v takes
// sbar_v L_vu), a few FP64 operations per dimension.  part[(item * 3 + c) * n + i] receives the
// item's sum over its paths of w_p a'bar/L_ii (c = 0), w_p b'bar/L_ii (c = 1), w_p dL_ii (c = 2).
template <typename T>
__device__ void rev_item(const SovProblem& P, int item, const uint64_t* __restrict__ alpha,
                         const T* __restrict__ Yt, T* __restrict__ St,
                         const double* __restrict__ omega, double* __restrict__ part,
                         RevSmem<T>& sm) {
    constexpr bool kF32 = sizeof(T) == 4;
    constexpr int NV = RV_B / RV_SUB;  // dimensions per thread
    const int t = threadIdx.x;
    const int pl = t % RV_PATHS, sub = t / RV_PATHS;
    const int tile = item / RV_ITEMS_PER_TILE, h = item % RV_ITEMS_PER_TILE;
    const int pc = h * RV_PATHS + pl;  // column of the path in the tile's Y / Sbar
    const int n = P.n;
    const int64_t p = (int64_t)tile * SOV_P + pc;
    const bool valid = p < P.Ntot;
    const int64_t pg = P.p0 + p;  // index of the path in the whole lattice rule
    const int64_t q = valid ? pg / P.Ns : 0;
    const uint64_t j = valid ? (uint64_t)(pg - q * P.Ns) + 1u : 1u;
    const uint64_t* __restrict__ dq = P.delta + q * P.dstride;
    const double* __restrict__ L = P.L;
    const int64_t ld = P.ld;
    const double wp = valid ? omega[p] : 0.0;
    const bool live = wp > 0.0;
    const int nblk = (n + RV_B - 1) / RV_B;
    for (int blk = nblk - 1; blk >= 0; --blk) {
        const int r0 = blk * RV_B;
        const int nb = min(RV_B, n - r0);
        T acc[NV], yb[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) {
            acc[c] = (T)0;
            yb[c] = (T)0;
        }
        // (a) limit shift from earlier blocks: acc[v] = sum_{k < r0} L(r0+v, k) y_k, summed as
        // in the forward sweep (limit_sum_step)
        T mid[NV];
#pragma unroll
        for (int c = 0; c < NV; ++c) mid[c] = (T)0;
        for (int k0 = 0; k0 < r0; k0 += RV_B) {
            __syncthreads();
            for (int e = t; e < RV_B * RV_B; e += RV_THREADS) {
                const int v = e % RV_B, kk = e / RV_B;
                const int row = r0 + v;
                sm.Lk[kk][v] = (row < n) ? (T)L[row + (int64_t)(k0 + kk) * ld] : (T)0;
            }
            __syncthreads();
            limit_sum_step<T, NV>(sm.Lk, Yt, k0, pc, sub, acc, mid);
        }
#pragma unroll
        for (int c = 0; c < NV; ++c) acc[c] += mid[c];
        // (b) ybar from the later dimensions: yb[v] = sum_{i >= r0+nb} L(i, r0+v) sbar_i
        for (int i0 = r0 + RV_B; i0 < n; i0 += RV_B) {
            __syncthreads();
            for (int e = t; e < RV_B * RV_B; e += RV_THREADS) {
                const int ii = e % RV_B, v = e / RV_B;
                const int row = i0 + ii;
                sm.Lk[ii][v] = (row < n && v < nb) ? (T)L[row + (int64_t)(r0 + v) * ld] : (T)0;
            }
            __syncthreads();
            const int ni = min(RV_B, n - i0);
            T part_[NV];
#pragma unroll
            for (int c = 0; c < NV; ++c) part_[c] = kF32 ? (T)0 : yb[c];
            for (int ii = 0; ii < ni; ++ii) {
                const T sb = St[(int64_t)(i0 + ii) * SOV_P + pc];
#pragma unroll
                for (int c = 0; c < NV; ++c)
                    part_[c] = fma(sm.Lk[ii][sub + RV_SUB * c], sb, part_[c]);
            }
#pragma unroll
            for (int c = 0; c < NV; ++c) yb[c] = kF32 ? yb[c] + part_[c] : part_[c];
        }
        // (c) block operands
        __syncthreads();
        for (int e = t; e < RV_B * RV_B; e += RV_THREADS) {
            const int v = e % RV_B, u = e / RV_B;
            sm.Ld[v][u] = (v < nb && u <= v) ? (T)L[(r0 + v) + (int64_t)(r0 + u) * ld] : (T)0;
        }
        if (t < RV_B) {
            sm.a[t] = (t < nb) ? P.a[r0 + t] : 0.0;
            sm.b[t] = (t < nb) ? P.b[r0 + t] : 1.0;
            sm.alpha[t] = (t < nb) ? alpha[r0 + t] : 0u;
        }
#pragma unroll
        for (int c = 0; c < NV; ++c) sm.yb[sub + RV_SUB * c][pl] = yb[c];
        __syncthreads();
        // (d) limits of the thread's dimensions from the stored y, and the ybar-free terms
        {
            T y[RV_B];
#pragma unroll
            for (int v = 0; v < RV_B; ++v) y[v] = (v < nb) ? Yt[(int64_t)(r0 + v) * SOV_P + pc] : (T)0;
#pragma unroll
            for (int c = 0; c < NV; ++c) {
                const int v = sub + RV_SUB * c;
                double ca = 0.0, cya = 0.0, cb = 0.0, cyb = 0.0, ta = 0.0, tb = 0.0;
                if (v < nb && live) {
                    T s = acc[c];
#pragma unroll
                    for (int u = 0; u < RV_B; ++u)
                        if (u < v) s = fma(sm.Ld[v][u], y[u], s);
                    const double lii = (double)sm.Ld[v][v];
                    const double A = (sm.a[v] - (double)s) / lii;
                    const double Bv = (sm.b[v] - (double)s) / lii;
                    const double w = lattice_w(j, sm.alpha[v], dq[r0 + v]);
                    double delta;
                    if (A > 0.0) {
                        delta = 0.5 * erfc(A * 0.70710678118654752440) -
                                ((Bv == INFINITY) ? 0.0 : 0.5 * erfc(Bv * 0.70710678118654752440));
                    } else {
                        delta = ((Bv == INFINITY) ? 1.0 : 0.5 * erfc(-Bv * 0.70710678118654752440)) -
                                ((A == -INFINITY) ? 0.0 : 0.5 * erfc(-A * 0.70710678118654752440));
                    }
                    const double pa = (A == -INFINITY) ? 0.0 : phi_d(A);
                    const double pb = (Bv == INFINITY) ? 0.0 : phi_d(Bv);
                    double yv = 0.0;
#pragma unroll
                    for (int u = 0; u < RV_B; ++u)
                        if (u == v) yv = (double)y[u];
                    const double py = phi_d(yv);
                    ca = -pa / delta;
                    cya = (1.0 - w) * pa / py;
                    cb = pb / delta;
                    cyb = w * pb / py;
                    ta = (pa != 0.0) ? A : 0.0;
                    tb = (pb != 0.0) ? Bv : 0.0;
                }
                sm.ca[v][pl] = ca;
                sm.cya[v][pl] = cya;
                sm.cb[v][pl] = cb;
                sm.cyb[v][pl] = cyb;
                sm.ta[v][pl] = ta;
                sm.tb[v][pl] = tb;
            }
        }
        __syncthreads();
        // (e) reverse chain of the block (warp 0, one thread per path)
        if (sub == 0) {
            T ybv[RV_B];
#pragma unroll
            for (int v = 0; v < RV_B; ++v) ybv[v] = sm.yb[v][pl];
#pragma unroll
            for (int v = RV_B - 1; v >= 0; --v) {
                double ga = 0.0, gb = 0.0, gd = 0.0, sbar = 0.0;
                if (v < nb && live) {
                    const double lii = (double)sm.Ld[v][v];
                    const double ybd = (double)ybv[v];
                    const double apbar = sm.ca[v][pl] + ybd * sm.cya[v][pl];
                    const double bpbar = sm.cb[v][pl] + ybd * sm.cyb[v][pl];
                    sbar = -(apbar + bpbar) / lii;
                    ga = wp * apbar / lii;
                    gb = wp * bpbar / lii;
                    gd = wp * (-(apbar * sm.ta[v][pl]) - bpbar * sm.tb[v][pl]) / lii;
                    const T sbt = (T)sbar;
#pragma unroll
                    for (int u = 0; u < v; ++u) ybv[u] = fma(sbt, sm.Ld[v][u], ybv[u]);
                }
                if (v < nb) St[(int64_t)(r0 + v) * SOV_P + pc] = (T)sbar;
                // reductions over the item's 32 paths (warp shuffles)
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    ga += __shfl_xor_sync(0xffffffffu, ga, o);
                    gb += __shfl_xor_sync(0xffffffffu, gb, o);
                    gd += __shfl_xor_sync(0xffffffffu, gd, o);
                }
                if (pl == 0 && v < nb) {
                    part[((int64_t)item * 3 + 0) * n + r0 + v] = ga;
                    part[((int64_t)item * 3 + 1) * n + r0 + v] = gb;
                    part[((int64_t)item * 3 + 2) * n + r0 + v] = gd;
                }
            }
        }
    }
}

template <typename T>
__global__ void __launch_bounds__(RV_THREADS, 3) k_sov_rev(const SovProblem P, int nitems,
                                                        int* __restrict__ counter,
                                                        const uint64_t* __restrict__ alpha,
                                                        const T* __restrict__ Y,
                                                        T* __restrict__ Sbar, int64_t ystride,
                                                        const double* __restrict__ omega,
                                                        double* __restrict__ part) {
    __shared__ RevSmem<T> sm;
    __shared__ int s_item;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const int64_t off = (int64_t)(it / RV_ITEMS_PER_TILE) * ystride;
        rev_item(P, it, alpha, Y + off, Sbar + off, omega, part, sm);
    }
}

// ---------------------------------------------------------------- forward sweep of the adjoint

// The forward sweep of Eq. 2 that keeps every path's y for the reverse sweep, on the same 32-path
// work items as k_sov_rev: 128 threads, thread (sub = t / 32, pl = t % 32) forms for path pl the
// limit shifts of the block's dimensions v = sub, sub + 4, .. from the earlier dimensions (each v
// summed by one thread in dimension order; FP32: per 16-dimension partial sums, exactly as the
// reverse sweep recomputes them), then warp 0 runs the block's dimensions one after the other
// (Alg. 3) with the elementwise step in FP64 and writes y.  logw[p] receives log prod Delta.
template <typename T>
struct FwdSmem {
    T Lk[RV_B][RV_B];
    T Ld[RV_B][RV_B + 1];
    T acc[RV_B][RV_PATHS];
    double a[RV_B], b[RV_B];
    uint64_t alpha[RV_B];
};

template <typename T>
__global__ void __launch_bounds__(RV_THREADS, 4) k_sov_fwd_keep(const SovProblem P, int nitems,
                                                                int* __restrict__ counter,
                                                                const uint64_t* __restrict__ alpha,
                                                                T* __restrict__ Y,
                                                                int64_t ystride) {
    constexpr int NV = RV_B / RV_SUB;
    __shared__ FwdSmem<T> sm;
    __shared__ int s_item;
    const int t = threadIdx.x;
    const int pl = t % RV_PATHS, sub = t / RV_PATHS;
    const int n = P.n;
    const double* __restrict__ L = P.L;
    const int64_t ld = P.ld;
    for (;;) {
        __syncthreads();
        if (t == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= nitems) break;
        const int tile = item / RV_ITEMS_PER_TILE, h = item % RV_ITEMS_PER_TILE;
        T* __restrict__ Yt = Y + (int64_t)tile * ystride;
        const int pc = h * RV_PATHS + pl;
        const int64_t p = (int64_t)tile * SOV_P + pc;
        const bool valid = p < P.Ntot;
        const int64_t pg = P.p0 + p;  // index of the path in the whole lattice rule
        const int64_t q = valid ? pg / P.Ns : 0;
        const uint64_t j = valid ? (uint64_t)(pg - q * P.Ns) + 1u : 1u;
        const uint64_t* __restrict__ dq = P.delta + q * P.dstride;
        LogProd lp;
        for (int r0 = 0; r0 < n; r0 += RV_B) {
            const int nb = min(RV_B, n - r0);
            T acc[NV], mid[NV];
#pragma unroll
            for (int c = 0; c < NV; ++c) {
                acc[c] = (T)0;
                mid[c] = (T)0;
            }
            for (int k0 = 0; k0 < r0; k0 += RV_B) {
                __syncthreads();
                for (int e = t; e < RV_B * RV_B; e += RV_THREADS) {
                    const int v = e % RV_B, kk = e / RV_B;
                    const int row = r0 + v;
                    sm.Lk[kk][v] = (row < n) ? (T)L[row + (int64_t)(k0 + kk) * ld] : (T)0;
                }
                __syncthreads();
                limit_sum_step<T, NV>(sm.Lk, Yt, k0, pc, sub, acc, mid);
            }
#pragma unroll
            for (int c = 0; c < NV; ++c) acc[c] += mid[c];
            __syncthreads();
            for (int e = t; e < RV_B * RV_B; e += RV_THREADS) {
                const int v = e % RV_B, u = e / RV_B;
                sm.Ld[v][u] = (v < nb && u <= v) ? (T)L[(r0 + v) + (int64_t)(r0 + u) * ld] : (T)0;
            }
            if (t < RV_B) {
                sm.a[t] = (t < nb) ? P.a[r0 + t] : 0.0;
                sm.b[t] = (t < nb) ? P.b[r0 + t] : 1.0;
                sm.alpha[t] = (t < nb) ? alpha[r0 + t] : 0u;
            }
#pragma unroll
            for (int c = 0; c < NV; ++c) sm.acc[sub + RV_SUB * c][pl] = acc[c];
            __syncthreads();
            if (sub == 0) {
                T y[RV_B];
#pragma unroll
                for (int v = 0; v < RV_B; ++v) {
                    y[v] = (T)0;
                    if (v < nb) {
                        T s = sm.acc[v][pl];
#pragma unroll
                        for (int u = 0; u < v; ++u) s = fma(sm.Ld[v][u], y[u], s);
                        const double w = lattice_w(j, sm.alpha[v], dq[r0 + v]);
                        double delta;
                        y[v] = (T)sov_step_f64(sm.a[v], sm.b[v], (double)s, (double)sm.Ld[v][v], w,
                                               delta);
                        lp.mul(delta);
                        if (valid) Yt[(int64_t)(r0 + v) * SOV_P + pc] = y[v];
                    }
                }
            }
            // the block's y are read by all four threads of each path in the next block
        }
        if (sub == 0 && valid) P.logw[p] = lp.log_value();
    }
}

// out[c * n + i] = sum over work items (fixed order) of part[(item * 3 + c) * n + i]
__global__ void k_sum_parts(const double* __restrict__ part, int ntiles, int n,
                            double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int c = blockIdx.y;
    if (i >= n) return;
    double s = 0.0;
    for (int tl = 0; tl < ntiles; ++tl) s += part[((int64_t)tl * 3 + c) * n + i];
    out[(int64_t)c * n + i] = s;
}

// dL(i, k) for i > k: sum over paths of w_p sbar_{p,i} y_{p,k}; dL(i, i) = dsum[2n + i].
// Paths are laid out per tile: X[tile][dim][128].  One 64 x 64 lower output tile per block.
// The products of one 128-path tile are summed in T, the tiles' partial sums in FP64 (for
// T = float the rounding error then grows with the tile's 128 terms, not with all N paths).
// mode 0: write every lower entry (dL(i, i) from dsum); mode 1: write the strictly lower entries
// only; mode 2: add into the strictly lower entries (batches of path tiles: Sbar, Y and omega are
// the batch's, Ntot its path count; the diagonal is written once at the end by k_grad_diag).
template <typename T>
__global__ void __launch_bounds__(256) k_grad_L(int n, int ntiles, int64_t Ntot,
                                                const T* __restrict__ Sbar,
                                                const T* __restrict__ Y,
                                                const double* __restrict__ omega,
                                                const double* __restrict__ dsum,
                                                double* __restrict__ G, int64_t ldg, int mode) {
    __shared__ T As[32][64 + 1];  // As[pp][r] = w_p sbar_{p, R0 + r}
    __shared__ T Bs[32][64 + 1];  // Bs[pp][c] = y_{p, C0 + c}
    const int x = blockIdx.x;
    int ti = (int)((sqrt(8.0 * x + 1.0) - 1.0) * 0.5);
    while ((ti + 1) * (ti + 2) / 2 <= x) ++ti;
    while (ti * (ti + 1) / 2 > x) --ti;
    const int tj = x - ti * (ti + 1) / 2;
    const int R0 = ti * 64, C0 = tj * 64;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    double acc[4][4] = {};
    for (int tl = 0; tl < ntiles; ++tl) {
        const T* St = Sbar + (int64_t)tl * n * SOV_P;
        const T* Yt = Y + (int64_t)tl * n * SOV_P;
        T tacc[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) tacc[u][v] = (T)0;
        for (int c0 = 0; c0 < SOV_P; c0 += 32) {
            __syncthreads();
            for (int e = t; e < 32 * 64; e += 256) {
                const int pp = e % 32, r = e / 32;
                const int64_t pth = (int64_t)tl * SOV_P + c0 + pp;
                // padding paths of the last tile are masked, not weighted by zero: their y and
                // sbar slots are never written
                const bool vp = pth < Ntot;
                As[pp][r] = (vp && R0 + r < n)
                                ? (T)(omega[pth] * (double)St[(int64_t)(R0 + r) * SOV_P + c0 + pp])
                                : (T)0;
                Bs[pp][r] = (vp && C0 + r < n) ? Yt[(int64_t)(C0 + r) * SOV_P + c0 + pp] : (T)0;
            }
            __syncthreads();
#pragma unroll 4
            for (int pp = 0; pp < 32; ++pp) {
                T a[4], b[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) a[u] = As[pp][tx + 16 * u];
#pragma unroll
                for (int v = 0; v < 4; ++v) b[v] = Bs[pp][ty + 16 * v];
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) tacc[u][v] = fma(a[u], b[v], tacc[u][v]);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] += (double)tacc[u][v];
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int c = C0 + ty + 16 * v;
        if (c >= n) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = R0 + tx + 16 * u;
            if (r >= n || r < c) continue;
            if (mode == 0)
                G[r + (int64_t)c * ldg] = (r == c) ? dsum[2 * (int64_t)n + r] : acc[u][v];
            else if (r > c)
                G[r + (int64_t)c * ldg] = (mode == 1) ? acc[u][v] : G[r + (int64_t)c * ldg] + acc[u][v];
        }
    }
}

// dL(i, i) = dsum[2n + i] (the diagonal terms summed over all work items).
__global__ void k_grad_diag(int n, const double* __restrict__ dsum, double* __restrict__ G,
                            int64_t ldg) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) G[i + (int64_t)i * ldg] = dsum[2 * (int64_t)n + i];
}

// ---------------------------------------------------------------- generic FP64 GEMM

// C(i, j) += alpha * sum_k A(i, k) B(k, j) for i < m, j < nn, with element strides:
//   A(i,k) = A[i*sar + k*sac], B(k,j) = B[k*sbr + j*sbc], C(i,j) = C[i + j*ldc] (column-major).
// triA: 0 = dense, 1 = lower (A(i,k) = 0 for k > i), 2 = upper (A(i,k) = 0 for k < i).
// lowerC: only entries with i + ci0 >= j + cj0 are written (a lower triangle of the parent).
// Split K: block z sums k in [z kchunk, (z + 1) kchunk) and, when P is not null, writes its
// partial tile to P[z m nn + i + j m] instead of updating C (k_gemm_reduce adds the partials in
// a fixed order).
__global__ void __launch_bounds__(256) k_gemm64(int m, int nn, int kk, double alpha,
                                                const double* __restrict__ A, int64_t sar,
                                                int64_t sac, const double* __restrict__ B,
                                                int64_t sbr, int64_t sbc, double* __restrict__ C,
                                                int64_t ldc, int triA, int lowerC, int ci0,
                                                int cj0, int kchunk, double* __restrict__ P) {
    __shared__ double As[16][64 + 1];  // As[k][i]
    __shared__ double Bs[16][64 + 1];  // Bs[k][j]
    const int I0 = blockIdx.x * 64, J0 = blockIdx.y * 64;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int kbeg = blockIdx.z * kchunk, kend = min(kk, kbeg + kchunk);
    double acc[4][4] = {};
    for (int k0 = kbeg; k0 < kend; k0 += 16) {
        __syncthreads();
        for (int e = t; e < 16 * 64; e += 256) {
            const int i = e % 64, k = e / 64;
            const int gi = I0 + i, gk = k0 + k;
            double av = 0.0;
            if (gi < m && gk < kend && !(triA == 1 && gk > gi) && !(triA == 2 && gk < gi))
                av = A[gi * sar + gk * sac];
            As[k][i] = av;
            const int gj = J0 + i;
            Bs[k][i] = (gj < nn && gk < kend) ? B[gk * sbr + gj * sbc] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = As[k][tx + 16 * u];
#pragma unroll
            for (int v = 0; v < 4; ++v) b[v] = Bs[k][ty + 16 * v];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int j = J0 + ty + 16 * v;
        if (j >= nn) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = I0 + tx + 16 * u;
            if (i >= m) continue;
            if (P) {
                P[(int64_t)blockIdx.z * m * nn + i + (int64_t)j * m] = acc[u][v];
                continue;
            }
            if (lowerC && i + ci0 < j + cj0) continue;
            C[i + (int64_t)j * ldc] += alpha * acc[u][v];
        }
    }
}

// C(i, j) += alpha sum_z P[z m nn + i + j m], z in order (deterministic)
__global__ void k_gemm_reduce(int m, int nn, int nz, const double* __restrict__ P, double alpha,
                              double* __restrict__ C, int64_t ldc, int lowerC, int ci0, int cj0) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * nn) return;
    const int i = (int)(e % m), j = (int)(e / m);
    if (lowerC && i + ci0 < j + cj0) return;
    double s = 0.0;
    for (int z = 0; z < nz; ++z) s += P[(int64_t)z * m * nn + e];
    C[i + (int64_t)j * ldc] += alpha * s;
}

// Split-K workspace bound of gemm64 (doubles): at most 4 SM-counts of 64 x 64 partial tiles.
static size_t gemm64_ws_doubles(const mvn_ctx* ctx) { return (size_t)4 * ctx->sm_count * 64 * 64; }

// C += alpha A B.  GEMMs with few output tiles and a long K (the panel-transpose products of the
// Cholesky adjoint: K up to n, one row of 64 x 64 tiles) are split along K over about two CTAs
// per SM, into partial tiles in P (gemm64_ws_doubles) summed by k_gemm_reduce.
static mvn_status gemm64(mvn_ctx* ctx, int m, int nn, int kk, double alpha, const double* A,
                         int64_t sar, int64_t sac, const double* B, int64_t sbr, int64_t sbc,
                         double* C, int64_t ldc, double* P, int triA = 0, int lowerC = 0,
                         int ci0 = 0, int cj0 = 0) {
    if (m <= 0 || nn <= 0 || kk <= 0) return MVN_OK;
    const int64_t tiles = (int64_t)((m + 63) / 64) * ((nn + 63) / 64);
    int nz = 1;
    if (P && kk >= 256 && tiles < 2 * ctx->sm_count) {
        nz = (int)std::min<int64_t>((2 * ctx->sm_count + tiles - 1) / tiles, kk / 128);
        while (nz > 1 && (size_t)nz * tiles * 64 * 64 > gemm64_ws_doubles(ctx)) --nz;
    }
    const int kchunk = (nz == 1) ? kk : (((kk + nz - 1) / nz + 15) / 16) * 16;
    nz = (kk + kchunk - 1) / kchunk;
    dim3 grid((m + 63) / 64, (nn + 63) / 64, nz);
    MVN_TIMED(ctx, "k_gemm64",
              (k_gemm64<<<grid, 256, 0, ctx->stream>>>(m, nn, kk, alpha, A, sar, sac, B, sbr, sbc,
                                                       C, ldc, triA, lowerC, ci0, cj0, kchunk,
                                                       nz > 1 ? P : nullptr)));
    if (nz > 1) {
        const int64_t cnt = (int64_t)m * nn;
        k_gemm_reduce<<<(unsigned)((cnt + 255) / 256), 256, 0, ctx->stream>>>(
            m, nn, nz, P, alpha, C, ldc, lowerC, ci0, cj0);
        MVN_LAUNCHED(ctx);
    }
    return MVN_OK;
}

// ---------------------------------------------------------------- Cholesky adjoint

#define CG_NB 64

// Unblocked reverse of the column Cholesky on one nb x nb diagonal block (in shared memory):
// on entry G = dF/dL_jj (lower), on exit dF/dA' (lower) of the block's input.
__global__ void __launch_bounds__(256) k_cgrad_diag(const double* __restrict__ L, int64_t ld,
                                                    double* __restrict__ G, int64_t ldg, int c0,
                                                    int nb) {
    __shared__ double Ls[CG_NB][CG_NB + 1];
    __shared__ double Gs[CG_NB][CG_NB + 1];
    const int t = threadIdx.x;
    for (int e = t; e < nb * nb; e += 256) {
        const int i = e % nb, k = e / nb;
        Ls[i][k] = (i >= k) ? L[(c0 + i) + (int64_t)(c0 + k) * ld] : 0.0;
        Gs[i][k] = (i >= k) ? G[(c0 + i) + (int64_t)(c0 + k) * ldg] : 0.0;
    }
    __syncthreads();
    for (int jj = nb - 1; jj >= 0; --jj) {
        const double ljj = Ls[jj][jj];
        const double rjj = 1.0 / ljj;
        // off-diagonal entries of column jj: L_ij = (A_ij - sum_{k<jj} L_ik L_jk) / L_jj, so
        // g_i = G_ij / L_jj becomes the adjoint of A_ij;  G_ik -= g_i L_jk, G_jk -= g_i L_ik
        // (k < jj);  G_jj -= g_i L_ij
        for (int i = jj + 1 + t; i < nb; i += 256) Gs[i][jj] *= rjj;
        __syncthreads();
        // row jj (one thread per k, sum over i in order) and the rows below (one entry each)
        for (int k = t; k <= jj; k += 256) {
            double s = 0.0;
            for (int i = nb - 1; i > jj; --i) s = fma(Gs[i][jj], Ls[i][k], s);
            Gs[jj][k] -= s;
        }
        for (int e = t; e < (nb - jj - 1) * jj; e += 256) {
            const int i = jj + 1 + e % (nb - jj - 1), k = e / (nb - jj - 1);
            Gs[i][k] = fma(-Gs[i][jj], Ls[jj][k], Gs[i][k]);
        }
        __syncthreads();
        // pivot: L_jj = sqrt(A_jj - sum_{k<jj} L_jk^2);  g = G_jj / (2 L_jj); G_jk -= 2 g L_jk
        const double g = Gs[jj][jj] * (0.5 * rjj);
        for (int k = t; k < jj; k += 256) Gs[jj][k] = fma(-2.0 * g, Ls[jj][k], Gs[jj][k]);
        __syncthreads();
        if (t == 0) Gs[jj][jj] = g;
        __syncthreads();
    }
    for (int e = t; e < nb * nb; e += 256) {
        const int i = e % nb, k = e / nb;
        if (i >= k) G[(c0 + i) + (int64_t)(c0 + k) * ldg] = Gs[i][k];
    }
}

// Panel: rows r >= r1 of block column j: Z L_jj = Xbar (solved from the right, in place).
__global__ void __launch_bounds__(128) k_cgrad_panel(const double* __restrict__ L, int64_t ld,
                                                     double* __restrict__ G, int64_t ldg, int c0,
                                                     int nb, int r1, int n) {
    __shared__ double Ls[CG_NB][CG_NB + 1];
    const int t = threadIdx.x;
    for (int e = t; e < nb * nb; e += 128) {
        const int i = e % nb, k = e / nb;
        Ls[i][k] = (i >= k) ? L[(c0 + i) + (int64_t)(c0 + k) * ld] : 0.0;
    }
    __syncthreads();
    const int r = r1 + blockIdx.x * 128 + t;
    if (r >= n) return;
    double z[CG_NB];
#pragma unroll
    for (int c = CG_NB - 1; c >= 0; --c) {
        if (c < nb) {
            double s = G[r + (int64_t)(c0 + c) * ldg];
#pragma unroll
            for (int d = c + 1; d < CG_NB; ++d)
                if (d < nb) s -= z[d] * Ls[d][c];
            z[c] = s / Ls[c][c];
        } else {
            z[c] = 0.0;
        }
    }
#pragma unroll
    for (int c = 0; c < CG_NB; ++c)
        if (c < nb) G[r + (int64_t)(c0 + c) * ldg] = z[c];
}

mvn_status cholesky_grad_launch(mvn_ctx* ctx, int n, const double* L, int64_t ld, double* G,
                                int64_t ldg, double* P) {
    const int nblk = (n + CG_NB - 1) / CG_NB;
    for (int jb = nblk - 1; jb >= 0; --jb) {
        const int c0 = jb * CG_NB;
        const int nb = std::min(CG_NB, n - c0);
        const int r1 = c0 + nb, m = n - r1;
        double* Gp = G + r1 + (int64_t)c0 * ldg;        // panel adjoint (m x nb)
        const double* Xp = L + r1 + (int64_t)c0 * ld;   // panel of L (m x nb)
        if (m > 0) {
            MVN_TIMED(ctx, "k_cgrad_panel",
                      (k_cgrad_panel<<<(m + 127) / 128, 128, 0, ctx->stream>>>(L, ld, G, ldg, c0,
                                                                               nb, r1, n)));
            // Gjj -= lower(Zp^T Xp)
            MVN_TRY(gemm64(ctx, nb, nb, m, -1.0, Gp, ldg, 1, Xp, 1, ld,
                           G + c0 + (int64_t)c0 * ldg, ldg, P, 0, 1, 0, 0));
            if (c0 > 0) {
                // G(r1:n, 0:c0) -= Zp L(c0:c0+nb, 0:c0)
                MVN_TRY(gemm64(ctx, m, c0, nb, -1.0, Gp, 1, ldg, L + c0, 1, ld, G + r1, ldg, P));
                // G(c0:c0+nb, 0:c0) -= Zp^T L(r1:n, 0:c0)
                MVN_TRY(gemm64(ctx, nb, c0, m, -1.0, Gp, ldg, 1, L + r1, 1, ld, G + c0, ldg, P));
            }
        }
        MVN_TIMED(ctx, "k_cgrad_diag",
                  (k_cgrad_diag<<<1, 256, 0, ctx->stream>>>(L, ld, G, ldg, c0, nb)));
        if (c0 > 0) {
            // G(c0:c0+nb, 0:c0) -= (Ajj + Ajj^T) L(c0:c0+nb, 0:c0),  Ajj lower
            const double* Aj = G + c0 + (int64_t)c0 * ldg;
            MVN_TRY(gemm64(ctx, nb, c0, nb, -1.0, Aj, 1, ldg, L + c0, 1, ld, G + c0, ldg, P, 1));
            MVN_TRY(gemm64(ctx, nb, c0, nb, -1.0, Aj, ldg, 1, L + c0, 1, ld, G + c0, ldg, P, 2));
        }
    }
    return MVN_OK;
}

extern "C" mvn_status mvn_cholesky_grad(mvn_ctx* ctx, int n, const double* L, int64_t ld,
                                        double* Lbar) {
    if (!ctx) return MVN_ERR_ARG;
    if (n < 0 || ld < (n > 0 ? n : 1) || (n > 0 && (!L || !Lbar)))
        return mvn_fail(ctx, MVN_ERR_ARG, "mvn_cholesky_grad: invalid argument");
    if (n == 0) return MVN_OK;
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    MVN_TRY(ws_reserve(ctx, sizeof(double) * gemm64_ws_doubles(ctx)));
    return cholesky_grad_launch(ctx, n, L, ld, Lbar, ld, (double*)ctx->ws);
}

// ---------------------------------------------------------------- SOV gradient

// T = double: the FP64 adjoint (FP64 everywhere).
// T = float: the mixed adjoint.  Its forward sweep (k_sov_fwd_keep) forms the limit shifts in FP32
// and keeps every tile's y in FP32, with the elementwise step of Eq. 2 in FP64: the
// per-dimension errors of an FP32 step add up along the n dimensions of log P, those of the FP32
// limit sums much less.  The reverse sweep forms the limit shifts and ybar in FP32 and the
// elementwise derivative terms in FP64; dL sums FP32 products per 128-path tile and the tiles in
// FP64.
template <typename T>
static mvn_status sov_grad_run(mvn_ctx* ctx, int n, const double* a, const double* b,
                               const double* L, int64_t ld, const mvn_qmc* qmc, double* out3,
                               double* dlogp_da, double* dlogp_db, double* dlogp_dL) {
    constexpr bool F64 = sizeof(T) == 8;
    const int M = qmc->n_shifts;
    const int64_t Ns = qmc->n_points, Ntot = Ns * M;
    const int64_t ntiles = (Ntot + SOV_P - 1) / SOV_P;
    const int nn = std::max(n, 1);
    const int64_t ystride = (int64_t)nn * SOV_P;
    // path tiles whose y and ybar fit under the context's limit; more tiles than that run in
    // batches, each recomputing its forward sweep after a first forward pass over all paths has
    // given the log-weights (and so the softmax weights of every path)
    const int64_t per_tile = 2 * ystride * (int64_t)sizeof(T);
    const int64_t batch_tiles =
        std::max<int64_t>(1, std::min<int64_t>(ntiles, ctx->grad_y_limit / per_tile));
    const int64_t nbatch = (ntiles + batch_tiles - 1) / batch_tiles;
    if ((double)ntiles * RV_ITEMS_PER_TILE * 3.0 * nn * 8.0 > 100e9)
        return mvn_fail(ctx, MVN_ERR_ARG, "gradient partial sums beyond 100 GB");
    MVN_TRY(lattice_ensure(ctx, nn));
    const size_t need = ws_round(sizeof(uint64_t) * (size_t)M * nn) + ws_round(sizeof(double) * Ntot) * 2 +
                        2 * ws_round(sizeof(T) * (size_t)batch_tiles * ystride) +
                        ws_round(sizeof(double) * 3 * (size_t)RV_ITEMS_PER_TILE * ntiles * nn) +
                        ws_round(sizeof(double) * 3 * (size_t)nn) + 4 * ws_round(sizeof(double)) + 4096;
    MVN_TRY(ws_reserve(ctx, need));
    WsCarver wc(ctx->ws);
    uint64_t* delta = wc.take<uint64_t>((size_t)M * nn);
    double* logw = wc.take<double>(Ntot);
    double* omega = wc.take<double>(Ntot);
    T* Y = wc.take<T>((size_t)batch_tiles * ystride);
    T* Sb = wc.take<T>((size_t)batch_tiles * ystride);
    double* part = wc.take<double>(3 * (size_t)RV_ITEMS_PER_TILE * ntiles * nn);
    double* dsum = wc.take<double>(3 * (size_t)nn);
    double* lse = wc.take<double>(1);
    int* counter = wc.take<int>(2);
    MVN_TRY(check_limits_device(ctx, n, a, b));
    MVN_TRY(lattice_shifts(ctx, qmc->seed, M, nn, delta));
    SovProblem P;
    memset(&P, 0, sizeof(P));
    P.n = n;
    P.M = M;
    P.Ns = Ns;
    P.Ntot = Ntot;
    P.a = a;
    P.b = b;
    P.L = L;
    P.ld = ld;
    P.delta = delta;
    P.dstride = nn;
    P.logw = logw;
    int fwd_per_sm = 1, rev_per_sm = 1;
    MVN_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fwd_per_sm, k_sov_fwd_keep<T>,
                                                                RV_THREADS, 0));
    MVN_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&rev_per_sm, k_sov_rev<T>,
                                                                RV_THREADS, 0));
    // the problem restricted to path tiles [t0, t0 + nt): its paths start at p0 = 128 t0
    auto batch_problem = [&](int64_t t0, int64_t nt) {
        SovProblem B = P;
        B.p0 = t0 * SOV_P;
        B.Ntot = std::min<int64_t>(Ntot - B.p0, nt * SOV_P);
        B.logw = logw + B.p0;
        return B;
    };
    // forward sweep keeping the batch's y (32-path work items, four per tile, persistent grid)
    auto forward = [&](const SovProblem& B, int64_t nt) -> mvn_status {
        MVN_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(int), ctx->stream));
        const int nfwd = (int)(RV_ITEMS_PER_TILE * nt);
        const int grid_fwd = std::max(1, std::min(nfwd, std::max(fwd_per_sm, 1) * ctx->sm_count));
        MVN_TIMED(ctx, F64 ? "k_sov_grad_fwd_f64" : "k_sov_grad_fwd_f32",
                  (k_sov_fwd_keep<T><<<grid_fwd, RV_THREADS, 0, ctx->stream>>>(
                      B, nfwd, counter, ctx->d_alpha, Y, ystride)));
        return MVN_OK;
    };
    if (n == 0) {
        MVN_CUDA(ctx, cudaMemsetAsync(logw, 0, sizeof(double) * Ntot, ctx->stream));
    } else {
        for (int64_t t0 = 0; t0 < ntiles; t0 += batch_tiles) {
            const int64_t nt = std::min(batch_tiles, ntiles - t0);
            MVN_TRY(forward(batch_problem(t0, nt), nt));
        }
    }
    MVN_TRY(sov_reduce_launch_opt(ctx, logw, Ns, M, qmc->err_k, out3, 1, Ntot, true));
    k_lse_all<<<1, 512, 0, ctx->stream>>>(logw, Ntot, lse);
    MVN_LAUNCHED(ctx);
    k_weights<<<(unsigned)((Ntot + 255) / 256), 256, 0, ctx->stream>>>(logw, Ntot, lse, omega);
    MVN_LAUNCHED(ctx);
    if (n == 0) return MVN_OK;
    const int T64 = (n + 63) / 64;
    for (int64_t t0 = 0; t0 < ntiles; t0 += batch_tiles) {
        const int64_t nt = std::min(batch_tiles, ntiles - t0);
        const SovProblem B = batch_problem(t0, nt);
        if (nbatch > 1) MVN_TRY(forward(B, nt));  // the batch's y again (the buffer was reused)
        // reverse sweep: work items of 32 paths (four per tile), persistent grid
        const int nrev = (int)(RV_ITEMS_PER_TILE * nt);
        const int grid_rev = std::max(1, std::min(nrev, std::max(rev_per_sm, 1) * ctx->sm_count));
        MVN_CUDA(ctx, cudaMemsetAsync(counter + 1, 0, sizeof(int), ctx->stream));
        double* part_b = part + (size_t)RV_ITEMS_PER_TILE * t0 * 3 * n;
        MVN_TIMED(ctx, F64 ? "k_sov_rev_f64" : "k_sov_rev_f32",
                  (k_sov_rev<T><<<grid_rev, RV_THREADS, 0, ctx->stream>>>(
                      B, nrev, counter + 1, ctx->d_alpha, Y, Sb, ystride, omega + B.p0,
                      part_b)));
        if (dlogp_dL && nbatch > 1) {
            MVN_TIMED(ctx, F64 ? "k_grad_L_f64" : "k_grad_L_f32",
                      (k_grad_L<T><<<(unsigned)((int64_t)T64 * (T64 + 1) / 2), 256, 0,
                                     ctx->stream>>>(n, (int)nt, B.Ntot, Sb, Y, omega + B.p0,
                                                    dsum, dlogp_dL, ld, t0 == 0 ? 1 : 2)));
        }
    }
    const int nrev_all = (int)(RV_ITEMS_PER_TILE * ntiles);
    k_sum_parts<<<dim3((n + 255) / 256, 3), 256, 0, ctx->stream>>>(part, nrev_all, n, dsum);
    MVN_LAUNCHED(ctx);
    if (dlogp_da)
        MVN_CUDA(ctx, cudaMemcpyAsync(dlogp_da, dsum, sizeof(double) * n,
                                      cudaMemcpyDeviceToDevice, ctx->stream));
    if (dlogp_db)
        MVN_CUDA(ctx, cudaMemcpyAsync(dlogp_db, dsum + n, sizeof(double) * n,
                                      cudaMemcpyDeviceToDevice, ctx->stream));
    if (dlogp_dL) {
        if (nbatch == 1) {
            MVN_TIMED(ctx, F64 ? "k_grad_L_f64" : "k_grad_L_f32",
                      (k_grad_L<T><<<(unsigned)((int64_t)T64 * (T64 + 1) / 2), 256, 0,
                                     ctx->stream>>>(n, (int)ntiles, Ntot, Sb, Y, omega, dsum,
                                                    dlogp_dL, ld, 0)));
        } else {
            k_grad_diag<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, dsum, dlogp_dL, ld);
            MVN_LAUNCHED(ctx);
        }
    }
    return MVN_OK;
}

extern "C" mvn_status mvn_grad_set_ylimit(mvn_ctx* ctx, int64_t bytes) {
    if (!ctx) return MVN_ERR_ARG;
    if (bytes < 0) return mvn_fail(ctx, MVN_ERR_ARG, "negative limit");
    ctx->grad_y_limit = bytes > 0 ? bytes : MVN_GRAD_Y_LIMIT_DEFAULT;
    return MVN_OK;
}

extern "C" mvn_status mvn_sov_grad(mvn_ctx* ctx, int n, const double* a, const double* b,
                                   const double* L, int64_t ld, const mvn_qmc* qmc,
                                   mvn_prec prec, double* out3, double* dlogp_da,
                                   double* dlogp_db, double* dlogp_dL) {
    if (!ctx) return MVN_ERR_ARG;
    MVN_TRY(check_qmc(ctx, qmc));
    MVN_TRY(check_problem_host(ctx, n, a, b, L, ld));
    if (!out3) return mvn_fail(ctx, MVN_ERR_ARG, "out3 is null");
    if (prec != MVN_FP64 && prec != MVN_MIXED && prec != MVN_MIXED_SIMT)
        return mvn_fail(ctx, MVN_ERR_ARG, "unknown precision");
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    if (prec == MVN_FP64)
        return sov_grad_run<double>(ctx, n, a, b, L, ld, qmc, out3, dlogp_da, dlogp_db, dlogp_dL);
    return sov_grad_run<float>(ctx, n, a, b, L, ld, qmc, out3, dlogp_da, dlogp_db, dlogp_dL);
}
