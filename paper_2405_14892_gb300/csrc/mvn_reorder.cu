// mvn_reorder.cu -- Cholesky factorisation with the univariate variable reordering of Gibson,
// Glasbey and Elston (1994; Genz and Bretz 2009, Sec. 4.1.3), a variance-reducing variant of the
// SOV estimator of Eq. 2 that the paper does not use: step i places next the variable whose
// conditional interval probability Phi(b'_j) - Phi(a'_j) is smallest, with
//   d_j = Sigma_jj - sum_{k<i} L_jk^2,  s_j = sum_{k<i} L_jk y_k,
//   a'_j = (a_j - s_j) / sqrt(d_j),  b'_j = (b_j - s_j) / sqrt(d_j),
// y_k the truncated-normal mean E[Z | a'_k < Z < b'_k] of the variables already placed; ties go to
// the variable earliest in the current order.
//
// Design (GB300, FP64): right-looking over 64-wide panels.  Inside a panel every column is one
// pivoted step of three small kernels -- the criterion over all remaining variables with a
// block-then-last-block arg-min, the symmetric swap of the chosen variable into place (rows of the
// factor so far, row and column of the not-yet-factored block), and the new column of the factor
// over all remaining rows (the panel's earlier columns subtracted, d and s updated).  After the
// panel the trailing block is updated by the FP64 tile SYRK of the plain Cholesky.  The vectors
// d, s and the limits stay in global memory (L2-resident); the panel's columns are read from L2
// by every step.
#include <math.h>

#include <algorithm>

#include "mvn_internal.cuh"

#define RO_NB 64
#define RO_THREADS 256
#define RO_MAX_BLOCKS 1024

// FP64 tile SYRK of the right-looking Cholesky (mvn_chol.cu)
__global__ void k_syrk(double* __restrict__ A, int64_t ld, int k0, int nb, int c0, int n,
                       const int* status);

__device__ __forceinline__ bool ro_failed(const int* status) {
    return *(volatile const int*)status != 0;
}

__device__ __forceinline__ double ro_Phi(double x) { return 0.5 * erfc(-x * 0.70710678118654752440); }
__device__ __forceinline__ double ro_Q(double x) { return 0.5 * erfc(x * 0.70710678118654752440); }

// conditional interval probability of standardised limits, tail-stable
__device__ __forceinline__ double ro_interval(double ap, double bp) {
    if (ap > 0.0) return ro_Q(ap) - ((bp == INFINITY) ? 0.0 : ro_Q(bp));
    return ((bp == INFINITY) ? 1.0 : ro_Phi(bp)) - ((ap == -INFINITY) ? 0.0 : ro_Phi(ap));
}

// truncated-normal mean of the placed variable (phi(a') - phi(b')) / (Phi(b') - Phi(a')); an
// interval probability that underflows takes the finite limit
__device__ __forceinline__ double ro_trunc_mean(double ap, double bp) {
    const double den = ro_interval(ap, bp);
    const double pa = (ap == -INFINITY) ? 0.0 : 0.39894228040143267794 * exp(-0.5 * ap * ap);
    const double pb = (bp == INFINITY) ? 0.0 : 0.39894228040143267794 * exp(-0.5 * bp * bp);
    return (den > 0.0) ? (pa - pb) / den : ((ap > 0.0) ? ap : bp);
}

__global__ void k_ro_init(int n, const double* __restrict__ A, int64_t ld,
                          const double* __restrict__ a, const double* __restrict__ b,
                          int32_t* __restrict__ perm, double* __restrict__ ap,
                          double* __restrict__ bp, double* __restrict__ d,
                          double* __restrict__ s) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    perm[i] = i;
    ap[i] = a[i];
    bp[i] = b[i];
    d[i] = A[i + (int64_t)i * ld];
    s[i] = 0.0;
}

// Step i: arg-min of the criterion over j in [i, n).  Each block reduces its rows (smaller j on
// ties) and the last block to finish reduces the blocks' results in block order; sel[0] receives
// the chosen j, or -1 with MVN_ERR_NOT_PD (info i + 1) if no conditional variance is positive.
__global__ void __launch_bounds__(RO_THREADS) k_ro_pick(int i, int n, const double* __restrict__ d,
                                                        const double* __restrict__ s,
                                                        const double* __restrict__ ap,
                                                        const double* __restrict__ bp,
                                                        double* __restrict__ pval,
                                                        int* __restrict__ pidx, int* counter,
                                                        int* sel, int* status) {
    __shared__ double sv[RO_THREADS];
    __shared__ int si[RO_THREADS];
    __shared__ bool last;
    if (ro_failed(status)) return;
    const int t = threadIdx.x;
    double best = INFINITY;
    int bj = -1;
    for (int j = i + blockIdx.x * RO_THREADS + t; j < n; j += gridDim.x * RO_THREADS) {
        const double dj = d[j];
        if (!(dj > 0.0)) continue;
        const double sd = sqrt(dj);
        const double c = ro_interval((ap[j] - s[j]) / sd, (bp[j] - s[j]) / sd);
        if (bj < 0 || c < best) {  // j grows along the loop: a tie keeps the earlier one
            best = c;
            bj = j;
        }
    }
    sv[t] = best;
    si[t] = bj;
    __syncthreads();
    for (int w = RO_THREADS / 2; w > 0; w >>= 1) {
        if (t < w) {
            const int oj = si[t + w];
            if (oj >= 0 && (si[t] < 0 || sv[t + w] < sv[t] || (sv[t + w] == sv[t] && oj < si[t]))) {
                sv[t] = sv[t + w];
                si[t] = oj;
            }
        }
        __syncthreads();
    }
    if (t == 0) {
        pval[blockIdx.x] = sv[0];
        pidx[blockIdx.x] = si[0];
        __threadfence();
        last = (atomicAdd(counter, 1) == (int)gridDim.x - 1);
    }
    __syncthreads();
    if (!last || t != 0) return;
    __threadfence();
    double bv = INFINITY;
    int bjj = -1;
    for (int k = 0; k < (int)gridDim.x; ++k) {
        const int oj = ((volatile int*)pidx)[k];
        const double ov = ((volatile double*)pval)[k];
        if (oj >= 0 && (bjj < 0 || ov < bv || (ov == bv && oj < bjj))) {
            bv = ov;
            bjj = oj;
        }
    }
    *counter = 0;
    *sel = bjj;
    if (bjj < 0) dev_raise(status, MVN_ERR_NOT_PD, i + 1);
}

// Step i: swap the chosen variable p = sel[0] into place i.  Thread k moves one pair:
//   k < i      : the factor's rows i and p in column k
//   k == i     : the diagonal entries (i, i) and (p, p) of the not-yet-factored block
//   i < k < p  : (k, i) and (p, k)   (lower triangle: row p's entries left of the diagonal)
//   k > p      : (k, i) and (k, p)
// and thread 0 the scalars of the two variables.  (p, i) stays where it is.
__global__ void k_ro_swap(int i, int n, double* __restrict__ A, int64_t ld, const int* sel,
                          int32_t* __restrict__ perm, double* __restrict__ ap,
                          double* __restrict__ bp, double* __restrict__ d,
                          double* __restrict__ s, const int* status) {
    if (ro_failed(status)) return;
    const int p = *sel;
    if (p <= i) return;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n || k == p) return;
    int64_t x, y;
    if (k < i) {
        x = i + (int64_t)k * ld;
        y = p + (int64_t)k * ld;
    } else if (k == i) {
        x = i + (int64_t)i * ld;
        y = p + (int64_t)p * ld;
    } else if (k < p) {
        x = k + (int64_t)i * ld;
        y = p + (int64_t)k * ld;
    } else {
        x = k + (int64_t)i * ld;
        y = k + (int64_t)p * ld;
    }
    const double t = A[x];
    A[x] = A[y];
    A[y] = t;
    if (k == 0) {  // thread 0 is never p (p > i >= 0)
        int32_t tq = perm[i];
        perm[i] = perm[p];
        perm[p] = tq;
        double u = ap[i];
        ap[i] = ap[p];
        ap[p] = u;
        u = bp[i];
        bp[i] = bp[p];
        bp[p] = u;
        u = d[i];
        d[i] = d[p];
        d[p] = u;
        u = s[i];
        s[i] = s[p];
        s[p] = u;
    }
}

// Step i: column i of the factor over the rows j >= i.  The block holds row i of the panel's
// earlier columns c0..i-1 in shared memory; L_ii = sqrt(d_i), L_ji = (A_ji - sum_{k in [c0, i)}
// L_jk L_ik) / L_ii (A is up to date through column c0), then d_j -= L_ji^2 and s_j += L_ji y_i
// with y_i the truncated-normal mean of the placed variable (every block recomputes it).
__global__ void __launch_bounds__(RO_THREADS) k_ro_col(int i, int c0, int n,
                                                       double* __restrict__ A, int64_t ld,
                                                       double* __restrict__ d,
                                                       double* __restrict__ s,
                                                       const double* __restrict__ ap,
                                                       const double* __restrict__ bp,
                                                       const int* status) {
    __shared__ double li[RO_NB];
    if (ro_failed(status)) return;
    const int t = threadIdx.x;
    const int w = i - c0;
    for (int k = t; k < w; k += RO_THREADS) li[k] = A[i + (int64_t)(c0 + k) * ld];
    __syncthreads();
    const double lii = sqrt(d[i]);
    const double si = s[i];
    const double yi = ro_trunc_mean((ap[i] - si) / lii, (bp[i] - si) / lii);
    const int j = i + blockIdx.x * RO_THREADS + t;
    if (j >= n) return;
    if (j == i) {
        A[i + (int64_t)i * ld] = lii;
        return;
    }
    double v = A[j + (int64_t)i * ld];
    for (int k = 0; k < w; ++k) v -= A[j + (int64_t)(c0 + k) * ld] * li[k];
    const double l = v / lii;
    A[j + (int64_t)i * ld] = l;
    d[j] -= l * l;
    s[j] += l * yi;
}

mvn_status chol_reorder_launch(mvn_ctx* ctx, int n, double* A, int64_t ld, const double* a,
                               const double* b, int32_t* perm, double* a_perm, double* b_perm,
                               char* ws) {
    WsCarver wc(ws);
    double* d = wc.take<double>(n);
    double* s = wc.take<double>(n);
    double* pval = wc.take<double>(RO_MAX_BLOCKS);
    int* pidx = wc.take<int>(RO_MAX_BLOCKS);
    int* cnt = wc.take<int>(2);  // [0] arg-min arrival counter, [1] selected variable
    MVN_CUDA(ctx, cudaMemsetAsync(cnt, 0, 2 * sizeof(int), ctx->stream));
    k_ro_init<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, A, ld, a, b, perm, a_perm, b_perm, d,
                                                        s);
    MVN_LAUNCHED(ctx);
    for (int c0 = 0; c0 < n; c0 += RO_NB) {
        const int c1 = std::min(n, c0 + RO_NB);
        for (int i = c0; i < c1; ++i) {
            const int rows = n - i;
            const int blocks = std::max(1, std::min(RO_MAX_BLOCKS, (rows + RO_THREADS - 1) / RO_THREADS));
            k_ro_pick<<<blocks, RO_THREADS, 0, ctx->stream>>>(i, n, d, s, a_perm, b_perm, pval,
                                                             pidx, cnt, cnt + 1, ctx->d_status);
            MVN_LAUNCHED(ctx);
            k_ro_swap<<<(n + 255) / 256, 256, 0, ctx->stream>>>(i, n, A, ld, cnt + 1, perm,
                                                                a_perm, b_perm, d, s,
                                                                ctx->d_status);
            MVN_LAUNCHED(ctx);
            k_ro_col<<<(rows + RO_THREADS - 1) / RO_THREADS, RO_THREADS, 0, ctx->stream>>>(
                i, c0, n, A, ld, d, s, a_perm, b_perm, ctx->d_status);
            MVN_LAUNCHED(ctx);
        }
        if (c1 < n) {
            const int T = (n - c1 + RO_NB - 1) / RO_NB;
            const int64_t tiles = (int64_t)T * (T + 1) / 2;
            MVN_TIMED(ctx, "k_syrk",
                      (k_syrk<<<(unsigned)tiles, 256, 0, ctx->stream>>>(A, ld, c0, c1 - c0, c1, n,
                                                                       ctx->d_status)));
        }
    }
    return MVN_OK;
}

size_t chol_reorder_ws_bytes(int n) {
    return 2 * ws_round(sizeof(double) * (size_t)std::max(n, 1)) +
           ws_round(sizeof(double) * RO_MAX_BLOCKS) + ws_round(sizeof(int) * RO_MAX_BLOCKS) +
           ws_round(2 * sizeof(int)) + 1024;
}

extern "C" mvn_status mvn_cholesky_reorder(mvn_ctx* ctx, int n, double* A, int64_t ld,
                                           const double* a, const double* b, int32_t* perm,
                                           double* a_perm, double* b_perm, int* info) {
    if (!ctx) return MVN_ERR_ARG;
    if (n < 0 || n > (1 << 21) || ld < (n > 0 ? n : 1) ||
        (n > 0 && (!A || !a || !b || !perm || !a_perm || !b_perm)))
        return mvn_fail(ctx, MVN_ERR_ARG, "mvn_cholesky_reorder: invalid argument");
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    if (info) *info = 0;
    if (n > 0) {
        MVN_TRY(ws_reserve(ctx, chol_reorder_ws_bytes(n)));
        MVN_TRY(chol_reorder_launch(ctx, n, A, ld, a, b, perm, a_perm, b_perm, (char*)ctx->ws));
    }
    if (info) return mvn_sync(ctx, info);
    return MVN_OK;
}
