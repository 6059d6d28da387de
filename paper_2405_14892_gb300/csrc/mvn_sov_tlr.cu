// mvn_sov_tlr.cu -- the SOV sweep on a tile low-rank Cholesky factor (Sec. III-E; the
// limit-update step (c) of Alg. 2 with the off-diagonal factor tiles kept low rank).
//
// With L_rc = U_rc V_rc^T for the tiles c < r of block row r, the limit shifts of block r are
//   s_r = sum_{c<r} U_rc (V_rc^T y_c)
// (2 m k_rc multiply-adds per path and tile instead of m^2), and the diagonal tile L_rr is dense.
// The paper's sweep expands the factor to a dense matrix first; here the factor stays in its
// compressed form, so the sweep's work follows the ranks.
//
// Design (GB300): one CTA owns a work item of 32 paths with four threads per path (128 threads),
// persistent over the items, so that a problem of 10,000 paths fills every SM.  Block row r:
// (A) for every earlier tile c and every chunk of 8 rank components, t = V_rc^T y_c, each thread
// summing a quarter of the rows (V staged through shared memory 64 rows at a time, y_c read from
// the CTA's own y buffer), the quarters added by shuffles and kept in a per-CTA buffer; (B) for
// 64 rows of block r at a time, each thread sums U_rc t over every c and component for 16 of
// them in registers and writes their shifts once; then the dense diagonal tile runs in blocks of
// 16 dimensions (the earlier dimensions of the tile as a mat-vec split over the four threads,
// then the block's dimensions one at a time with the elementwise step of Eq. 2, computed by all
// four threads of the path alike).
#include <math.h>
#include <string.h>

#include <algorithm>

#include "mvn_internal.cuh"
#include "mvn_sov.cuh"
#include "mvn_sov_simt.cuh"
#include "mvn_tlr.cuh"

#define LR_K 8     // rank components per chunk
#define LR_R 64    // rows of U / V / D staged per step
#define LR_PATHS 32  // paths per work item
#define LR_PARTS 4   // threads per path
#define LR_THREADS (LR_PATHS * LR_PARTS)
#define LR_B 16    // dimensions per diagonal block

struct TlrSweep {
    SovProblem P;            // limits, lattice, log-weights (P.L unused)
    int m, nt, kmax;
    const double* D;         // diagonal factor tiles, m x m (ld m)
    const double* U;         // off-diagonal tiles, m x kmax (ld m) each, tri_index order
    const double* V;
    const int* rank;         // per off-diagonal tile
    int nitems;              // 32-path work items
    int* counter;            // work-queue head (zeroed before the launch)
};

__device__ __forceinline__ int64_t lr_tri(int i, int j, int nt) {
    return (int64_t)j * nt - (int64_t)j * (j + 1) / 2 + (i - j - 1);
}

template <typename T>
struct LrSmem {
    T W[LR_R][LR_K + 1];      // a staged chunk of V or U (rows x rank components)
    T Ds[LR_B][LR_R + 1];     // a staged chunk of the diagonal tile (block rows x columns)
    T Dd[LR_B][LR_B + 1];     // the block's own lower triangle
    double a[LR_B], b[LR_B];
    uint64_t alpha[LR_B];
};

// Sum over the four threads of a path (adjacent lanes).
template <typename T>
__device__ __forceinline__ T lr_sum4(T v) {
    v += __shfl_xor_sync(0xffffffffu, v, 1);
    v += __shfl_xor_sync(0xffffffffu, v, 2);
    return v;
}

// One 32-path item.  Thread t: path pl = t / 4 of the item, part q = t % 4.  Y, S and the rank
// products are per-CTA buffers laid out [row][32 paths].
template <typename T, bool ELEM64>
__device__ void tlr_item(const TlrSweep& S, int item, const uint64_t* __restrict__ alpha,
                         T* __restrict__ Y, T* __restrict__ Sb, T* __restrict__ Tb,
                         LrSmem<T>& sm) {
    const SovProblem& P = S.P;
    const int t = threadIdx.x, pl = t >> 2, q = t & 3;
    const int n = P.n, m = S.m;
    const int64_t p = (int64_t)item * LR_PATHS + pl;
    const bool valid = p < P.Ntot;
    const int64_t pg = P.p0 + p;
    const int64_t qs = valid ? pg / P.Ns : 0;
    const uint64_t j = valid ? (uint64_t)(pg - qs * P.Ns) + 1u : 1u;
    const uint64_t* __restrict__ dq = P.delta + qs * P.dstride;
    LogProd lp;
    for (int r = 0; r < S.nt; ++r) {
        const int r0 = r * m;
        const int mr = min(m, n - r0);
        // (A) rank products t_c = V_rc^T y_c for every c < r (each thread a quarter of the rows)
        int toff = 0;
        for (int c = 0; c < r; ++c) {
            const int64_t idx = lr_tri(r, c, S.nt);
            const int k = S.rank[idx];
            const double* __restrict__ Vc = S.V + idx * (int64_t)m * S.kmax;
            const T* __restrict__ yc = Y + (int64_t)c * m * LR_PATHS;
            for (int k0 = 0; k0 < k; k0 += LR_K) {
                const int kn = min(LR_K, k - k0);
                T tt[LR_K];
#pragma unroll
                for (int kk = 0; kk < LR_K; ++kk) tt[kk] = (T)0;
                for (int u0 = 0; u0 < m; u0 += LR_R) {
                    __syncthreads();
                    for (int e = t; e < LR_R * LR_K; e += LR_THREADS) {
                        const int uu = e % LR_R, kk = e / LR_R;
                        sm.W[uu][kk] = (kk < kn) ? (T)Vc[(u0 + uu) + (int64_t)(k0 + kk) * m] : (T)0;
                    }
                    __syncthreads();
#pragma unroll 4
                    for (int i = 0; i < LR_R / LR_PARTS; ++i) {
                        const int uu = LR_PARTS * i + q;
                        const T y = yc[(int64_t)(u0 + uu) * LR_PATHS + pl];
#pragma unroll
                        for (int kk = 0; kk < LR_K; ++kk) tt[kk] = fma(sm.W[uu][kk], y, tt[kk]);
                    }
                }
#pragma unroll
                for (int kk = 0; kk < LR_K; ++kk) {
                    tt[kk] = lr_sum4(tt[kk]);
                    if (kk < kn && (kk & 3) == q)
                        Tb[(int64_t)(toff + k0 + kk) * LR_PATHS + pl] = tt[kk];
                }
            }
            toff += k;
        }
        __syncthreads();  // the rank products are visible to all four threads of a path
        // (B) shifts of 64 rows at a time: s_v = sum_c sum_k U_rc(v, k) t_c(k), each thread 16 rows
        for (int v0 = 0; v0 < mr; v0 += LR_R) {
            const int vn = min(LR_R, mr - v0);
            T acc[LR_R / LR_PARTS];
#pragma unroll
            for (int i = 0; i < LR_R / LR_PARTS; ++i) acc[i] = (T)0;
            int off = 0;
            for (int c = 0; c < r; ++c) {
                const int64_t idx = lr_tri(r, c, S.nt);
                const int k = S.rank[idx];
                const double* __restrict__ Uc = S.U + idx * (int64_t)m * S.kmax;
                for (int k0 = 0; k0 < k; k0 += LR_K) {
                    const int kn = min(LR_K, k - k0);
                    __syncthreads();
                    for (int e = t; e < LR_R * LR_K; e += LR_THREADS) {
                        const int vv = e % LR_R, kk = e / LR_R;
                        sm.W[vv][kk] = (kk < kn && vv < vn)
                                           ? (T)Uc[(v0 + vv) + (int64_t)(k0 + kk) * m]
                                           : (T)0;
                    }
                    __syncthreads();
                    T tt[LR_K];
#pragma unroll
                    for (int kk = 0; kk < LR_K; ++kk)
                        tt[kk] = (kk < kn) ? Tb[(int64_t)(off + k0 + kk) * LR_PATHS + pl] : (T)0;
#pragma unroll
                    for (int i = 0; i < LR_R / LR_PARTS; ++i)
#pragma unroll
                        for (int kk = 0; kk < LR_K; ++kk)
                            acc[i] = fma(sm.W[q * (LR_R / LR_PARTS) + i][kk], tt[kk], acc[i]);
                }
                off += k;
            }
#pragma unroll
            for (int i = 0; i < LR_R / LR_PARTS; ++i) {
                const int vv = q * (LR_R / LR_PARTS) + i;
                if (vv < vn) Sb[(int64_t)(v0 + vv) * LR_PATHS + pl] = acc[i];
            }
        }
        __syncthreads();
        // dense diagonal tile r in blocks of 16 dimensions
        const double* __restrict__ Dr = S.D + (int64_t)r * m * m;
        for (int b0 = 0; b0 < mr; b0 += LR_B) {
            const int nb = min(LR_B, mr - b0);
            // earlier dimensions of the tile: a quarter of the columns per thread, then summed
            T acc[LR_B];
#pragma unroll
            for (int v = 0; v < LR_B; ++v) acc[v] = (T)0;
            for (int k0 = 0; k0 < b0; k0 += LR_R) {
                const int kw = min(LR_R, b0 - k0);
                __syncthreads();
                for (int e = t; e < LR_B * LR_R; e += LR_THREADS) {
                    const int v = e % LR_B, kk = e / LR_B;
                    sm.Ds[v][kk] = (v < nb && kk < kw) ? (T)Dr[(b0 + v) + (int64_t)(k0 + kk) * m]
                                                        : (T)0;
                }
                __syncthreads();
                for (int kk = q; kk < kw; kk += LR_PARTS) {
                    const T yk = Y[(int64_t)(r0 + k0 + kk) * LR_PATHS + pl];
#pragma unroll
                    for (int v = 0; v < LR_B; ++v) acc[v] = fma(sm.Ds[v][kk], yk, acc[v]);
                }
            }
#pragma unroll
            for (int v = 0; v < LR_B; ++v) acc[v] = lr_sum4(acc[v]);
            __syncthreads();
            for (int e = t; e < LR_B * LR_B; e += LR_THREADS) {
                const int v = e % LR_B, u = e / LR_B;
                sm.Dd[v][u] = (v < nb && u <= v) ? (T)Dr[(b0 + v) + (int64_t)(b0 + u) * m] : (T)0;
            }
            if (t < LR_B) {
                const int g = r0 + b0 + t;
                sm.a[t] = (t < nb) ? P.a[g] : 0.0;
                sm.b[t] = (t < nb) ? P.b[g] : 1.0;
                sm.alpha[t] = (t < nb) ? alpha[g] : 0u;
            }
            __syncthreads();
            // the block's dimensions in order (every thread of a path computes the same values)
            T y[LR_B];
#pragma unroll
            for (int v = 0; v < LR_B; ++v) {
                if (v < nb) {
                    T s = acc[v] + Sb[(int64_t)(b0 + v) * LR_PATHS + pl];
#pragma unroll
                    for (int u = 0; u < v; ++u) s = fma(sm.Dd[v][u], y[u], s);
                    const double w = lattice_w(j, sm.alpha[v], dq[r0 + b0 + v]);
                    double delta;
                    if constexpr (ELEM64) {
                        y[v] = (T)sov_step_f64(sm.a[v], sm.b[v], (double)s, (double)sm.Dd[v][v], w,
                                               delta);
                    } else {
                        y[v] = (T)sov_step_f32(sm.a[v], sm.b[v], (float)s, (float)sm.Dd[v][v], w,
                                               delta);
                    }
                    lp.mul(delta);
                    if ((v & 3) == q) Y[(int64_t)(r0 + b0 + v) * LR_PATHS + pl] = y[v];
                } else {
                    y[v] = (T)0;
                }
            }
            __syncthreads();  // the block's y are visible to every part before they are read
        }
    }
    if (valid && q == 0 && P.logw) P.logw[p] = lp.log_value();
}

template <typename T, bool ELEM64>
__global__ void __launch_bounds__(LR_THREADS, 4) k_sov_tlr(const TlrSweep S,
                                                        const uint64_t* __restrict__ alpha,
                                                        T* __restrict__ Yscratch, int64_t ystride,
                                                        T* __restrict__ Sscratch, int64_t sstride,
                                                        T* __restrict__ Tscratch,
                                                        int64_t tstride) {
    __shared__ LrSmem<T> sm;
    __shared__ int s_item;
    T* Y = Yscratch + (int64_t)blockIdx.x * ystride;
    T* Sb = Sscratch + (int64_t)blockIdx.x * sstride;
    T* Tb = Tscratch + (int64_t)blockIdx.x * tstride;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(S.counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= S.nitems) break;
        tlr_item<T, ELEM64>(S, it, alpha, Y, Sb, Tb, sm);
    }
}

extern "C" mvn_status mvn_sov_tlr(mvn_ctx* ctx, const mvn_tlr* Lt, const double* a,
                                  const double* b, const mvn_qmc* qmc, mvn_prec prec,
                                  double* out3, double* path_logw) {
    if (!ctx) return MVN_ERR_ARG;
    if (!Lt || !Lt->factored)
        return mvn_fail(ctx, MVN_ERR_ARG, "mvn_sov_tlr: needs a factored TLR object");
    MVN_TRY(check_qmc(ctx, qmc));
    const int n = Lt->n, m = Lt->m;
    if (!a || !b || !out3) return mvn_fail(ctx, MVN_ERR_ARG, "mvn_sov_tlr: null pointer");
    if (prec != MVN_FP64 && prec != MVN_MIXED && prec != MVN_MIXED_SIMT)
        return mvn_fail(ctx, MVN_ERR_ARG, "unknown precision");
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    const bool f64 = (prec == MVN_FP64);
    const size_t elt = f64 ? sizeof(double) : sizeof(float);
    const int M = qmc->n_shifts;
    const int64_t Ns = qmc->n_points, Ntot = Ns * M;
    const int64_t nitems = (Ntot + LR_PATHS - 1) / LR_PATHS;
    if (nitems > (1 << 30)) return mvn_fail(ctx, MVN_ERR_ARG, "too many path items");
    MVN_TRY(lattice_ensure(ctx, n));
    int occ = 1;
    if (f64) {
        MVN_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sov_tlr<double, true>,
                                                                    LR_THREADS, 0));
    } else {
        MVN_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_sov_tlr<float, false>,
                                                                    LR_THREADS, 0));
    }
    const int grid = (int)std::max<int64_t>(
        1, std::min<int64_t>(nitems, (int64_t)ctx->sm_count * std::max(occ, 1)));
    // the largest sum over c < r of the ranks of block row r (entries of t per path)
    int64_t tmax = 1;
    for (int r = 1; r < Lt->nt; ++r) {
        int64_t sr = 0;
        for (int c = 0; c < r; ++c) sr += Lt->rank_h[(size_t)tri_index(r, c, Lt->nt)];
        tmax = std::max(tmax, sr);
    }
    const int64_t ystride = (int64_t)Lt->npad * LR_PATHS, sstride = (int64_t)m * LR_PATHS,
                  tstride = tmax * LR_PATHS;
    const size_t need = ws_round(sizeof(uint64_t) * (size_t)M * n) +
                        (path_logw ? 0 : ws_round(sizeof(double) * (size_t)Ntot)) +
                        ws_round(elt * (size_t)ystride * grid) +
                        ws_round(elt * (size_t)sstride * grid) +
                        ws_round(elt * (size_t)tstride * grid) + ws_round(sizeof(int)) + 1024;
    MVN_TRY(ws_reserve(ctx, need));
    WsCarver wc(ctx->ws);
    uint64_t* delta = wc.take<uint64_t>((size_t)M * n);
    double* logw = path_logw ? path_logw : wc.take<double>((size_t)Ntot);
    void* Ybuf = wc.take<char>(elt * (size_t)ystride * grid);
    void* Sbuf = wc.take<char>(elt * (size_t)sstride * grid);
    void* Tbuf = wc.take<char>(elt * (size_t)tstride * grid);
    int* counter = wc.take<int>(1);
    TlrSweep S;
    memset(&S, 0, sizeof(S));
    SovProblem& P = S.P;
    P.n = n;
    P.M = M;
    P.Ns = Ns;
    P.Ntot = Ntot;
    P.p0 = 0;
    P.a = a;
    P.b = b;
    P.delta = delta;
    P.dstride = n;
    P.logw = logw;
    S.m = m;
    S.nt = Lt->nt;
    S.kmax = Lt->kmax;
    S.D = Lt->D;
    S.U = Lt->U;
    S.V = Lt->V;
    S.rank = Lt->rank;
    S.nitems = (int)nitems;
    S.counter = counter;
    MVN_TRY(check_limits_device(ctx, n, a, b));
    MVN_TRY(lattice_shifts(ctx, qmc->seed, M, n, delta));
    MVN_CUDA(ctx, cudaMemsetAsync(counter, 0, sizeof(int), ctx->stream));
    if (f64) {
        MVN_TIMED(ctx, "k_sov_tlr_f64",
                  (k_sov_tlr<double, true><<<grid, LR_THREADS, 0, ctx->stream>>>(
                      S, ctx->d_alpha, (double*)Ybuf, ystride, (double*)Sbuf, sstride,
                      (double*)Tbuf, tstride)));
    } else {
        MVN_TIMED(ctx, "k_sov_tlr_f32",
                  (k_sov_tlr<float, false><<<grid, LR_THREADS, 0, ctx->stream>>>(
                      S, ctx->d_alpha, (float*)Ybuf, ystride, (float*)Sbuf, sstride,
                      (float*)Tbuf, tstride)));
    }
    return sov_reduce_launch(ctx, logw, Ns, M, qmc->err_k, out3, 1, Ntot);
}
