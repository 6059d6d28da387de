// mvn_sov.cu -- blocked SOV sweep (Eqs. 2-3, Algs. 2-3) on CUDA cores: FP64 path and the
// FP32-SIMT mixed path, the log-domain reduction (Alg. 2 "mean(p)"), the batched launch and the
// prefix recording used by the confidence-region loop (Alg. 1).
//
// Design (GB300): the only parallel axis of the method is the path (lattice point) axis
// (Sec. IV-C: dimensions depend on each other in sequence).  One CTA owns a tile of 128 paths,
// one path per thread, and walks all n dimensions in blocks of B.  For block r it forms the limit
// shift s = L(r, 0:r) y(0:r) of Alg. 2's GEMM step (c) from its own earlier y values (left-looking,
// one shift for both limits instead of separate A and B updates), then runs Alg. 3 on the
// diagonal block with the y values in registers.  Tiles are independent, so a persistent grid
// takes (problem, tile) items from a queue ordered longest first; no CTA ever waits on another.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "mvn_internal.cuh"
#include "mvn_sov.cuh"

#include "mvn_sov_simt.cuh"

// ---------------------------------------------------------------- reduction (Alg. 2 mean(p))

// Block-wide max m and sum_k exp(r_k - m) of r[0 .. cnt) in a fixed order (thread t takes
// k = t, t + nt, ...; tree reductions in shared memory `red` of blockDim.x doubles), so the
// pair does not depend on anything but the values and the block size.  Every thread gets it.
__device__ void block_max_sumexp(const double* __restrict__ r, int64_t cnt, double* red,
                                 double& m_out, double& s_out) {
    const int t = threadIdx.x, nt = blockDim.x;
    double m = -INFINITY;
    for (int64_t k = t; k < cnt; k += nt) m = fmax(m, r[k]);
    red[t] = m;
    __syncthreads();
    for (int w = nt / 2; w > 0; w >>= 1) {
        if (t < w) red[t] = fmax(red[t], red[t + w]);
        __syncthreads();
    }
    m = red[0];
    __syncthreads();
    double s = 0.0;
    if (m > -INFINITY)
        for (int64_t k = t; k < cnt; k += nt) s += exp(r[k] - m);
    red[t] = s;
    __syncthreads();
    for (int w = nt / 2; w > 0; w >>= 1) {
        if (t < w) red[t] += red[t + w];
        __syncthreads();
    }
    s_out = red[0];
    m_out = m;
    __syncthreads();
}

// log P_q of one shift from its (max, sum of exp(logw - max)) over its Ns paths.
__device__ __forceinline__ double shift_log_mean(double m, double s, int64_t Ns) {
    return (m > -INFINITY) ? m + log(s) - log((double)Ns) : -INFINITY;
}

// Alg. 2 "mean(p)" over the shifts, in the log domain, from the per-shift log means lq[0..M):
// log P = LSE_q(lq) - log M; P = exp(log P); err = err_k sd_q(P_q) / sqrt(M) (computed relative
// to P, then scaled); every weight 0 gives (-inf, 0, 0) and, if raise_numeric, MVN_ERR_NUMERIC.
// One thread, fixed order.
__device__ void estimate_from_shifts(const double* lq, int M, double err_k, double* o,
                                     int* status, int raise_numeric) {
    double m = -INFINITY;
    for (int qq = 0; qq < M; ++qq) m = fmax(m, lq[qq]);
    if (!(m > -INFINITY)) {
        o[0] = -INFINITY;
        o[1] = 0.0;
        o[2] = 0.0;
        if (raise_numeric) dev_raise(status, MVN_ERR_NUMERIC, 0);
        return;
    }
    double s = 0.0;
    for (int qq = 0; qq < M; ++qq) s += exp(lq[qq] - m);
    const double logP = m + log(s) - log((double)M);
    double mean = 0.0;
    for (int qq = 0; qq < M; ++qq) mean += exp(lq[qq] - logP);
    mean /= M;
    double ss = 0.0;
    for (int qq = 0; qq < M; ++qq) {
        double d = exp(lq[qq] - logP) - mean;
        ss += d * d;
    }
    const double sd_rel = (M > 1) ? sqrt(ss / (M - 1)) : 0.0;
    const double P = exp(logP);
    o[0] = logP;
    o[1] = P;
    o[2] = err_k * sd_rel / sqrt((double)M) * P;
}

// One block per problem: log P_q = LSE_j(logw_qj) - log Ns per shift q, then the estimate.
// Fixed reduction order (deterministic).  Raises MVN_ERR_NUMERIC if every weight is 0.
__global__ void k_sov_reduce(const double* __restrict__ logw, int64_t Ns, int M, double err_k,
                             double* __restrict__ out3, int64_t prob_stride, int* status,
                             int raise_numeric) {
    extern __shared__ double red[];  // blockDim.x + M
    double* lq = red + blockDim.x;
    const double* lw = logw + (int64_t)blockIdx.x * prob_stride;
    for (int qq = 0; qq < M; ++qq) {
        double m, s;
        block_max_sumexp(lw + (int64_t)qq * Ns, Ns, red, m, s);
        if (threadIdx.x == 0) lq[qq] = shift_log_mean(m, s, Ns);
    }
    __syncthreads();
    if (threadIdx.x == 0)
        estimate_from_shifts(lq, M, err_k, out3 + 3 * blockIdx.x, status, raise_numeric);
}

// Shard statistics: the local log-weights logw[0 .. p1 - p0) of the global paths [p0, p1);
// for every shift q, partial[2q], partial[2q+1] = (max, sum of exp(logw - max)) over the shard's
// paths of shift q, or (-inf, 0) if it has none.  One block; a shard that covers whole shifts
// gives exactly the pairs k_sov_reduce forms.
__global__ void k_sov_shift_stats(const double* __restrict__ logw, int64_t p0, int64_t p1,
                                  int64_t Ns, int M, double* __restrict__ partial) {
    extern __shared__ double red[];
    for (int qq = threadIdx.x; qq < M; qq += blockDim.x) {
        partial[2 * qq] = -INFINITY;
        partial[2 * qq + 1] = 0.0;
    }
    __syncthreads();
    if (p1 <= p0) return;
    const int q_first = (int)(p0 / Ns), q_last = (int)((p1 - 1) / Ns);
    for (int qq = q_first; qq <= q_last; ++qq) {
        const int64_t lo = max(p0, (int64_t)qq * Ns), hi = min(p1, (int64_t)(qq + 1) * Ns);
        double m, s;
        block_max_sumexp(logw + (lo - p0), hi - lo, red, m, s);
        if (threadIdx.x == 0) {
            partial[2 * qq] = m;
            partial[2 * qq + 1] = s;
        }
    }
}

// Combine the per-shift pairs of nparts shards (partials[r][2 M], disjoint path ranges that
// together cover the rule): per shift m = max_r m_r, s = sum_r s_r exp(m_r - m) in shard order,
// then the estimate.  With one shard covering all paths this is k_sov_reduce's result bit for
// bit (s_0 exp(0) = s_0).
__global__ void k_sov_combine(const double* __restrict__ partials, int nparts, int M, int64_t Ns,
                              double err_k, double* __restrict__ out3, int* status) {
    extern __shared__ double lq[];  // M
    for (int qq = threadIdx.x; qq < M; qq += blockDim.x) {
        double m = -INFINITY;
        for (int r = 0; r < nparts; ++r) m = fmax(m, partials[(int64_t)r * 2 * M + 2 * qq]);
        double s = 0.0;
        if (m > -INFINITY)
            for (int r = 0; r < nparts; ++r) {
                const double mr = partials[(int64_t)r * 2 * M + 2 * qq];
                if (mr > -INFINITY) s += partials[(int64_t)r * 2 * M + 2 * qq + 1] * exp(mr - m);
            }
        lq[qq] = shift_log_mean(m, s, Ns);
    }
    __syncthreads();
    if (threadIdx.x == 0) estimate_from_shifts(lq, M, err_k, out3, status, 1);
}

mvn_status sov_reduce_launch_opt(mvn_ctx* ctx, const double* logw, int64_t Ns, int M,
                                 double err_k, double* out3, int nprob, int64_t prob_stride,
                                 bool raise_numeric) {
    if (nprob <= 0) return MVN_OK;
    const int nt = 512;
    k_sov_reduce<<<nprob, nt, sizeof(double) * (nt + M), ctx->stream>>>(
        logw, Ns, M, err_k, out3, prob_stride, ctx->d_status, raise_numeric ? 1 : 0);
    MVN_LAUNCHED(ctx);
    return MVN_OK;
}

mvn_status sov_reduce_launch(mvn_ctx* ctx, const double* logw, int64_t Ns, int M, double err_k,
                             double* out3, int nprob, int64_t prob_stride) {
    return sov_reduce_launch_opt(ctx, logw, Ns, M, err_k, out3, nprob, prob_stride, true);
}

// ---------------------------------------------------------------- host side

mvn_status check_qmc(mvn_ctx* ctx, const mvn_qmc* qmc) {
    if (!qmc || qmc->n_points < 1 || qmc->n_shifts < 1 || qmc->n_shifts > 4096 ||
        (int64_t)qmc->n_points * qmc->n_shifts > ((int64_t)1 << 36))
        return mvn_fail(ctx, MVN_ERR_ARG,
                        "invalid QMC rule (n_points >= 1, 1 <= n_shifts <= 4096, total <= 2^36)");
    return MVN_OK;
}

mvn_status check_problem_host(mvn_ctx* ctx, int n, const double* a, const double* b,
                              const double* L, int64_t ld) {
    if (n < 0 || n > (1 << 22)) return mvn_fail(ctx, MVN_ERR_ARG, "dimension out of range");
    if (n > 0 && (!a || !b || !L)) return mvn_fail(ctx, MVN_ERR_ARG, "null pointer");
    if (ld < (n > 0 ? n : 1)) return mvn_fail(ctx, MVN_ERR_ARG, "ld < n");
    return MVN_OK;
}

// a_i <= b_i, no NaN, a_i != +inf, b_i != -inf; a violation raises MVN_ERR_ARG on the device
__global__ void k_check_limits(int n, const double* a, const double* b, int* status) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double x = a[i], y = b[i];
    if (!(x <= y) || x == INFINITY || y == -INFINITY) dev_raise(status, MVN_ERR_ARG, i + 1);
}

mvn_status check_limits_device(mvn_ctx* ctx, int n, const double* a, const double* b) {
    if (n == 0) return MVN_OK;
    k_check_limits<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, a, b, ctx->d_status);
    MVN_LAUNCHED(ctx);
    return MVN_OK;
}

static int sov_grid(mvn_ctx* ctx, mvn_prec prec, int nmax, int64_t ntiles) {
    const int occ = tune_sweep(ctx, prec, nmax, ntiles).simt_ctas_per_sm;
    int64_t g = std::min<int64_t>(ntiles, (int64_t)ctx->sm_count * occ);
    return (int)std::max<int64_t>(g, 1);
}

size_t sov_simt_ws_bytes(mvn_ctx* ctx, int nprob, int nmax, int64_t ntiles, mvn_prec prec) {
    const size_t elt = (prec == MVN_FP64) ? sizeof(double) : sizeof(float);
    const int grid = sov_grid(ctx, prec, nmax, ntiles);
    size_t b = ws_round(sizeof(int));
    if (nprob > 1)
        b += ws_round(sizeof(SovProblem) * nprob) + ws_round(sizeof(int2) * (size_t)ntiles);
    b += ws_round(elt * (size_t)std::max(nmax, 1) * SOV_P * grid);
    return b;
}

mvn_status sov_run_simt(mvn_ctx* ctx, const std::vector<SovProblem>& probs_h, mvn_prec prec,
                        char* ws) {
    const int nprob = (int)probs_h.size();
    int nmax = 0;
    int64_t ntiles = 0;
    for (auto& P : probs_h) {
        nmax = std::max(nmax, P.n);
        if (P.n > 0) ntiles += (P.Ntot + SOV_P - 1) / SOV_P;
    }
    if (ntiles == 0) return MVN_OK;
    if (ntiles > (1 << 30)) return mvn_fail(ctx, MVN_ERR_ARG, "too many path tiles");
    const bool f64 = (prec == MVN_FP64);
    const int grid = sov_grid(ctx, prec, nmax, ntiles);
    const size_t elt = f64 ? sizeof(double) : sizeof(float);
    const int64_t ystride = (int64_t)std::max(nmax, 1) * SOV_P;
    WsCarver wc(ws);
    SovBatch batch;
    batch.counter = wc.take<int>(1);
    batch.nitems = (int)ntiles;
    batch.probs = nullptr;
    batch.items = nullptr;
    batch.y_per_tile = 0;
    if (nprob == 1) {
        batch.single = probs_h[0];
    } else {
        memset(&batch.single, 0, sizeof(batch.single));
        SovProblem* d_probs = wc.take<SovProblem>(nprob);
        int2* d_items = wc.take<int2>((size_t)ntiles);
        std::vector<int> order(nprob);
        for (int i = 0; i < nprob; ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return probs_h[x].n > probs_h[y].n; });
        std::vector<int2> items;
        items.reserve((size_t)ntiles);
        for (int pi : order) {
            if (probs_h[pi].n == 0) continue;
            int64_t nt = (probs_h[pi].Ntot + SOV_P - 1) / SOV_P;
            for (int64_t tt = 0; tt < nt; ++tt) items.push_back(make_int2(pi, (int)tt));
        }
        // pageable copies: staged before returning, so the host vectors may go out of scope
        MVN_CUDA(ctx, cudaMemcpyAsync(d_probs, probs_h.data(), sizeof(SovProblem) * nprob,
                                      cudaMemcpyHostToDevice, ctx->stream));
        MVN_CUDA(ctx, cudaMemcpyAsync(d_items, items.data(), sizeof(int2) * items.size(),
                                      cudaMemcpyHostToDevice, ctx->stream));
        batch.probs = d_probs;
        batch.items = d_items;
    }
    void* d_Y = wc.take<char>(elt * (size_t)ystride * grid);
    MVN_CUDA(ctx, cudaMemsetAsync(batch.counter, 0, sizeof(int), ctx->stream));
    if (f64) {
        MVN_TIMED(ctx, "k_sov_simt_f64",
                  (k_sov_simt<32, double, true><<<grid, SOV_P, 0, ctx->stream>>>(
                      batch, ctx->d_alpha, (double*)d_Y, ystride)));
    } else {
        MVN_TIMED(ctx, "k_sov_simt_f32",
                  (k_sov_simt<64, float, false><<<grid, SOV_P, 0, ctx->stream>>>(
                      batch, ctx->d_alpha, (float*)d_Y, ystride)));
    }
    return MVN_OK;
}

size_t sov_any_ws_bytes(mvn_ctx* ctx, int nprob, int nmax, int64_t ntiles, mvn_prec prec) {
    // ntiles counts 128-path tiles, the same unit for both sweeps
    if (prec == MVN_MIXED) return sov_tc_ws_bytes(ctx, nprob, nmax, ntiles);
    return sov_simt_ws_bytes(ctx, nprob, nmax, ntiles, prec);
}

mvn_status sov_run_any(mvn_ctx* ctx, const std::vector<SovProblem>& probs, mvn_prec prec,
                       char* ws) {
    if (prec == MVN_MIXED) return sov_run_tc(ctx, probs, ws);
    return sov_run_simt(ctx, probs, prec, ws);
}

// ---------------------------------------------------------------- ABI: mvn_sov

extern "C" mvn_status mvn_sov(mvn_ctx* ctx, int n, const double* a, const double* b,
                              const double* L, int64_t ld, const mvn_qmc* qmc, mvn_prec prec,
                              double* out3, double* path_logw) {
    if (!ctx) return MVN_ERR_ARG;
    MVN_TRY(check_qmc(ctx, qmc));
    MVN_TRY(check_problem_host(ctx, n, a, b, L, ld));
    if (!out3) return mvn_fail(ctx, MVN_ERR_ARG, "out3 is null");
    if (prec != MVN_FP64 && prec != MVN_MIXED && prec != MVN_MIXED_SIMT)
        return mvn_fail(ctx, MVN_ERR_ARG, "unknown precision");
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    const int M = qmc->n_shifts;
    const int64_t Ns = qmc->n_points, Ntot = Ns * M;
    MVN_TRY(lattice_ensure(ctx, std::max(n, 1)));
    std::vector<SovProblem> probs(1);
    SovProblem& P = probs[0];
    const size_t need = ws_round(sizeof(uint64_t) * (size_t)M * std::max(n, 1)) +
                        (path_logw ? 0 : ws_round(sizeof(double) * (size_t)Ntot)) +
                        sov_any_ws_bytes(ctx, 1, n, (Ntot + 127) / 128, prec) + 1024;
    MVN_TRY(ws_reserve(ctx, need));
    WsCarver wc(ctx->ws);
    uint64_t* delta = wc.take<uint64_t>((size_t)M * std::max(n, 1));
    double* logw = path_logw ? path_logw : wc.take<double>((size_t)Ntot);
    P.n = n;
    P.M = M;
    P.Ns = Ns;
    P.Ntot = Ntot;
    P.a = a;
    P.b = b;
    P.L = L;
    P.ld = ld;
    P.delta = delta;
    P.dstride = std::max(n, 1);
    P.logw = logw;
    P.nprefix = 0;
    P.prefix = nullptr;
    P.logw_prefix = nullptr;
    MVN_TRY(check_limits_device(ctx, n, a, b));
    MVN_TRY(lattice_shifts(ctx, qmc->seed, M, n, delta));
    if (n == 0) {
        MVN_CUDA(ctx, cudaMemsetAsync(logw, 0, sizeof(double) * Ntot, ctx->stream));
    } else {
        MVN_TRY(sov_run_any(ctx, probs, prec, wc.base + ((wc.off + 255) & ~(size_t)255)));
    }
    return sov_reduce_launch(ctx, logw, Ns, M, qmc->err_k, out3, 1, Ntot);
}

// ---------------------------------------------------------------- ABI: shards of one problem
//
// The paths of the lattice rule are independent (Sec. IV-C: the QMC samples are processed in
// parallel), so one problem can be split into path ranges, one per GPU: each shard sweeps its
// range and reduces it to per-shift pairs, and the pairs of all shards combine into the estimate.

extern "C" mvn_status mvn_sov_partial(mvn_ctx* ctx, int n, const double* a, const double* b,
                                      const double* L, int64_t ld, const mvn_qmc* qmc,
                                      mvn_prec prec, int64_t p0, int64_t p1, double* partial,
                                      double* path_logw) {
    if (!ctx) return MVN_ERR_ARG;
    MVN_TRY(check_qmc(ctx, qmc));
    MVN_TRY(check_problem_host(ctx, n, a, b, L, ld));
    if (!partial) return mvn_fail(ctx, MVN_ERR_ARG, "partial is null");
    if (prec != MVN_FP64 && prec != MVN_MIXED && prec != MVN_MIXED_SIMT)
        return mvn_fail(ctx, MVN_ERR_ARG, "unknown precision");
    const int M = qmc->n_shifts;
    const int64_t Ns = qmc->n_points, Ntot = Ns * M;
    if (p0 < 0 || p1 < p0 || p1 > Ntot)
        return mvn_fail(ctx, MVN_ERR_ARG, "path range outside [0, n_points * n_shifts]");
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t cnt = p1 - p0;
    MVN_TRY(lattice_ensure(ctx, std::max(n, 1)));
    const size_t need = ws_round(sizeof(uint64_t) * (size_t)M * std::max(n, 1)) +
                        (path_logw ? 0 : ws_round(sizeof(double) * (size_t)std::max<int64_t>(cnt, 1))) +
                        sov_any_ws_bytes(ctx, 1, n, (cnt + 127) / 128, prec) + 1024;
    MVN_TRY(ws_reserve(ctx, need));
    WsCarver wc(ctx->ws);
    uint64_t* delta = wc.take<uint64_t>((size_t)M * std::max(n, 1));
    double* logw = path_logw ? path_logw : wc.take<double>((size_t)std::max<int64_t>(cnt, 1));
    std::vector<SovProblem> probs(1);
    SovProblem& P = probs[0];
    P.n = n;
    P.M = M;
    P.Ns = Ns;
    P.Ntot = cnt;
    P.p0 = p0;
    P.a = a;
    P.b = b;
    P.L = L;
    P.ld = ld;
    P.delta = delta;
    P.dstride = std::max(n, 1);
    P.logw = logw;
    P.nprefix = 0;
    P.prefix = nullptr;
    P.logw_prefix = nullptr;
    MVN_TRY(check_limits_device(ctx, n, a, b));
    MVN_TRY(lattice_shifts(ctx, qmc->seed, M, n, delta));
    if (cnt > 0) {
        if (n == 0) {
            MVN_CUDA(ctx, cudaMemsetAsync(logw, 0, sizeof(double) * cnt, ctx->stream));
        } else {
            MVN_TRY(sov_run_any(ctx, probs, prec, wc.base + ((wc.off + 255) & ~(size_t)255)));
        }
    }
    const int nt = 512;
    k_sov_shift_stats<<<1, nt, sizeof(double) * nt, ctx->stream>>>(logw, p0, p1, Ns, M, partial);
    MVN_LAUNCHED(ctx);
    return MVN_OK;
}

extern "C" mvn_status mvn_sov_combine(mvn_ctx* ctx, int nparts, const mvn_qmc* qmc,
                                      const double* partials, double* out3) {
    if (!ctx) return MVN_ERR_ARG;
    MVN_TRY(check_qmc(ctx, qmc));
    if (nparts < 1 || nparts > 65536 || !partials || !out3)
        return mvn_fail(ctx, MVN_ERR_ARG, "invalid shard list or output");
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    const int M = qmc->n_shifts;
    k_sov_combine<<<1, 256, sizeof(double) * M, ctx->stream>>>(partials, nparts, M,
                                                               qmc->n_points, qmc->err_k, out3,
                                                               ctx->d_status);
    MVN_LAUNCHED(ctx);
    return MVN_OK;
}

// ---------------------------------------------------------------- ABI: mvn_sov_batched

extern "C" mvn_status mvn_sov_batched(mvn_ctx* ctx, int nprob, const int* dims,
                                      const int64_t* limit_offsets, const double* a,
                                      const double* b, const double* L_shared, int64_t ld,
                                      const mvn_qmc* qmc, mvn_prec prec, double* out3) {
    if (!ctx) return MVN_ERR_ARG;
    MVN_TRY(check_qmc(ctx, qmc));
    if (nprob < 0 || (nprob > 0 && (!dims || !limit_offsets || !out3)))
        return mvn_fail(ctx, MVN_ERR_ARG, "invalid problem list");
    if (nprob == 0) return MVN_OK;
    int nmax = 0;
    for (int p = 0; p < nprob; ++p) {
        if (dims[p] < 0 || limit_offsets[p] < 0)
            return mvn_fail(ctx, MVN_ERR_ARG, "negative dimension or offset");
        nmax = std::max(nmax, dims[p]);
    }
    MVN_TRY(check_problem_host(ctx, nmax, a, b, L_shared, ld));
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    const int M = qmc->n_shifts;
    const int64_t Ns = qmc->n_points, Ntot = Ns * M;
    MVN_TRY(lattice_ensure(ctx, std::max(nmax, 1)));
    int64_t ntiles = 0;
    for (int p = 0; p < nprob; ++p)
        if (dims[p] > 0) ntiles += (Ntot + 127) / 128;
    const size_t need = ws_round(sizeof(uint64_t) * (size_t)M * std::max(nmax, 1)) +
                        ws_round(sizeof(double) * (size_t)Ntot * nprob) +
                        sov_any_ws_bytes(ctx, nprob, nmax, ntiles, prec) + 1024;
    MVN_TRY(ws_reserve(ctx, need));
    WsCarver wc(ctx->ws);
    uint64_t* delta = wc.take<uint64_t>((size_t)M * std::max(nmax, 1));
    double* logw = wc.take<double>((size_t)Ntot * nprob);
    std::vector<SovProblem> probs(nprob);
    for (int p = 0; p < nprob; ++p) {
        SovProblem& P = probs[p];
        P.n = dims[p];
        P.M = M;
        P.Ns = Ns;
        P.Ntot = Ntot;
        P.a = a + limit_offsets[p];
        P.b = b + limit_offsets[p];
        P.L = L_shared;
        P.ld = ld;
        P.delta = delta;  // the shifts of dimension i do not depend on the problem
        P.dstride = std::max(nmax, 1);
        P.logw = logw + (int64_t)p * Ntot;
        P.nprefix = 0;
        P.prefix = nullptr;
        P.logw_prefix = nullptr;
        if (P.n == 0) MVN_CUDA(ctx, cudaMemsetAsync(P.logw, 0, sizeof(double) * Ntot, ctx->stream));
    }
    MVN_TRY(lattice_shifts(ctx, qmc->seed, M, nmax, delta));
    MVN_TRY(sov_run_any(ctx, probs, prec, wc.base + ((wc.off + 255) & ~(size_t)255)));
    return sov_reduce_launch(ctx, logw, Ns, M, qmc->err_k, out3, nprob, Ntot);
}

// ---------------------------------------------------------------- ABI: mvn_sov_step_test
//
// The elementwise step of Eq. 2 exactly as the sweeps run it, on independent inputs (for parity
// of the tail branches, the underflow branch and the interior clamp, which the lattice reaches
// only rarely).  The lattice point comes from the 64-bit integer W as in the sweeps.
__global__ void k_sov_step_test(int prec, int64_t count, const double* __restrict__ a,
                                const double* __restrict__ b, const double* __restrict__ s,
                                const double* __restrict__ lii, const uint64_t* __restrict__ W,
                                double* __restrict__ y, double* __restrict__ delta) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= count) return;
    const double av = a[t], bv = b[t];
    if (prec == MVN_FP64) {
        double d;
        y[t] = sov_step_f64(av, bv, s[t], lii[t], lattice_w(1u, W[t], 0u), d);
        delta[t] = d;
    } else if (prec == MVN_MIXED_SIMT) {  // the CUDA-core mixed sweep's step
        double d;
        y[t] = (double)sov_step_f32(av, bv, (float)s[t], (float)lii[t], lattice_w(1u, W[t], 0u),
                                    d);
        delta[t] = d;
    } else {  // the tensor-core sweep's FP32-only step
        float w, wc, dh, dl;
        uint64_t m;
        int dex;
        lattice_wf(1u, W[t], 0u, w, wc, m);
        y[t] = (double)sov_step_f32p((float)av, (float)bv, av, bv, av == -INFINITY,
                                     bv == INFINITY, (float)s[t], (float)lii[t], w, wc, m, dh,
                                     dl, dex);
        delta[t] = ldexp((double)dh + (double)dl, dex);
    }
}

extern "C" mvn_status mvn_sov_step_test(mvn_ctx* ctx, mvn_prec prec, int64_t count,
                                        const double* a, const double* b, const double* s,
                                        const double* lii, const uint64_t* W, double* y,
                                        double* delta) {
    if (!ctx) return MVN_ERR_ARG;
    if (prec != MVN_FP64 && prec != MVN_MIXED && prec != MVN_MIXED_SIMT)
        return mvn_fail(ctx, MVN_ERR_ARG, "unknown precision");
    if (count < 0 || count > ((int64_t)1 << 31))
        return mvn_fail(ctx, MVN_ERR_ARG, "count out of range");
    if (count == 0) return MVN_OK;
    if (!a || !b || !s || !lii || !W || !y || !delta)
        return mvn_fail(ctx, MVN_ERR_ARG, "null pointer");
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    k_sov_step_test<<<(unsigned)((count + 255) / 256), 256, 0, ctx->stream>>>(
        (int)prec, count, a, b, s, lii, W, y, delta);
    MVN_LAUNCHED(ctx);
    return MVN_OK;
}

// ---------------------------------------------------------------- ABI: mvn_sov_fp64_noalloc
//
// FP64 SOV estimate for callers that cannot allocate device memory at call time: code that
// runs under a caching allocator that must not see foreign cudaMalloc calls, in a real-time
// loop where an allocation's implicit synchronisation is not allowed, or in an embedding that
// hands the library device buffers and nothing else.
// Such a caller cannot create an mvn_ctx (which owns a growing workspace), so this entry point
// takes a stream instead and keeps all of its scratch in one file-scope device array of fixed
// size, which every GPU that loads the library holds until the process exits.
//
// Limits: n <= 256 dimensions, n_points * n_shifts <= 262,144 paths, n_shifts <= 64.
// The sweep runs on a fixed persistent grid of 32 CTAs.
#define NA_NMAX 256
#define NA_PATHS_MAX 262144
#define NA_SHIFTS_MAX 64
#define NA_GRID 32
#define NA_PRIME_BOUND 4096  // > the 256th prime (1619)

struct NoAllocScratch {
    double Y[(size_t)NA_GRID * NA_NMAX * SOV_P];   // per-CTA transformed variables (8 MiB)
    double logw[NA_PATHS_MAX];                     // per-path log-weights (2 MiB)
    uint64_t delta[NA_SHIFTS_MAX * NA_NMAX];       // lattice shifts
    uint64_t alpha[NA_NMAX];                       // lattice generators
    int primes[NA_NMAX];
    uint8_t flags[NA_PRIME_BOUND];
    int counter;                                   // work-queue head (zeroed by every call)
    int status[MVN_STATUS_WORDS];                  // device status word of the kernels
};
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// lattice-table kernels defined in mvn_ctx.cu
__global__ void k_prime_flags(uint8_t* flag, int bound);
__global__ void k_prime_compact(const uint8_t* flag, int bound, int* primes, int count);
__global__ void k_alpha(const int* primes, int n, uint64_t* alpha);
__global__ void k_shifts(uint64_t seed, int M, int n, uint64_t* delta);

// Identity of the calling thread's current CUDA context (driver entry points reached through the
// runtime, so the library does not link the driver library itself).  Returns false if there is
// no current context or the entry points are unavailable.
typedef int (*PfnCtxGetCurrent)(void**);
typedef int (*PfnCtxGetId)(void*, unsigned long long*);
static bool current_context_id(unsigned long long* id) {
    static PfnCtxGetCurrent get_cur = nullptr;
    static PfnCtxGetId get_id = nullptr;
    static bool looked_up = false;
    if (!looked_up) {  // called with the caller's mutex held
        looked_up = true;
        void* f = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_cur = (PfnCtxGetCurrent)f;
        f = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = (PfnCtxGetId)f;
    }
    if (!get_cur || !get_id) return false;
    void* ctx = nullptr;
    if (get_cur(&ctx) != 0 || !ctx) return false;
    return get_id(ctx, id) == 0;
}

// Device address of the scratch array (the symbol name is only a host-side stand-in: passing it
// to a kernel would not give the device address).  Looked up once per device and context: a
// device reset (cudaDeviceReset) or a new primary context reloads the module, so a context whose
// identity differs from the cached one gets a fresh lookup.  Without the context identity (driver
// entry points unavailable) the address is looked up on every call.
static NoAllocScratch* noalloc_scratch_ptr(int device, cudaError_t* err) {
    struct Entry {
        NoAllocScratch* ptr;
        unsigned long long ctx;
    };
    static Entry cache[256] = {};
    static std::mutex mu;
    std::lock_guard<std::mutex> lock(mu);
    if (device < 0 || device >= 256) {
        *err = cudaErrorInvalidDevice;
        return nullptr;
    }
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    Entry& e = cache[device];
    if (!e.ptr || !have_id || e.ctx != id) {
        void* p = nullptr;
        *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (*err != cudaSuccess) return nullptr;
        e.ptr = (NoAllocScratch*)p;
        // the lookup makes the device's primary context current if it was not yet
        e.ctx = current_context_id(&id) ? id : 0;
    }
    *err = cudaSuccess;
    return e.ptr;
}

extern "C" mvn_status mvn_sov_fp64_noalloc(int n, const double* a, const double* b,
                                           const double* L, int64_t ld, const mvn_qmc* qmc,
                                           double* out3, double* path_logw, void* cuda_stream) {
    if (!qmc || !out3 || n < 0 || n > NA_NMAX || ld < (n > 0 ? n : 1) ||
        (n > 0 && (!a || !b || !L)) || qmc->n_points < 1 || qmc->n_shifts < 1 ||
        qmc->n_shifts > NA_SHIFTS_MAX ||
        (int64_t)qmc->n_points * qmc->n_shifts > NA_PATHS_MAX)
        return MVN_ERR_ARG;  // sizes beyond the fixed scratch are rejected before any work
    cudaStream_t st = (cudaStream_t)cuda_stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return MVN_ERR_CUDA;
    cudaError_t e;
    NoAllocScratch* S = noalloc_scratch_ptr(dev, &e);
    if (!S) return MVN_ERR_CUDA;
    const int M = qmc->n_shifts;
    const int64_t Ns = qmc->n_points, Ntot = Ns * M;
    double* logw = path_logw ? path_logw : S->logw;
    // the queue head and the status word must start at zero; the rest is written before read
    if (cudaMemsetAsync(&S->counter, 0, sizeof(int) * (1 + MVN_STATUS_WORDS), st) != cudaSuccess)
        return MVN_ERR_CUDA;
    const int nt = n > 0 ? n : 1;
    k_prime_flags<<<(NA_PRIME_BOUND + 255) / 256, 256, 0, st>>>(S->flags, NA_PRIME_BOUND);
    k_prime_compact<<<1, 1024, 0, st>>>(S->flags, NA_PRIME_BOUND, S->primes, nt);
    k_alpha<<<(nt + 127) / 128, 128, 0, st>>>(S->primes, nt, S->alpha);
    k_shifts<<<(M * nt + 255) / 256, 256, 0, st>>>(qmc->seed, M, nt, S->delta);
    if (n == 0) {
        if (cudaMemsetAsync(logw, 0, sizeof(double) * Ntot, st) != cudaSuccess) return MVN_ERR_CUDA;
    } else {
        SovBatch batch;
        memset(&batch, 0, sizeof(batch));
        SovProblem& P = batch.single;
        P.n = n;
        P.M = M;
        P.Ns = Ns;
        P.Ntot = Ntot;
        P.a = a;
        P.b = b;
        P.L = L;
        P.ld = ld;
        P.delta = S->delta;
        P.dstride = nt;
        P.logw = logw;
        batch.probs = nullptr;
        batch.nitems = (int)((Ntot + SOV_P - 1) / SOV_P);
        batch.counter = &S->counter;
        k_sov_simt<32, double, true><<<NA_GRID, SOV_P, 0, st>>>(batch, S->alpha, S->Y,
                                                                (int64_t)NA_NMAX * SOV_P);
    }
    k_sov_reduce<<<1, 512, sizeof(double) * (512 + M), st>>>(logw, Ns, M, qmc->err_k, out3, Ntot,
                                                             S->status, 0);
    return cudaGetLastError() == cudaSuccess ? MVN_OK : MVN_ERR_CUDA;
}
