// mvn_excursion.cu -- confidence-region (excursion set) detection, Alg. 1 with Eqs. 4-5:
// marginals p_M,i = P(X_i > u), their descending order, the Cholesky factor of the permuted
// covariance, and the loop of prefix problems (the PMVN calls of Alg. 1) as ONE sweep: with
// the shared lattice the k-prefix problem's per-path weight equals the running weight of the full
// sweep after k dimensions, so every F(o_k) is read off the same sweep.
#include <math.h>

#include <algorithm>
#include <vector>

#include "mvn_internal.cuh"
#include "mvn_sov.cuh"

mvn_status chol_f64_launch(mvn_ctx* ctx, int n, double* A, int64_t ld);
size_t chol_oz_ws_bytes(int n);
mvn_status chol_oz_launch(mvn_ctx* ctx, int n, double* A, int64_t ld, char* ws);
mvn_status sov_reduce_launch_opt(mvn_ctx* ctx, const double* logw, int64_t Ns, int M,
                                 double err_k, double* out3, int nprob, int64_t prob_stride,
                                 bool raise_numeric);

// marginal[i] = Q((u - mu_i) / sqrt(Sigma_ii));  key[i] = descending sort key, idx[i] = i.
__global__ void k_marginal(int n, int npad, const double* __restrict__ mu,
                           const double* __restrict__ S, int64_t ld, double u,
                           double* __restrict__ marginal, uint64_t* __restrict__ key,
                           int* __restrict__ idx) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npad) return;
    if (i < n) {
        double z = (u - mu[i]) / sqrt(S[i + (int64_t)i * ld]);
        double pm = 0.5 * erfc(z * 0.70710678118654752440);
        marginal[i] = pm;
        // pm >= 0: its bit pattern increases with pm; complement sorts descending
        key[i] = ~(uint64_t)__double_as_longlong(pm);
        idx[i] = i;
    } else {
        key[i] = ~0ull;
        idx[i] = 0x7fffffff;
    }
}

// one compare-exchange stage of a bitonic sort of (key, idx) pairs, ascending lexicographic
__global__ void k_bitonic(uint64_t* __restrict__ key, int* __restrict__ idx, int npad, int k,
                          int j) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= npad) return;
    int l = i ^ j;
    if (l <= i) return;
    bool up = (i & k) == 0;
    uint64_t ki = key[i], kl = key[l];
    int ii = idx[i], il = idx[l];
    bool gt = (ki > kl) || (ki == kl && ii > il);
    if (gt == up) {
        key[i] = kl;
        key[l] = ki;
        idx[i] = il;
        idx[l] = ii;
    }
}

// Sp(i, j) = Sigma(o_i, o_j) for i >= j (reads the lower triangle of Sigma); a_perm = u - mu[o]
__global__ void k_permute(int n, const int* __restrict__ order, const double* __restrict__ S,
                          int64_t ld, double* __restrict__ Sp, const double* __restrict__ mu,
                          double u, double* __restrict__ a_perm, double* __restrict__ b_perm) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = blockIdx.y;
    if (i >= n || i < j) return;
    const int oi = order[i], oj = order[j];
    const int r = max(oi, oj), c = min(oi, oj);
    Sp[i + (int64_t)j * n] = S[r + (int64_t)c * ld];
    if (j == 0) {
        a_perm[i] = u - mu[oi];
        b_perm[i] = INFINITY;
    }
}

// F[t] = out3[3 * map[t] + 1]; K = the largest listed k with F >= level; region[o_i] = (i < K)
__global__ void k_region(int n, int nprob, const int* __restrict__ ks_user,
                         const double* __restrict__ out3, const int* __restrict__ map,
                         double level, const int* __restrict__ order, double* __restrict__ F,
                         uint8_t* __restrict__ region) {
    __shared__ int Ks;
    if (threadIdx.x == 0) {
        int K = 0;
        for (int t = 0; t < nprob; ++t) {
            double f = out3[3 * map[t] + 1];
            F[t] = f;
            if (f >= level && ks_user[t] > K) K = ks_user[t];
        }
        Ks = K;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) region[order[i]] = (i < Ks) ? 1 : 0;
}

// ---------------------------------------------------------------- plan and device work

// Host-side plan of one confidence-region call: validated arguments, the sorted distinct
// prefix lengths ks (the sweep records the running weight after each), the map from the
// caller's prefix list to ks, and the workspace size.
struct ExcPlan {
    int n = 0, nprob = 0, nk = 0, nsweep = 0, npad = 1, M = 0;
    int64_t Ns = 0, Ntot = 0;
    std::vector<int> ks, map, ks_user;
    size_t ws_bytes = 0;  // device work (excluding the three index tables)
};

static mvn_status exc_plan(mvn_ctx* ctx, int n, const double* mu, const double* Sigma,
                           int64_t ld, int nprob, const int* prefix_dims, const mvn_qmc* qmc,
                           mvn_prec prec, const int32_t* order, const double* marginal,
                           const double* F, const uint8_t* region, ExcPlan& pl) {
    MVN_TRY(check_qmc(ctx, qmc));
    if (n < 1 || n > 65535 || ld < n || !mu || !Sigma || !order || !marginal || !F ||
        !region)
        return mvn_fail(ctx, MVN_ERR_ARG, "mvn_excursion: invalid argument");
    if (prec != MVN_FP64 && prec != MVN_MIXED && prec != MVN_MIXED_SIMT)
        return mvn_fail(ctx, MVN_ERR_ARG, "unknown precision");
    if (prefix_dims) {
        if (nprob < 1) return mvn_fail(ctx, MVN_ERR_ARG, "nprob < 1");
        pl.ks_user.assign(prefix_dims, prefix_dims + nprob);
    } else {
        nprob = n;
        pl.ks_user.resize(n);
        for (int k = 0; k < n; ++k) pl.ks_user[k] = k + 1;
    }
    for (int k : pl.ks_user)
        if (k < 1 || k > n) return mvn_fail(ctx, MVN_ERR_ARG, "prefix length out of 1..n");
    pl.ks = pl.ks_user;
    std::sort(pl.ks.begin(), pl.ks.end());
    pl.ks.erase(std::unique(pl.ks.begin(), pl.ks.end()), pl.ks.end());
    pl.map.resize(nprob);
    for (int t = 0; t < nprob; ++t)
        pl.map[t] = (int)(std::lower_bound(pl.ks.begin(), pl.ks.end(), pl.ks_user[t]) -
                          pl.ks.begin());
    pl.n = n;
    pl.nprob = nprob;
    pl.nk = (int)pl.ks.size();
    pl.nsweep = pl.ks.back();
    pl.M = qmc->n_shifts;
    pl.Ns = qmc->n_points;
    pl.Ntot = pl.Ns * pl.M;
    pl.npad = 1;
    while (pl.npad < n) pl.npad <<= 1;
    // the Cholesky workspace (MVN_MIXED) and the sweep's are used one after the other on the
    // stream, so they share one region
    size_t shared = sov_any_ws_bytes(ctx, 1, pl.nsweep, (pl.Ntot + 127) / 128, prec);
    if (prec == MVN_MIXED) shared = std::max(shared, chol_oz_ws_bytes(n));
    pl.ws_bytes = ws_round(sizeof(double) * (size_t)n * n) +       // Sp / L
                  ws_round(sizeof(uint64_t) * pl.npad) + ws_round(sizeof(int) * pl.npad) +
                  2 * ws_round(sizeof(double) * n) +                // a_perm, b_perm
                  ws_round(sizeof(uint64_t) * (size_t)pl.M * pl.nsweep) +  // shifts
                  ws_round(sizeof(double) * (size_t)pl.Ntot * pl.nk) +     // prefix weights
                  ws_round(sizeof(double) * 3 * pl.nk) +            // per-prefix estimates
                  ws_round(shared) + 1024;
    return MVN_OK;
}

// Enqueue the whole pipeline on ctx->stream.  d_ks (nk), d_map and d_ksu (nprob) are the plan's
// tables on the device; ws holds pl.ws_bytes.  The lattice table must already cover nsweep
// dimensions (lattice_ensure), so nothing here allocates or synchronises.
static mvn_status exc_enqueue(mvn_ctx* ctx, const ExcPlan& pl, const double* mu,
                              const double* Sigma, int64_t ld, double u, double one_minus_alpha,
                              const mvn_qmc* qmc, mvn_prec prec, const int* d_ks,
                              const int* d_map, const int* d_ksu, int32_t* order,
                              double* marginal, double* F, uint8_t* region, char* ws) {
    const int n = pl.n, npad = pl.npad, M = pl.M, nk = pl.nk, nsweep = pl.nsweep;
    const int64_t Ns = pl.Ns, Ntot = pl.Ntot;
    WsCarver wc(ws);
    double* Sp = wc.take<double>((size_t)n * n);
    uint64_t* key = wc.take<uint64_t>(npad);
    int* idx = wc.take<int>(npad);
    double* a_perm = wc.take<double>(n);
    double* b_perm = wc.take<double>(n);
    uint64_t* delta = wc.take<uint64_t>((size_t)M * nsweep);
    double* lwp = wc.take<double>((size_t)Ntot * nk);
    double* est = wc.take<double>(3 * (size_t)nk);
    char* shared_ws = wc.base + ((wc.off + 255) & ~(size_t)255);

    // marginals and order (Alg. 1)
    k_marginal<<<(npad + 255) / 256, 256, 0, ctx->stream>>>(n, npad, mu, Sigma, ld, u, marginal,
                                                            key, idx);
    MVN_LAUNCHED(ctx);
    for (int k = 2; k <= npad; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            k_bitonic<<<(npad + 255) / 256, 256, 0, ctx->stream>>>(key, idx, npad, k, j);
            MVN_LAUNCHED(ctx);
        }
    MVN_CUDA(ctx, cudaMemcpyAsync(order, idx, sizeof(int) * n, cudaMemcpyDeviceToDevice,
                                  ctx->stream));
    // permuted covariance, limits, Cholesky (Alg. 1)
    k_permute<<<dim3((n + 255) / 256, n), 256, 0, ctx->stream>>>(n, order, Sigma, ld, Sp, mu, u,
                                                                 a_perm, b_perm);
    MVN_LAUNCHED(ctx);
    if (prec == MVN_MIXED) {
        MVN_TRY(chol_oz_launch(ctx, n, Sp, n, shared_ws));
    } else {
        MVN_TRY(chol_f64_launch(ctx, n, Sp, n));
    }
    // one sweep with prefix recording (Alg. 1 loop of PMVN calls)
    MVN_TRY(lattice_shifts(ctx, qmc->seed, M, nsweep, delta));
    std::vector<SovProblem> probs(1);
    SovProblem& P = probs[0];
    P.n = nsweep;
    P.M = M;
    P.Ns = Ns;
    P.Ntot = Ntot;
    P.a = a_perm;
    P.b = b_perm;
    P.L = Sp;
    P.ld = n;
    P.delta = delta;
    P.dstride = nsweep;
    P.logw = nullptr;
    P.nprefix = nk;
    P.prefix = d_ks;
    P.logw_prefix = lwp;
    MVN_TRY(sov_run_any(ctx, probs, prec, shared_ws));
    MVN_TRY(sov_reduce_launch_opt(ctx, lwp, Ns, M, qmc->err_k, est, nk, Ntot, false));
    k_region<<<1, 256, 0, ctx->stream>>>(n, pl.nprob, d_ksu, est, d_map, one_minus_alpha, order,
                                         F, region);
    MVN_LAUNCHED(ctx);
    return MVN_OK;
}

extern "C" mvn_status mvn_excursion(mvn_ctx* ctx, int n, const double* mu, const double* Sigma,
                                    int64_t ld, double u, double one_minus_alpha, int nprob,
                                    const int* prefix_dims, const mvn_qmc* qmc, mvn_prec prec,
                                    int tile, int32_t* order, double* marginal, double* F,
                                    uint8_t* region) {
    if (!ctx) return MVN_ERR_ARG;
    if (tile < 0) return mvn_fail(ctx, MVN_ERR_ARG, "negative tile size");  // panel width is fixed at 64
    ExcPlan pl;
    MVN_TRY(exc_plan(ctx, n, mu, Sigma, ld, nprob, prefix_dims, qmc, prec, order, marginal, F,
                     region, pl));
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    MVN_TRY(lattice_ensure(ctx, pl.nsweep));
    const size_t tables = 3 * ws_round(sizeof(int) * pl.nprob);
    MVN_TRY(ws_reserve(ctx, ws_round(pl.ws_bytes) + tables));
    char* ws = (char*)ctx->ws;
    int* d_ks = (int*)(ws + ws_round(pl.ws_bytes));
    int* d_map = (int*)((char*)d_ks + ws_round(sizeof(int) * pl.nprob));
    int* d_ksu = (int*)((char*)d_map + ws_round(sizeof(int) * pl.nprob));
    MVN_CUDA(ctx, cudaMemcpyAsync(d_ks, pl.ks.data(), sizeof(int) * pl.nk,
                                  cudaMemcpyHostToDevice, ctx->stream));
    MVN_CUDA(ctx, cudaMemcpyAsync(d_map, pl.map.data(), sizeof(int) * pl.nprob,
                                  cudaMemcpyHostToDevice, ctx->stream));
    MVN_CUDA(ctx, cudaMemcpyAsync(d_ksu, pl.ks_user.data(), sizeof(int) * pl.nprob,
                                  cudaMemcpyHostToDevice, ctx->stream));
    return exc_enqueue(ctx, pl, mu, Sigma, ld, u, one_minus_alpha, qmc, prec, d_ks, d_map, d_ksu,
                       order, marginal, F, region, ws);
}

// ---------------------------------------------------------------- the pipeline as a CUDA graph

// The graph owns a private context (its own stream, workspace, lattice table, auxiliary streams
// and status word), so no later call on the caller's context can move or overwrite a buffer the
// captured kernels use, and the index tables in its own device memory.
struct mvn_graph {
    mvn_ctx* parent = nullptr;
    mvn_ctx* priv = nullptr;
    cudaStream_t cap = nullptr;
    int* d_tables = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t kernels = 0;
};

static void graph_free(mvn_graph* g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->d_tables) cudaFree(g->d_tables);
    if (g->priv) mvn_destroy(g->priv);
    if (g->cap) cudaStreamDestroy(g->cap);
    cudaGetLastError();
    delete g;
}

extern "C" mvn_status mvn_excursion_graph(mvn_ctx* ctx, int n, const double* mu,
                                          const double* Sigma, int64_t ld, double u,
                                          double one_minus_alpha, int nprob,
                                          const int* prefix_dims, const mvn_qmc* qmc,
                                          mvn_prec prec, int32_t* order, double* marginal,
                                          double* F, uint8_t* region, mvn_graph** out) {
    if (!ctx) return MVN_ERR_ARG;
    if (!out) return mvn_fail(ctx, MVN_ERR_ARG, "out is null");
    *out = nullptr;
    ExcPlan pl;
    MVN_TRY(exc_plan(ctx, n, mu, Sigma, ld, nprob, prefix_dims, qmc, prec, order, marginal, F,
                     region, pl));
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    // the caller's pending work on mu and Sigma comes first
    MVN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    mvn_graph* g = new mvn_graph();
    g->parent = ctx;
    mvn_status st = MVN_OK;
    auto fail = [&](mvn_status s, const char* what) {
        const char* why = (g->priv && !g->priv->err.empty()) ? g->priv->err.c_str() : "";
        mvn_fail(ctx, s, "mvn_excursion_graph: %s%s%s", what, *why ? ": " : "", why);
        cudaStreamCaptureStatus cs;
        if (g->cap && cudaStreamIsCapturing(g->cap, &cs) == cudaSuccess &&
            cs != cudaStreamCaptureStatusNone) {
            cudaGraph_t junk = nullptr;
            cudaStreamEndCapture(g->cap, &junk);
            if (junk) cudaGraphDestroy(junk);
        }
        graph_free(g);
        return s;
    };
    if (cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking) != cudaSuccess)
        return fail(MVN_ERR_CUDA, "stream creation failed");
    if ((st = mvn_create(&g->priv, ctx->device, g->cap)) != MVN_OK)
        return fail(st, "context creation failed");
    mvn_ctx* pv = g->priv;
    pv->tune = ctx->tune;  // the caller's autotuned launch shapes
    const size_t tb = ws_round(sizeof(int) * pl.nprob);
    if (cudaMalloc(&g->d_tables, 3 * tb) != cudaSuccess)
        return fail(MVN_ERR_OOM, "table allocation failed");
    int* d_ks = g->d_tables;
    int* d_map = (int*)((char*)g->d_tables + tb);
    int* d_ksu = (int*)((char*)g->d_tables + 2 * tb);
    if (cudaMemcpy(d_ks, pl.ks.data(), sizeof(int) * pl.nk, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(d_map, pl.map.data(), sizeof(int) * pl.nprob, cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(d_ksu, pl.ks_user.data(), sizeof(int) * pl.nprob, cudaMemcpyHostToDevice) !=
            cudaSuccess)
        return fail(MVN_ERR_CUDA, "table upload failed");
    // one eager run: sizes the workspace, builds the lattice table and the auxiliary streams,
    // and checks the problem (a non-positive pivot fails here, not in a replay)
    if ((st = lattice_ensure(pv, pl.nsweep)) != MVN_OK) return fail(st, "lattice table");
    if ((st = ws_reserve(pv, pl.ws_bytes)) != MVN_OK) return fail(st, "workspace");
    if ((st = exc_enqueue(pv, pl, mu, Sigma, ld, u, one_minus_alpha, qmc, prec, d_ks, d_map,
                          d_ksu, order, marginal, F, region, (char*)pv->ws)) != MVN_OK)
        return fail(st, "eager run");
    int info = 0;
    if ((st = mvn_sync(pv, &info)) != MVN_OK) return fail(st, "eager run");
    // capture the same work
    const int64_t l0 = pv->launches;
    if (cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeRelaxed) != cudaSuccess)
        return fail(MVN_ERR_CUDA, "capture begin failed");
    if ((st = exc_enqueue(pv, pl, mu, Sigma, ld, u, one_minus_alpha, qmc, prec, d_ks, d_map,
                          d_ksu, order, marginal, F, region, (char*)pv->ws)) != MVN_OK)
        return fail(st, "capture");
    if (cudaStreamEndCapture(g->cap, &g->graph) != cudaSuccess || !g->graph)
        return fail(MVN_ERR_CUDA, "capture end failed");
    if (cudaGraphInstantiate(&g->exec, g->graph, 0) != cudaSuccess)
        return fail(MVN_ERR_CUDA, "graph instantiation failed");
    g->kernels = pv->launches - l0;
    *out = g;
    return MVN_OK;
}

extern "C" mvn_status mvn_graph_launch(mvn_graph* g) {
    if (!g || !g->exec) return MVN_ERR_ARG;
    mvn_ctx* ctx = g->parent;
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    MVN_CUDA(ctx, cudaGraphLaunch(g->exec, ctx->stream));
    ctx->launches += g->kernels;
    return MVN_OK;
}

extern "C" mvn_status mvn_graph_sync(mvn_graph* g, int* info) {
    if (!g) return MVN_ERR_ARG;
    mvn_ctx* ctx = g->parent;
    MVN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    const mvn_status st = mvn_sync(g->priv, info);
    if (st != MVN_OK) mvn_fail(ctx, st, "%s", g->priv->err.c_str());
    return st;
}

extern "C" int64_t mvn_graph_kernels(const mvn_graph* g) { return g ? g->kernels : 0; }

extern "C" mvn_status mvn_graph_destroy(mvn_graph* g) {
    if (!g) return MVN_OK;
    cudaSetDevice(g->parent->device);
    cudaStreamSynchronize(g->parent->stream);
    graph_free(g);
    return MVN_OK;
}
