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

extern "C" mvn_status mvn_excursion(mvn_ctx* ctx, int n, const double* mu, const double* Sigma,
                                    int64_t ld, double u, double one_minus_alpha, int nprob,
                                    const int* prefix_dims, const mvn_qmc* qmc, mvn_prec prec,
                                    int tile, int32_t* order, double* marginal, double* F,
                                    uint8_t* region) {
    if (!ctx) return MVN_ERR_ARG;
    (void)tile;
    MVN_TRY(check_qmc(ctx, qmc));
    if (n < 1 || n > 65535 || ld < n || !mu || !Sigma || !order || !marginal || !F ||
        !region)
        return mvn_fail(ctx, MVN_ERR_ARG, "mvn_excursion: invalid argument");
    if (prec != MVN_FP64 && prec != MVN_MIXED && prec != MVN_MIXED_SIMT)
        return mvn_fail(ctx, MVN_ERR_ARG, "unknown precision");
    std::vector<int> ks_user;
    if (prefix_dims) {
        if (nprob < 1) return mvn_fail(ctx, MVN_ERR_ARG, "nprob < 1");
        ks_user.assign(prefix_dims, prefix_dims + nprob);
    } else {
        nprob = n;
        ks_user.resize(n);
        for (int k = 0; k < n; ++k) ks_user[k] = k + 1;
    }
    for (int k : ks_user)
        if (k < 1 || k > n) return mvn_fail(ctx, MVN_ERR_ARG, "prefix length out of 1..n");
    std::vector<int> ks(ks_user);
    std::sort(ks.begin(), ks.end());
    ks.erase(std::unique(ks.begin(), ks.end()), ks.end());
    std::vector<int> map(nprob);
    for (int t = 0; t < nprob; ++t)
        map[t] = (int)(std::lower_bound(ks.begin(), ks.end(), ks_user[t]) - ks.begin());
    const int nk = (int)ks.size();
    const int nsweep = ks.back();

    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    const int M = qmc->n_shifts;
    const int64_t Ns = qmc->n_points, Ntot = Ns * M;
    MVN_TRY(lattice_ensure(ctx, nsweep));
    int npad = 1;
    while (npad < n) npad <<= 1;
    const size_t need = ws_round(sizeof(double) * (size_t)n * n) +      // Sp / L
                        ws_round(sizeof(uint64_t) * npad) + ws_round(sizeof(int) * npad) +
                        2 * ws_round(sizeof(double) * n) +               // a_perm, b_perm
                        ws_round(sizeof(uint64_t) * (size_t)M * nsweep) +  // shifts
                        ws_round(sizeof(double) * (size_t)Ntot * nk) +   // prefix weights
                        ws_round(sizeof(double) * 3 * nk) +             // per-prefix estimates
                        3 * ws_round(sizeof(int) * nprob) +
                        sov_any_ws_bytes(ctx, 1, nsweep, (Ntot + 127) / 128, prec) + 4096;
    MVN_TRY(ws_reserve(ctx, need));
    WsCarver wc(ctx->ws);
    double* Sp = wc.take<double>((size_t)n * n);
    uint64_t* key = wc.take<uint64_t>(npad);
    int* idx = wc.take<int>(npad);
    double* a_perm = wc.take<double>(n);
    double* b_perm = wc.take<double>(n);
    uint64_t* delta = wc.take<uint64_t>((size_t)M * nsweep);
    double* lwp = wc.take<double>((size_t)Ntot * nk);
    double* est = wc.take<double>(3 * (size_t)nk);
    int* d_ks = wc.take<int>(nprob);
    int* d_map = wc.take<int>(nprob);
    int* d_ksu = wc.take<int>(nprob);
    char* sov_ws = wc.base + ((wc.off + 255) & ~(size_t)255);

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
    MVN_TRY(chol_f64_launch(ctx, n, Sp, n));
    // one sweep with prefix recording (Alg. 1 loop of PMVN calls)
    MVN_CUDA(ctx, cudaMemcpyAsync(d_ks, ks.data(), sizeof(int) * nk, cudaMemcpyHostToDevice,
                                  ctx->stream));
    MVN_CUDA(ctx, cudaMemcpyAsync(d_map, map.data(), sizeof(int) * nprob, cudaMemcpyHostToDevice,
                                  ctx->stream));
    MVN_CUDA(ctx, cudaMemcpyAsync(d_ksu, ks_user.data(), sizeof(int) * nprob,
                                  cudaMemcpyHostToDevice, ctx->stream));
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
    MVN_TRY(sov_run_any(ctx, probs, prec, sov_ws));
    MVN_TRY(sov_reduce_launch_opt(ctx, lwp, Ns, M, qmc->err_k, est, nk, Ntot, false));
    k_region<<<1, 256, 0, ctx->stream>>>(n, nprob, d_ksu, est, d_map, one_minus_alpha, order, F,
                                         region);
    MVN_LAUNCHED(ctx);
    return MVN_OK;
}
