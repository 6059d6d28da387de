// mvn_tune.cu -- autotuner of launch shapes (not in the paper: the paper's tile size is a user
// parameter of its CPU runtime).  It times candidate shapes of the MVN_MIXED Cholesky (split-K
// work-item sizes of the bulk and tail updates) and of the sweeps (persistent grid, CTAs per SM)
// on a synthetic problem of the requested size on this device, keeps the fastest in the context
// and optionally in a cache file of JSON lines keyed by (device name, SM count, precision, size
// buckets).  No choice changes a result: the Cholesky update sums exact integers in any order
// and the sweeps compute each path independently of the grid.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "mvn_internal.cuh"

static int log2_bucket(int64_t x) {
    int b = 0;
    while (b < 62 && ((int64_t)1 << b) < x) ++b;
    return b;
}

static std::tuple<int, int, int> chol_key(int n) { return {100 + MVN_MIXED, log2_bucket(n), 0}; }
static std::tuple<int, int, int> sweep_key(mvn_prec prec, int n, int64_t ntiles) {
    return {(int)prec, log2_bucket(n), log2_bucket(ntiles)};
}

TuneParams tune_chol(const mvn_ctx* ctx, int n) {
    auto it = ctx->tune.find(chol_key(n));
    return it == ctx->tune.end() ? TuneParams() : it->second;
}

TuneParams tune_sweep(const mvn_ctx* ctx, mvn_prec prec, int n, int64_t ntiles) {
    auto it = ctx->tune.find(sweep_key(prec, n, ntiles));
    return it == ctx->tune.end() ? TuneParams() : it->second;
}

// ---------------------------------------------------------------- cache file (JSON lines)

static std::string device_name(int device) {
    cudaDeviceProp p;
    if (cudaGetDeviceProperties(&p, device) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::string s(p.name);
    for (auto& c : s)
        if (c == '"' || c == '\\') c = '_';
    return s;
}

static bool read_int(const char* line, const char* key, int* v) {
    char pat[64];
    snprintf(pat, sizeof(pat), "\"%s\": ", key);
    const char* p = strstr(line, pat);
    return p && sscanf(p + strlen(pat), "%d", v) == 1;
}

// Entry for (device, sms, prec, nb, tb) in `path`, the last one if several; false if none.
static bool cache_lookup(const char* path, const std::string& dev, int sms, int prec, int nb,
                         int tb, mvn_tune_result* r) {
    FILE* f = fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    std::string want = "\"device\": \"" + dev + "\"";
    while (fgets(line, sizeof(line), f)) {
        int s = 0, pr = 0, n = 0, t = 0;
        if (!strstr(line, want.c_str()) || !read_int(line, "sms", &s) ||
            !read_int(line, "prec", &pr) || !read_int(line, "n_log2", &n) ||
            !read_int(line, "tiles_log2", &t))
            continue;
        if (s != sms || pr != prec || n != nb || t != tb) continue;
        mvn_tune_result e = {};
        if (read_int(line, "chol_bulk_p", &e.chol_bulk_p) &&
            read_int(line, "chol_tail_p", &e.chol_tail_p) &&
            read_int(line, "sweep_ctas_per_sm", &e.sweep_ctas_per_sm) &&
            e.chol_bulk_p >= 1 && e.chol_bulk_p <= 4096 && e.chol_tail_p >= 1 &&
            e.chol_tail_p <= 2 && e.sweep_ctas_per_sm >= 1 && e.sweep_ctas_per_sm <= 4) {
            *r = e;
            found = true;
        }
    }
    fclose(f);
    return found;
}

static void cache_append(const char* path, const std::string& dev, int sms, int prec, int nb,
                         int tb, const mvn_tune_result& r, double ms_chol, double ms_sweep) {
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f,
            "{\"device\": \"%s\", \"sms\": %d, \"prec\": %d, \"n_log2\": %d, \"tiles_log2\": %d, "
            "\"chol_bulk_p\": %d, \"chol_tail_p\": %d, \"sweep_ctas_per_sm\": %d, "
            "\"chol_ms\": %.4f, \"sweep_ms\": %.4f}\n",
            dev.c_str(), sms, prec, nb, tb, r.chol_bulk_p, r.chol_tail_p, r.sweep_ctas_per_sm,
            ms_chol, ms_sweep);
    fclose(f);
}

static void set_entries(mvn_ctx* ctx, mvn_prec prec, int n, int64_t ntiles,
                        const mvn_tune_result& r) {
    TuneParams c;
    c.chol_bulk_p = r.chol_bulk_p;
    c.chol_tail_p = r.chol_tail_p;
    ctx->tune[chol_key(n)] = c;
    TuneParams s;
    s.tc_ctas_per_sm = (prec == MVN_MIXED) ? r.sweep_ctas_per_sm : TuneParams().tc_ctas_per_sm;
    s.simt_ctas_per_sm = (prec == MVN_MIXED) ? TuneParams().simt_ctas_per_sm : r.sweep_ctas_per_sm;
    ctx->tune[sweep_key(prec, n, ntiles)] = s;
}

// ---------------------------------------------------------------- timing

struct TuneBuffers {
    double *coords = nullptr, *S0 = nullptr, *A = nullptr, *a = nullptr, *b = nullptr,
           *out3 = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~TuneBuffers() {
        for (double* p : {coords, S0, A, a, b, out3})
            if (p) cudaFree(p);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaGetLastError();
    }
};

// Median of `reps` timed runs of fn (after one untimed run), in ms.
template <class F>
static mvn_status time_ms(mvn_ctx* ctx, TuneBuffers& tb, int reps, F fn, double* ms) {
    MVN_TRY(fn());
    MVN_TRY(mvn_sync(ctx, nullptr));
    std::vector<double> t;
    for (int r = 0; r < reps; ++r) {
        MVN_CUDA(ctx, cudaEventRecord(tb.e0, ctx->stream));
        MVN_TRY(fn());
        MVN_CUDA(ctx, cudaEventRecord(tb.e1, ctx->stream));
        MVN_TRY(mvn_sync(ctx, nullptr));
        float f = 0.f;
        MVN_CUDA(ctx, cudaEventElapsedTime(&f, tb.e0, tb.e1));
        t.push_back(f);
    }
    std::sort(t.begin(), t.end());
    *ms = t[t.size() / 2];
    return MVN_OK;
}

extern "C" mvn_status mvn_autotune(mvn_ctx* ctx, int n, int64_t n_paths, mvn_prec prec,
                                   const char* cache_path, mvn_tune_result* out) {
    if (!ctx) return MVN_ERR_ARG;
    if (!out || n < 1 || n > 65536 || n_paths < 1 || n_paths > ((int64_t)1 << 32))
        return mvn_fail(ctx, MVN_ERR_ARG, "mvn_autotune: invalid argument");
    if (prec != MVN_FP64 && prec != MVN_MIXED && prec != MVN_MIXED_SIMT)
        return mvn_fail(ctx, MVN_ERR_ARG, "unknown precision");
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    const int64_t ntiles = (n_paths + 127) / 128;
    const std::string dev = device_name(ctx->device);
    const int nb = log2_bucket(n), tbk = log2_bucket(ntiles);
    mvn_tune_result r = {};
    if (cache_path && cache_lookup(cache_path, dev, ctx->sm_count, (int)prec, nb, tbk, &r)) {
        r.from_cache = 1;
        set_entries(ctx, prec, n, ntiles, r);
        *out = r;
        return MVN_OK;
    }
    // synthetic problem of this size: exponential covariance (range 0.1, nugget 1e-4) on the
    // first n points of a regular grid of [0,1]^2, limits a = -inf, b = 0.5
    TuneBuffers tb;
    const int g = (int)ceil(sqrt((double)n));
    std::vector<double> c(2 * (size_t)n), hb(n, 0.5), ha(n, -INFINITY);
    for (int i = 0; i < n; ++i) {
        c[2 * i] = (g > 1) ? (double)(i / g) / (g - 1) : 0.0;
        c[2 * i + 1] = (g > 1) ? (double)(i % g) / (g - 1) : 0.0;
    }
    const size_t nn = (size_t)n * n;
    MVN_CUDA(ctx, cudaMalloc(&tb.coords, sizeof(double) * 2 * n));
    MVN_CUDA(ctx, cudaMalloc(&tb.S0, sizeof(double) * nn));
    MVN_CUDA(ctx, cudaMalloc(&tb.A, sizeof(double) * nn));
    MVN_CUDA(ctx, cudaMalloc(&tb.a, sizeof(double) * n));
    MVN_CUDA(ctx, cudaMalloc(&tb.b, sizeof(double) * n));
    MVN_CUDA(ctx, cudaMalloc(&tb.out3, sizeof(double) * 3));
    MVN_CUDA(ctx, cudaEventCreate(&tb.e0));
    MVN_CUDA(ctx, cudaEventCreate(&tb.e1));
    MVN_CUDA(ctx, cudaMemcpy(tb.coords, c.data(), sizeof(double) * 2 * n, cudaMemcpyHostToDevice));
    MVN_CUDA(ctx, cudaMemcpy(tb.a, ha.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    MVN_CUDA(ctx, cudaMemcpy(tb.b, hb.data(), sizeof(double) * n, cudaMemcpyHostToDevice));
    MVN_TRY(mvn_matern(ctx, n, tb.coords, 1.0, 0.1, 0.5, 1e-4, tb.S0, n));

    // Cholesky shapes (MVN_MIXED only: the FP64 factorisation has none to tune)
    r.chol_bulk_p = TuneParams().chol_bulk_p;
    r.chol_tail_p = TuneParams().chol_tail_p;
    double best_chol = 0.0;
    const mvn_prec cprec = (prec == MVN_MIXED) ? MVN_MIXED : MVN_FP64;
    auto chol = [&]() -> mvn_status {
        MVN_CUDA(ctx, cudaMemcpyAsync(tb.A, tb.S0, sizeof(double) * nn, cudaMemcpyDeviceToDevice,
                                      ctx->stream));
        return mvn_cholesky(ctx, n, tb.A, n, 0, cprec, nullptr);
    };
    if (prec == MVN_MIXED) {
        best_chol = 1e30;
        for (int tail : {1, 2})
            for (int bulk : {4, 8, 16, 32, 64}) {
                mvn_tune_result cand = r;
                cand.chol_bulk_p = bulk;
                cand.chol_tail_p = tail;
                cand.sweep_ctas_per_sm = TuneParams().tc_ctas_per_sm;
                set_entries(ctx, prec, n, ntiles, cand);
                double ms = 0.0;
                MVN_TRY(time_ms(ctx, tb, 2, chol, &ms));
                if (ms < best_chol) {
                    best_chol = ms;
                    r.chol_bulk_p = bulk;
                    r.chol_tail_p = tail;
                }
            }
    }
    // the factor the sweep candidates use (its values do not affect the timing ranking much)
    {
        mvn_tune_result cand = r;
        cand.sweep_ctas_per_sm = 2;
        set_entries(ctx, prec, n, ntiles, cand);
        MVN_TRY(chol());
        MVN_TRY(mvn_sync(ctx, nullptr));
    }
    // sweep grid: the same number of path tiles, on at most 2,048 dimensions (each tile's time
    // grows with n^2, the ranking of the grids comes from how the tiles fill the SMs)
    const int nsw = std::min(n, 2048);
    mvn_qmc q;
    memset(&q, 0, sizeof(q));
    q.n_shifts = (int32_t)std::min<int64_t>(10, n_paths);
    q.n_points = (n_paths + q.n_shifts - 1) / q.n_shifts;
    q.seed = 1;
    q.err_k = 3.0;
    double best_sweep = 1e30;
    const int max_ctas = (prec == MVN_MIXED) ? 2 : 3;
    for (int ctas = 1; ctas <= max_ctas; ++ctas) {
        mvn_tune_result cand = r;
        cand.sweep_ctas_per_sm = ctas;
        set_entries(ctx, prec, nsw, ntiles, cand);
        double ms = 0.0;
        MVN_TRY(time_ms(ctx, tb, 2, [&]() -> mvn_status {
            return mvn_sov(ctx, nsw, tb.a, tb.b, tb.A, n, &q, prec, tb.out3, nullptr);
        }, &ms));
        if (ms < best_sweep) {
            best_sweep = ms;
            r.sweep_ctas_per_sm = ctas;
        }
    }
    if (nsw != n) ctx->tune.erase(sweep_key(prec, nsw, ntiles));
    r.from_cache = 0;
    set_entries(ctx, prec, n, ntiles, r);
    if (cache_path) cache_append(cache_path, dev, ctx->sm_count, (int)prec, nb, tbk, r, best_chol,
                                 best_sweep);
    *out = r;
    return MVN_OK;
}

extern "C" mvn_status mvn_tune_set(mvn_ctx* ctx, int n, int64_t n_paths, mvn_prec prec,
                                   const mvn_tune_result* params) {
    if (!ctx) return MVN_ERR_ARG;
    if (!params || n < 1 || n_paths < 1 || params->chol_bulk_p < 1 ||
        params->chol_bulk_p > 4096 || params->chol_tail_p < 1 || params->chol_tail_p > 2 ||
        params->sweep_ctas_per_sm < 1 || params->sweep_ctas_per_sm > (prec == MVN_MIXED ? 2 : 3))
        return mvn_fail(ctx, MVN_ERR_ARG, "mvn_tune_set: invalid argument");
    if (prec != MVN_FP64 && prec != MVN_MIXED && prec != MVN_MIXED_SIMT)
        return mvn_fail(ctx, MVN_ERR_ARG, "unknown precision");
    set_entries(ctx, prec, n, (n_paths + 127) / 128, *params);
    return MVN_OK;
}
