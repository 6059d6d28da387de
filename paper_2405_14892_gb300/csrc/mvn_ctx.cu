// mvn_ctx.cu -- context, workspace, device status word and lattice tables.
#include <math.h>
#include <stdarg.h>
#include <string.h>

#include "mvn_internal.cuh"

mvn_status mvn_fail(mvn_ctx* ctx, mvn_status st, const char* fmt, ...) {
    if (ctx) {
        char buf[1024];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return st;
}

extern "C" mvn_status mvn_create(mvn_ctx** out, int device, void* cuda_stream) {
    if (!out) return MVN_ERR_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return MVN_ERR_CUDA;
    }
    mvn_ctx* ctx = new mvn_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    if (cudaSetDevice(device) != cudaSuccess ||
        cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device) !=
            cudaSuccess ||
        cudaMalloc(&ctx->d_status, sizeof(int) * MVN_STATUS_WORDS) != cudaSuccess ||
        cudaMemset(ctx->d_status, 0, sizeof(int) * MVN_STATUS_WORDS) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->d_status) cudaFree(ctx->d_status);
        delete ctx;
        return MVN_ERR_CUDA;
    }
    *out = ctx;
    return MVN_OK;
}

cudaEvent_t timing_event(mvn_ctx* ctx) { return timing_event_on(ctx, ctx->stream); }

cudaEvent_t timing_event_on(mvn_ctx* ctx, cudaStream_t stream) {
    if (!ctx->timing) return nullptr;
    if (ctx->ev_used == ctx->ev_pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        ctx->ev_pool.push_back(e);
    }
    cudaEvent_t e = ctx->ev_pool[ctx->ev_used++];
    cudaEventRecord(e, stream);
    return e;
}

mvn_status ctx_aux(mvn_ctx* ctx) {
    if (ctx->aux[0]) return MVN_OK;
    int least = 0, greatest = 0;
    MVN_CUDA(ctx, cudaDeviceGetStreamPriorityRange(&least, &greatest));
    MVN_CUDA(ctx, cudaStreamCreateWithPriority(&ctx->aux[0], cudaStreamNonBlocking, greatest));
    MVN_CUDA(ctx, cudaStreamCreateWithPriority(&ctx->aux[1], cudaStreamNonBlocking, least));
    for (auto& e : ctx->aux_ev) MVN_CUDA(ctx, cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    return MVN_OK;
}

void timing_record(mvn_ctx* ctx, const char* name, cudaEvent_t a, cudaEvent_t b) {
    if (ctx->timing && a && b) ctx->ktimes[name].push_back({a, b});
}

extern "C" mvn_status mvn_timing(mvn_ctx* ctx, int enable) {
    if (!ctx) return MVN_ERR_ARG;
    MVN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->timing = enable != 0;
    ctx->ktimes.clear();
    ctx->ev_used = 0;
    return MVN_OK;
}

extern "C" mvn_status mvn_kernel_time(mvn_ctx* ctx, const char* name, double* total_ms,
                                      int64_t* launches) {
    if (!ctx || !name || !total_ms || !launches) return MVN_ERR_ARG;
    MVN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    *total_ms = 0.0;
    *launches = 0;
    auto it = ctx->ktimes.find(name);
    if (it == ctx->ktimes.end()) return MVN_OK;
    for (auto& pr : it->second) {
        float ms = 0.0f;
        MVN_CUDA(ctx, cudaEventElapsedTime(&ms, pr.first, pr.second));
        *total_ms += ms;
    }
    *launches = (int64_t)it->second.size();
    return MVN_OK;
}

extern "C" mvn_status mvn_destroy(mvn_ctx* ctx) {
    if (!ctx) return MVN_ERR_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto e : ctx->ev_pool) cudaEventDestroy(e);
    for (auto e : ctx->aux_ev)
        if (e) cudaEventDestroy(e);
    for (auto s : ctx->aux)
        if (s) cudaStreamDestroy(s);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->d_alpha) cudaFree(ctx->d_alpha);
    if (ctx->d_status) cudaFree(ctx->d_status);
    delete ctx;
    return MVN_OK;
}

extern "C" mvn_status mvn_set_stream(mvn_ctx* ctx, void* cuda_stream) {
    if (!ctx) return MVN_ERR_ARG;
    ctx->stream = (cudaStream_t)cuda_stream;
    return MVN_OK;
}

extern "C" const char* mvn_last_error(const mvn_ctx* ctx) {
    return ctx ? ctx->err.c_str() : "null context";
}

extern "C" int64_t mvn_launch_count(const mvn_ctx* ctx) { return ctx ? ctx->launches : -1; }

extern "C" mvn_status mvn_sync(mvn_ctx* ctx, int* info) {
    if (!ctx) return MVN_ERR_ARG;
    if (info) *info = 0;
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    MVN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    int h[MVN_STATUS_WORDS];
    MVN_CUDA(ctx, cudaMemcpy(h, ctx->d_status, sizeof(h), cudaMemcpyDeviceToHost));
    if (h[0] != 0) {
        MVN_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(int) * 2));
        if (info) *info = h[1];
        const char* what = h[0] == MVN_ERR_NOT_PD    ? "matrix not positive definite"
                           : h[0] == MVN_ERR_NUMERIC ? "every path has weight 0"
                           : h[0] == MVN_ERR_TIMEOUT ? "device wait timed out"
                                                     : "device error";
        return mvn_fail(ctx, (mvn_status)h[0], "%s (info %d)", what, h[1]);
    }
    return MVN_OK;
}

mvn_status ws_reserve(mvn_ctx* ctx, size_t bytes) {
    bytes = ws_round(bytes);
    if (bytes <= ctx->ws_size) return MVN_OK;
    // growing: wait for work that may still use the old arena, then replace it
    MVN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->ws) cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_size = 0;
    size_t want = (bytes + (2u << 20) - 1) & ~(size_t)((2u << 20) - 1);
    const char* fail = getenv("MVN_FAULT_WS_ALLOC");  // host-side fault injection for tests
    if (fail && atoi(fail) != 0) return mvn_fail(ctx, MVN_ERR_OOM, "workspace allocation failed (injected)");
    if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
        cudaGetLastError();
        ctx->ws = nullptr;
        return mvn_fail(ctx, MVN_ERR_OOM, "workspace allocation of %zu bytes failed", want);
    }
    ctx->ws_size = want;
    return MVN_OK;
}

// ---------------------------------------------------------------- lattice generators

// flag[x] = 1 if x is prime (trial division by 2 and odd d <= sqrt(x))
__global__ void k_prime_flags(uint8_t* flag, int bound) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= bound) return;
    uint8_t f = x >= 2;
    if (x > 3) {
        if ((x & 1) == 0) f = 0;
        for (int d = 3; f && d * d <= x; d += 2)
            if (x % d == 0) f = 0;
    }
    flag[x] = f;
}

// Ordered compaction of the prime flags (one block of 1024 threads): primes[k] = k-th prime.
__global__ void k_prime_compact(const uint8_t* flag, int bound, int* primes, int count) {
    __shared__ int warp_tot[32];
    __shared__ int base_s;
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    if (t == 0) base_s = 0;
    __syncthreads();
    for (int c0 = 0; c0 < bound; c0 += 1024) {
        int base = base_s;
        if (base >= count) break;
        int x = c0 + t;
        int f = (x < bound) ? flag[x] : 0;
        unsigned m = __ballot_sync(0xffffffffu, f);
        int pre = __popc(m & ((1u << lane) - 1u));
        if (lane == 0) warp_tot[w] = __popc(m);
        __syncthreads();
        int off = 0, tot = 0;
        for (int k = 0; k < 32; ++k) {
            if (k < w) off += warp_tot[k];
            tot += warp_tot[k];
        }
        int idx = base + off + pre;
        if (f && idx < count) primes[idx] = x;
        __syncthreads();
        if (t == 0) base_s = base + tot;
        __syncthreads();
    }
}

// alpha_i = floor(sqrt(p_i) * 2^64) mod 2^64, exactly: with s = floor(sqrt(p)), the answer is
// the largest F < 2^64 with (s 2^64 + F)^2 <= p 2^128, found bit by bit in 192-bit arithmetic.
__global__ void k_alpha(const int* primes, int n, uint64_t* alpha) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t p = (uint64_t)primes[i];
    uint64_t s = (uint64_t)sqrt((double)p);
    while (s * s > p) --s;
    while ((s + 1) * (s + 1) <= p) ++s;
    uint64_t F = 0;
    for (int bit = 63; bit >= 0; --bit) {
        uint64_t c = F | (1ull << bit);
        // X = s*2^64 + c;  X^2 = s^2 2^128 + 2 s c 2^64 + c^2
        uint64_t q0 = c * c, q1 = __umul64hi(c, c);
        uint64_t r0 = c * (2 * s), r1 = __umul64hi(c, 2 * s);
        uint64_t t0 = r0 + q1;
        uint64_t t1 = (t0 < r0) ? 1u : 0u;
        uint64_t hi = s * s + r1 + t1;
        bool le = (hi < p) || (hi == p && t0 == 0 && q0 == 0);
        if (le) F = c;
    }
    alpha[i] = F;
}

mvn_status lattice_ensure(mvn_ctx* ctx, int n) {
    if (n <= ctx->n_alpha) return MVN_OK;
    int want = n < 1024 ? 1024 : n;
    double ln = log((double)want);
    int bound = (int)(want * (ln + log(ln)) + 64);
    uint8_t* flag = nullptr;
    int* primes = nullptr;
    uint64_t* alpha = nullptr;
    MVN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    MVN_CUDA(ctx, cudaMalloc(&flag, bound));
    MVN_CUDA(ctx, cudaMalloc(&primes, sizeof(int) * want));
    MVN_CUDA(ctx, cudaMalloc(&alpha, sizeof(uint64_t) * want));
    k_prime_flags<<<(bound + 255) / 256, 256, 0, ctx->stream>>>(flag, bound);
    MVN_LAUNCHED(ctx);
    k_prime_compact<<<1, 1024, 0, ctx->stream>>>(flag, bound, primes, want);
    MVN_LAUNCHED(ctx);
    k_alpha<<<(want + 127) / 128, 128, 0, ctx->stream>>>(primes, want, alpha);
    MVN_LAUNCHED(ctx);
    MVN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(flag);
    cudaFree(primes);
    if (ctx->d_alpha) cudaFree(ctx->d_alpha);
    ctx->d_alpha = alpha;
    ctx->n_alpha = want;
    return MVN_OK;
}

__global__ void k_shifts(uint64_t seed, int M, int n, uint64_t* delta) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)M * n) return;
    int q = (int)(t / n), i = (int)(t - (int64_t)q * n);
    delta[t] = splitmix64_at(seed, ((uint64_t)q << 32) | (uint64_t)i);
}

mvn_status lattice_shifts(mvn_ctx* ctx, uint64_t seed, int M, int n, uint64_t* delta) {
    int64_t tot = (int64_t)M * n;
    if (tot == 0) return MVN_OK;
    k_shifts<<<(unsigned)((tot + 255) / 256), 256, 0, ctx->stream>>>(seed, M, n, delta);
    MVN_LAUNCHED(ctx);
    return MVN_OK;
}

// Test hook: copy the first n lattice generators to a device buffer.
extern "C" mvn_status mvn_lattice_alpha(mvn_ctx* ctx, int n, uint64_t* out) {
    if (!ctx || n < 0 || (n > 0 && !out)) return MVN_ERR_ARG;
    if (n == 0) return MVN_OK;
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    MVN_TRY(lattice_ensure(ctx, n));
    MVN_CUDA(ctx, cudaMemcpyAsync(out, ctx->d_alpha, sizeof(uint64_t) * n,
                                  cudaMemcpyDeviceToDevice, ctx->stream));
    return MVN_OK;
}

extern "C" mvn_status mvn_lattice_shifts(mvn_ctx* ctx, uint64_t seed, int M, int n,
                                         uint64_t* out) {
    if (!ctx || n < 0 || M < 0 || ((int64_t)n * M > 0 && !out)) return MVN_ERR_ARG;
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    return lattice_shifts(ctx, seed, M, n, out);
}
