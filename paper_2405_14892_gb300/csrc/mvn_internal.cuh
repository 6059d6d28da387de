// mvn_internal.cuh -- internal declarations of the GB300 MVN library (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <map>
#include <tuple>
#include <string>
#include <vector>

#include "../../include/mvn.h"

// Device status word layout (ctx->d_status):
//   [0] first error code (mvn_status) raised on the device, 0 if none
//   [1] LAPACK-style info of the last failed factorisation (1-based column)
//   [2] scratch counter used by persistent kernels
#define MVN_STATUS_WORDS 8
// default limit of the adjoint's y and ybar buffers (8 GiB)
#define MVN_GRAD_Y_LIMIT_DEFAULT ((int64_t)8 << 30)

// Launch shapes the autotuner chooses (mvn_tune.cu); every choice gives bit-identical results
// (the Cholesky update sums exact integers, the sweeps are per path), only the time differs.
struct TuneParams {
    int chol_bulk_p = 16;      // K sub-chunks (32 wide) per work item of the bulk Cholesky update
    int chol_tail_p = 2;       // the same for the tail update (one 64-wide block column)
    int tc_ctas_per_sm = 2;    // persistent grid of the tensor-core sweep
    int simt_ctas_per_sm = 2;  // persistent grid of the CUDA-core sweep
};

struct mvn_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    int sm_count = 0;
    std::string err;
    int64_t launches = 0;
    // device status word
    int* d_status = nullptr;
    // grow-only workspace arena: slots are handed out per call (see ws_reserve)
    void* ws = nullptr;
    size_t ws_size = 0;
    // lattice generators alpha_i (u64) for i < n_alpha, computed on the device once
    uint64_t* d_alpha = nullptr;
    int n_alpha = 0;
    // internal streams (high and low priority) and events for work that forks off `stream`
    // and joins it again within one call (created on first use)
    cudaStream_t aux[2] = {nullptr, nullptr};
    cudaEvent_t aux_ev[8] = {};
    // autotuned launch shapes, keyed by (precision, log2 bucket of n, log2 bucket of path tiles)
    std::map<std::tuple<int, int, int>, TuneParams> tune;
    // per-kernel timing (mvn_timing): CUDA events recorded around selected launches
    bool timing = false;
    std::vector<cudaEvent_t> ev_pool;
    size_t ev_used = 0;
    std::map<std::string, std::vector<std::pair<cudaEvent_t, cudaEvent_t>>> ktimes;
    // bytes of the y and ybar buffers of mvn_sov_grad (path tiles beyond it run in batches)
    int64_t grad_y_limit = MVN_GRAD_Y_LIMIT_DEFAULT;
};

// Events around one launch when timing is enabled (returns nullptr otherwise).
cudaEvent_t timing_event(mvn_ctx* ctx);
cudaEvent_t timing_event_on(mvn_ctx* ctx, cudaStream_t stream);
// Create the internal streams and events (aux[0] high priority, aux[1] low priority).
mvn_status ctx_aux(mvn_ctx* ctx);
void timing_record(mvn_ctx* ctx, const char* name, cudaEvent_t a, cudaEvent_t b);
#define MVN_TIMED(ctx, name, launch)                                                         \
    do {                                                                                     \
        cudaEvent_t ta_ = timing_event(ctx);                                                 \
        launch;                                                                              \
        MVN_LAUNCHED(ctx);                                                                   \
        cudaEvent_t tb_ = timing_event(ctx);                                                 \
        timing_record(ctx, name, ta_, tb_);                                                  \
    } while (0)

// The same for a launch on another stream of the context.
#define MVN_TIMED_ON(ctx, strm, name, launch)                                                \
    do {                                                                                     \
        cudaEvent_t ta_ = timing_event_on(ctx, strm);                                        \
        launch;                                                                              \
        MVN_LAUNCHED(ctx);                                                                   \
        cudaEvent_t tb_ = timing_event_on(ctx, strm);                                        \
        timing_record(ctx, name, ta_, tb_);                                                  \
    } while (0)

// Record an error message on the context and return the status.
mvn_status mvn_fail(mvn_ctx* ctx, mvn_status st, const char* fmt, ...);
// Check a CUDA runtime result; on error record it and return MVN_ERR_CUDA.
#define MVN_CUDA(ctx, call)                                                                  \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return mvn_fail((ctx), MVN_ERR_CUDA, "%s: %s (%s:%d)", #call,                    \
                            cudaGetErrorString(e_), __FILE__, __LINE__);                     \
    } while (0)
#define MVN_TRY(expr)                                                                        \
    do {                                                                                     \
        mvn_status s_ = (expr);                                                              \
        if (s_ != MVN_OK) return s_;                                                         \
    } while (0)
// After a kernel launch: count it and check the launch error.
#define MVN_LAUNCHED(ctx)                                                                    \
    do {                                                                                     \
        (ctx)->launches++;                                                                   \
        MVN_CUDA((ctx), cudaGetLastError());                                                 \
    } while (0)

// Tuned launch shapes for a Cholesky of order n (MVN_MIXED) and for a sweep of problems of
// dimension up to n over `ntiles` 128-path tiles; defaults where the tuner has no entry.
TuneParams tune_chol(const mvn_ctx* ctx, int n);
TuneParams tune_sweep(const mvn_ctx* ctx, mvn_prec prec, int n, int64_t ntiles);

// Workspace: reserve `bytes` (256-byte aligned partition) of the arena, growing it if needed.
// Growth synchronises the stream first (an allocation never happens mid-stream).
mvn_status ws_reserve(mvn_ctx* ctx, size_t bytes);
// Carve slices out of the reserved arena in order.
struct WsCarver {
    char* base;
    size_t off = 0;
    explicit WsCarver(void* b) : base((char*)b) {}
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~(size_t)255;
        T* p = (T*)(base + off);
        off += count * sizeof(T);
        return p;
    }
};
static inline size_t ws_round(size_t bytes) { return (bytes + 255) & ~(size_t)255; }

// Ensure ctx->d_alpha holds the lattice generators of at least n dimensions.
mvn_status lattice_ensure(mvn_ctx* ctx, int n);
// Fill delta[q * n + i] = SplitMix64(seed, q * 2^32 + i) on the device.
mvn_status lattice_shifts(mvn_ctx* ctx, uint64_t seed, int M, int n, uint64_t* delta);

// Raise an error code in the device status word (first error wins).
__device__ __forceinline__ void dev_raise(int* status, int code, int info) {
    if (atomicCAS(status, 0, code) == 0 && info) status[1] = info;
}

// ---------------------------------------------------------------- lattice point (device)
// w = ((W >> 11) + 1/2) 2^-53,  W = j * alpha + delta (mod 2^64)
__device__ __forceinline__ double lattice_w(uint64_t j, uint64_t alpha, uint64_t delta) {
    uint64_t W = j * alpha + delta;
    return ((double)(W >> 11) + 0.5) * 0x1p-53;
}

// SplitMix64 output for counter c under key `seed` (Steele, Lea, Flood 2014).
__host__ __device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1u) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// ---------------------------------------------------------------- launch helpers (host)
mvn_status sov_reduce_launch(mvn_ctx* ctx, const double* logw, int64_t Ns, int M, double err_k,
                             double* out3, int nprob, int64_t prob_stride);
