// mvn_sov_tc.cu -- the SOV sweep with the limit-update GEMM (Alg. 2 step (c)) on the tcgen05
// tensor cores (MVN_MIXED).
//
// One CTA owns 128 paths (= the 128 TMEM lanes, one thread per path) and walks the dimensions in
// super-blocks of 128.  For super-block R (dimensions d0 = 128 R ..) the part of the limit shift
// that comes from all earlier dimensions,
//   S(paths, d0:d0+128) = Y(paths, 0:d0) L(d0:d0+128, 0:d0)^T,
// is an M = 128, N = 128, K = d0 GEMM whose operands stream through shared memory with 1-D bulk
// copies (K = 32 per stage, 3-stage mbarrier ring, later stages prefetched into L2) and
// accumulate in tensor memory.  FP32 accuracy of the shift is recovered from FP16 operands by
// two-slice splits,
//   L 2^-e_v = Lh + Ll,  y = Yh + Yl,   S_v = 2^e_v (Yh Lh^T + Yh Ll^T + Yl Lh^T)
// (the Yl Ll^T term, ~2^-22 relative, dropped), all three products into one TMEM accumulator;
// e_v is a per-row power of two that keeps row v of L below 2^12 (no FP16 overflow for any
// scale of Sigma).  The tensor cores accumulate in FP32 with truncation, so the accumulator is
// drained into FP32 registers every K = 128 (two ping-pong TMEM buffers), which keeps the
// accumulated error near that of an FP32 sum.  A fifth warp drives the copy/MMA pipeline and
// meets the path threads only at mbarriers, so that copies, MMAs and drains overlap.
// The 128 x 128 diagonal block (Alg. 3) then runs on the CUDA cores in FP32, one dimension at a
// time in a rolled loop: the far shifts and the new y values sit in tensor memory (one column
// per dimension, one lane per path), the packed lower triangle of the block is brought into the
// idle stage area by one bulk copy, and s_v = far_v + sum_{u<v} L_vu y_u is a left-looking dot
// over y read back 16 columns at a time.  Each thread finally writes its path's y values (both
// slices) to a per-CTA global buffer in the swizzled operand layout, from where later
// super-blocks stream them back.  Paths are independent: no CTA waits on another.
#include <cuda_fp16.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "mvn_internal.cuh"
#include "mvn_sov.cuh"
#include "mvn_sov_step.cuh"
#include "mvn_tc.cuh"

#define TC_P 128            // paths per CTA (MMA M, TMEM lanes)
#define TC_N 128            // dimensions per super-block (MMA N)
#define TC_KS 32            // K per pipeline stage (one 64-byte swizzled row of FP16)
#define TC_NST 3            // pipeline stages
#define TC_PF 6             // stages prefetched into L2 ahead of the shared-memory copy
#define TC_G 4              // stages per TMEM accumulation group (K = 128), then drained
#define TC_TILE 8192        // one FP16 slice of a 128-row x 32-column tile (64-byte swizzle)
#define TC_STAGE (4 * TC_TILE)  // Yh, Yl, Lh, Ll
#define TC_TMEM_COLS 256    // two accumulation buffers of 128 columns
#define TC_TRI (TC_N * (TC_N + 1) / 2 + 16)    // packed lower triangle (+ zero pad)
#define TC_RCP TC_TRI                          // then 1 / L_vv
#define TC_BAND (TC_RCP + TC_N)                // then the band L(v + p, v), p < 16, by v
#define TC_DPACK (TC_BAND + 16 * TC_N)         // floats of one packed diagonal block
#define TC_WAIT_BUDGET 4000000000LL  // cycles (~2 s) before a wait gives up

// Split-factor tile pair (hi, lo) of super-block rb (rows 128 rb ..) and K sub-chunk kc < 4 rb.
__host__ __device__ __forceinline__ size_t tc_lt_off(int rb, int kc) {
    return ((size_t)2 * rb * (rb - 1) + kc) * 2 * TC_TILE;
}

// ---------------------------------------------------------------- operand preparation

// Row maxima max_u |L_vu| over the lower triangle: CTA (row block of 128, column chunk of 512),
// thread = row; the maxima of non-negative doubles are combined as their bit patterns (ordered
// like the values).  rowmax must start at zero.
#define TC_RM_COLS 512
__global__ void k_row_max(int n, const double* __restrict__ L, int64_t ld,
                          unsigned long long* __restrict__ rowmax) {
    const int v = blockIdx.x * TC_N + threadIdx.x;
    const int u0 = blockIdx.y * TC_RM_COLS;
    if (v >= n || u0 > v) return;
    const int u1 = min(u0 + TC_RM_COLS, v + 1);
    double mx = 0.0;
#pragma unroll 8
    for (int u = u0; u < u1; ++u) mx = fmax(mx, fabs(L[v + (int64_t)u * ld]));
    if (mx > 0.0) atomicMax(rowmax + v, (unsigned long long)__double_as_longlong(mx));
}

// e_v with 2^(e_v + 12) > max_u |L_vu|, and 2^e_v.
__global__ void k_row_exp(int nrows, const unsigned long long* __restrict__ rowmax,
                          int* __restrict__ eL, float* __restrict__ escale) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= nrows) return;
    const double mx = __longlong_as_double((long long)rowmax[v]);
    int e = 0;
    if (mx > 0.0) frexp(mx, &e);  // mx = m 2^e, m in [0.5, 1)
    e -= 12;
    eL[v] = e;
    escale[v] = ldexpf(1.0f, e);
}

// FP16 slices of L 2^-e_v for the tile pair (rb, kc), kc < 4 rb: one CTA of 128 threads, thread
// = row, writing whole 64-byte tile rows.  Rows >= n are zero.
__global__ void __launch_bounds__(128) k_split_L(int n, const double* __restrict__ L, int64_t ld,
                                                 const int* __restrict__ eL,
                                                 uint8_t* __restrict__ Lt) {
    const int kc = blockIdx.x, rb = blockIdx.y;
    if (kc >= 4 * rb) return;
    const int r = threadIdx.x, v = TC_N * rb + r;
    uint8_t* hi = Lt + tc_lt_off(rb, kc);
    uint8_t* lo = hi + TC_TILE;
    const int e = (v < n) ? -eL[v] : 0;
#pragma unroll
    for (int c8 = 0; c8 < 4; ++c8) {
        __align__(16) __half h[8], l[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int u = TC_KS * kc + 8 * c8 + q;
            const double x = (v < n) ? ldexp(L[v + (int64_t)u * ld], e) : 0.0;
            h[q] = __double2half(x);
            l[q] = __double2half(x - (double)__half2float(h[q]));
        }
        const uint32_t off = tc::sw64_off((uint32_t)r, (uint32_t)(8 * c8));
        *reinterpret_cast<uint4*>(hi + off) = *reinterpret_cast<const uint4*>(h);
        *reinterpret_cast<uint4*>(lo + off) = *reinterpret_cast<const uint4*>(l);
    }
}

// Packed FP32 diagonal block of super-block rb: the lower triangle of L(d0:d0+128, d0:d0+128),
// row-packed (v (v + 1) / 2 + u), then 16 zeros (the left-looking dot reads up to 15 entries past
// a row; they meet y values that are still zero); then 1 / L_vv (the same FP32 division as in
// the step); then the band below the diagonal by column, band[16 v + p] = L(v + p, v) for
// 1 <= p < 16 (zero past the block, p = 0 unused), for the right-looking update in vector loads.
// Rows beyond n: zero, diagonal one.
__global__ void k_pack_D(int n, const double* __restrict__ L, int64_t ld, float* __restrict__ D) {
    const int rb = blockIdx.x, d0 = TC_N * rb;
    float* out = D + (size_t)rb * TC_DPACK;
    for (int e = threadIdx.x; e < TC_N * TC_N; e += blockDim.x) {
        const int v = e % TC_N, u = e / TC_N;  // consecutive threads: consecutive rows
        if (u > v) continue;
        float x;
        if (d0 + v < n)
            x = (float)L[(d0 + v) + (int64_t)(d0 + u) * ld];
        else
            x = (u == v) ? 1.0f : 0.0f;
        out[v * (v + 1) / 2 + u] = x;
        if (u == v) out[TC_RCP + v] = 1.0f / x;
        const int p = v - u;
        if (p > 0 && p < 16) out[TC_BAND + 16 * u + p] = x;
    }
    if (threadIdx.x < 16) out[TC_N * (TC_N + 1) / 2 + threadIdx.x] = 0.0f;
    for (int e = threadIdx.x; e < TC_N * 16; e += blockDim.x) {
        const int u = e >> 4, p = e & 15;
        if (p == 0 || u + p >= TC_N) out[TC_BAND + e] = 0.0f;
    }
}

// ---------------------------------------------------------------- shared memory

// ~102 KB: two CTAs fit on one SM (157 tiles of 20,000 paths are resident at once).  The
// stages (far GEMM) and the packed diagonal block (diagonal work) are never live together.
struct __align__(1024) TcSmem {
    union {
        uint8_t stage[TC_NST][TC_STAGE];  // [Yh 8K | Yl 8K | Lh 8K | Ll 8K]
        float D[TC_DPACK];                // packed diagonal block of the super-block
    };
    double a[TC_N], b[TC_N];
    float af[TC_N], bf[TC_N];
    float escale[TC_N];
    uint64_t alpha[TC_N];
    unsigned char ainf[TC_N], binf[TC_N];
    uint64_t full[TC_NST], empty[TC_NST], accf[2], drained[2], ybar, dbar, fin;
    uint32_t tmem;
    int item;
    int abort;
};

static_assert(sizeof(TcSmem) <= 112 * 1024, "two CTAs per SM need <= 112 KB each");
static_assert(TC_DPACK * 4 <= TC_NST * TC_STAGE, "the diagonal block lives in the stage area");
static_assert(TC_BAND % 4 == 0 && (TC_DPACK * 4) % 16 == 0, "vector loads / bulk copy alignment");
static_assert(TC_P == TC_N, "one path thread per dimension of a super-block loads its limits");

// ---------------------------------------------------------------- roles and barriers
//
// A CTA has TC_P path threads (warps 0-3; thread t owns path t of the tile and TMEM lane t) and
// two pipeline warps: lane 0 of warp 4 streams the far GEMMs' operands (the producer), lane 0 of
// warp 5 issues their MMAs.  The roles meet only at mbarriers, so bulk copies, MMAs and TMEM
// drains overlap, and the issue costs of the copies and of the MMAs fall on different threads:
//   - the stages of all far GEMMs form one sequence; stage number q uses slot q % TC_NST, whose
//     "full" barrier completes for the (q / TC_NST)-th time when its bulk copies land and whose
//     "empty" barrier completes when the MMAs reading it are done;
//   - stages are grouped by TC_G; group number g accumulates into TMEM buffer g % 2 and commits
//     to accf[g % 2]; the path threads drain it and arrive on drained[g % 2] (TC_P arrivals),
//     which the first MMA of group g + 2 waits for;
//   - ybar completes once per super-block whose y the path threads have written (they then no
//     longer use its TMEM buffers or its diagonal block in the stage area): the far GEMM of the
//     next super-block starts after it, on both pipeline threads.
// All parities follow from these counters, so no barrier phase is skipped or waited twice.  The
// path threads synchronise among themselves with barrier 1 and reduce their abort decisions in
// it, so that they always leave the loop together.
#define TC_THREADS (TC_P + 64)
#define TC_PRODUCER TC_P         // thread that issues the bulk copies
#define TC_ISSUER (TC_P + 32)    // thread that issues the MMAs

struct TcPipe {
    uint32_t q = 0;       // global stage number of the next load (producer) / MMA stage (issuer)
    uint32_t g_next = 0;  // global group number of the next far GEMM's group 0 (issuer)
    uint32_t ywait = 0;   // completions of ybar waited for
};

__device__ __forceinline__ uint32_t tc_buf_col(uint32_t g) { return (g & 1u) * TC_N; }

__device__ __forceinline__ int tc_groups(int rb) { return (4 * rb + TC_G - 1) / TC_G; }

// Bounded wait that also gives up as soon as another role of the CTA has aborted.
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!tc::mbar_try_wait(bar, parity)) {
        if (*abort_flag || clock64() - t0 > TC_WAIT_BUDGET) return false;
    }
    return true;
}

// Barrier 1 over the TC_P path threads; returns whether any of them passed `flag`.
__device__ __forceinline__ bool tc_path_sync_or(bool flag) {
    uint32_t r;
    __syncwarp();
    asm volatile(
        "{\n .reg .pred a, b;\n setp.ne.u32 a, %1, 0;\n"
        " bar.red.or.pred b, 1, %2, a;\n selp.u32 %0, 1, 0, b;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)flag), "n"(TC_P)
        : "memory");
    return r != 0;
}
__device__ __forceinline__ void tc_path_sync() {
    __syncwarp();
    asm volatile("bar.sync 1, %0;" ::"n"(TC_P) : "memory");
}

// Operand stream of the far GEMM of super-block rb (K = 128 rb), run by the producer: each
// stage's bulk copies (Y and L tile pairs) as soon as its slot is free, and the stage TC_PF
// ahead prefetched into L2, so that the copy into shared memory does not wait for HBM.
// Returns false on timeout or abort.
__device__ bool tc_far_load(TcSmem& sm, TcPipe& pp, const uint8_t* Ybuf, const uint8_t* Lt,
                            int rb) {
    const uint8_t* Lsb = Lt + tc_lt_off(rb, 0);
    const int kcs = 4 * rb;
    volatile int* abort_flag = &sm.abort;
    for (int kp = 0; kp < min(kcs, TC_PF); ++kp) {
        tc::bulk_prefetch_l2(Ybuf + (size_t)kp * 2 * TC_TILE, 2 * TC_TILE);
        tc::bulk_prefetch_l2(Lsb + (size_t)kp * 2 * TC_TILE, 2 * TC_TILE);
    }
    for (int kc = 0; kc < kcs; ++kc, ++pp.q) {
        const uint32_t q = pp.q;
        const int slot = (int)(q % TC_NST);
        if (q >= TC_NST && !tc_wait(&sm.empty[slot], ((q / TC_NST) - 1) & 1u, abort_flag))
            return false;
        uint8_t* st = sm.stage[slot];
        tc::mbar_arrive_expect_tx(&sm.full[slot], TC_STAGE);
        tc::bulk_g2s(st, Ybuf + (size_t)kc * 2 * TC_TILE, 2 * TC_TILE, &sm.full[slot]);
        tc::bulk_g2s(st + 2 * TC_TILE, Lsb + (size_t)kc * 2 * TC_TILE, 2 * TC_TILE,
                     &sm.full[slot]);
        const int kp = kc + TC_PF;
        if (kp < kcs) {
            tc::bulk_prefetch_l2(Ybuf + (size_t)kp * 2 * TC_TILE, 2 * TC_TILE);
            tc::bulk_prefetch_l2(Lsb + (size_t)kp * 2 * TC_TILE, 2 * TC_TILE);
        }
    }
    return true;
}

// MMAs of the far GEMM of super-block rb, run by the issuer: a stage's three split products as
// soon as its data has landed (and, for a group's first stage, its TMEM buffer has been
// drained); each stage's slot is released by a commit to its "empty" barrier, each group's
// buffer by a commit to accf.  Returns false on timeout or abort.
__device__ bool tc_far_mma(TcSmem& sm, TcPipe& pp, int rb) {
    const uint32_t idesc = tc::idesc_f16_f32(TC_P, TC_N);
    const int kcs = 4 * rb;
    volatile int* abort_flag = &sm.abort;
    for (int kc = 0; kc < kcs; ++kc, ++pp.q) {
        const uint32_t q = pp.q;
        const int slot = (int)(q % TC_NST);
        const uint32_t g = pp.g_next + (uint32_t)(kc / TC_G);
        // a group's first MMA overwrites buffer g % 2: group g - 2 must have been drained
        if (kc % TC_G == 0 && g >= 2u &&
            !tc_wait(&sm.drained[g & 1u], ((g >> 1) - 1u) & 1u, abort_flag))
            return false;
        if (!tc_wait(&sm.full[slot], (q / TC_NST) & 1u, abort_flag)) return false;
        tc::tc_fence_after();
        const uint32_t acc = sm.tmem + tc_buf_col(g);
        const uint32_t base = tc::smem_u32(sm.stage[slot]);
#pragma unroll
        for (int k16 = 0; k16 < 2; ++k16) {
            const uint32_t ko = k16 * 32;
            const uint64_t ah = tc::sdesc_sw64(base + ko);
            const uint64_t al = tc::sdesc_sw64(base + TC_TILE + ko);
            const uint64_t bh = tc::sdesc_sw64(base + 2 * TC_TILE + ko);
            const uint64_t bl = tc::sdesc_sw64(base + 3 * TC_TILE + ko);
            const uint32_t first = (kc % TC_G == 0 && k16 == 0) ? 0u : 1u;
            tc::mma_f16(acc, ah, bh, idesc, first);
            tc::mma_f16(acc, ah, bl, idesc, 1u);
            tc::mma_f16(acc, al, bh, idesc, 1u);
        }
        tc::mma_commit(&sm.empty[slot]);
        if (kc % TC_G == TC_G - 1 || kc == kcs - 1) tc::mma_commit(&sm.accf[g & 1u]);
    }
    pp.g_next += (uint32_t)tc_groups(rb);
    return true;
}

// Far part of the limit shift of this thread's path for super-block rb (K = 128 rb): the groups
// g0, g0 + 1, .. are drained from TMEM as they complete and added into FP32 registers; each
// buffer goes back to the pipeline thread through drained[].  Returns false if a wait timed out
// or another role aborted.
__device__ bool tc_far_drain(TcSmem& sm, int rb, uint32_t g0, float (&s)[TC_N]) {
    const int t = threadIdx.x;
    const int ng = tc_groups(rb);
#pragma unroll
    for (int v = 0; v < TC_N; ++v) s[v] = 0.0f;
    const uint32_t lane_base = ((uint32_t)(t >> 5) * 32u) << 16;
    volatile int* abort_flag = &sm.abort;
    for (int gi = 0; gi < ng; ++gi) {
        const uint32_t g = g0 + (uint32_t)gi;
        if (!tc_wait(&sm.accf[g & 1u], (g >> 1) & 1u, abort_flag)) return false;
        tc::tc_fence_after();
        const uint32_t col = sm.tmem + lane_base + tc_buf_col(g);
#pragma unroll
        for (int c = 0; c < TC_N; c += 16) {
            float v[16];
            tc::tmem_ld16(col + c, v);
#pragma unroll
            for (int i = 0; i < 16; ++i) s[c + i] += v[i];
        }
        tc::tc_fence_before();
        tc::mbar_arrive(&sm.drained[g & 1u]);
    }
#pragma unroll
    for (int v = 0; v < TC_N; ++v) s[v] *= sm.escale[v];
    return true;
}

// Write 32 y values of this thread's path (two FP16 slices) as row `t` of the Y tiles of
// sub-chunk kc.
__device__ __forceinline__ void tc_write_y32(uint8_t* __restrict__ Ybuf, int kc, int t,
                                             const float (&y)[32]) {
    uint8_t* hi = Ybuf + (size_t)kc * 2 * TC_TILE;
    uint8_t* lo = hi + TC_TILE;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        __align__(16) __half h[8], l[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const float v = y[8 * c + e];
            h[e] = __float2half_rn(v);
            l[e] = __float2half_rn(v - __half2float(h[e]));
        }
        const uint32_t off = tc::sw64_off((uint32_t)t, (uint32_t)(8 * c));
        *reinterpret_cast<uint4*>(hi + off) = *reinterpret_cast<const uint4*>(h);
        *reinterpret_cast<uint4*>(lo + off) = *reinterpret_cast<const uint4*>(l);
    }
}

struct TcBatch {
    SovProblem single;
    const SovProblem* probs;
    const int2* items;
    int nitems;
    int* counter;
    const uint8_t* Lt;     // split factor tile pairs
    const float* escale;   // per-row scale 2^e_v of the split factor
    const float* Dpack;    // packed diagonal blocks
    uint8_t* Yscratch;     // per-CTA Y buffers
    int64_t ystride;       // bytes per CTA buffer
    int* status;
};

// Shared set-up of the tensor-core kernels: barriers and TMEM.
__device__ __forceinline__ void tc_setup(TcSmem& sm) {
    const int t = threadIdx.x;
    if (t == 0) {
        for (int s = 0; s < TC_NST; ++s) {
            tc::mbar_init(&sm.full[s], 1);
            tc::mbar_init(&sm.empty[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            tc::mbar_init(&sm.accf[b], 1);
            tc::mbar_init(&sm.drained[b], TC_P);
        }
        tc::mbar_init(&sm.ybar, TC_P);
        tc::mbar_init(&sm.dbar, 1);
        tc::mbar_init(&sm.fin, 1);
        tc::mbar_fence_init();
        sm.abort = 0;
    }
    if ((t >> 5) == 0) {
        tc::tmem_alloc(&sm.tmem, TC_TMEM_COLS);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
}

// Before shared and tensor memory are released: every copy this CTA issued has landed and every
// MMA it issued has completed (bounded waits; also after an aborted wait).  Path thread 0 issued
// the diagonal-block copies, the producer the stage copies, the issuer the MMAs.  A wait that
// runs out here means work may still be in flight when the memory is released, so the result
// cannot be trusted: it raises MVN_ERR_TIMEOUT like the waits of the main loop.
__device__ __forceinline__ void tc_quiesce(TcSmem& sm, const TcPipe& pp, uint32_t dphase,
                                           int* status) {
    const int t = threadIdx.x;
    bool ok = true;
    if (t == 0 && dphase > 0) ok &= tc::mbar_wait(&sm.dbar, (dphase - 1) & 1u, TC_WAIT_BUDGET);
    if (t == TC_PRODUCER) {
        const uint32_t q0 = pp.q > TC_NST ? pp.q - TC_NST : 0u;
        for (uint32_t q = q0; q < pp.q; ++q)
            ok &= tc::mbar_wait(&sm.full[q % TC_NST], (q / TC_NST) & 1u, TC_WAIT_BUDGET);
    }
    if (t == TC_ISSUER) {
        tc::mma_commit(&sm.fin);
        ok &= tc::mbar_wait(&sm.fin, 0, TC_WAIT_BUDGET);
    }
    if (!ok) dev_raise(status, MVN_ERR_TIMEOUT, 0);
}

__device__ __forceinline__ void tc_teardown(TcSmem& sm) {
    tc::tc_fence_before();
    __syncthreads();
    if ((threadIdx.x >> 5) == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(sm.tmem, TC_TMEM_COLS);
    }
}

__device__ __forceinline__ TcSmem& tc_smem(uint8_t* raw) {
    return *reinterpret_cast<TcSmem*>((reinterpret_cast<uintptr_t>(raw) + 1023) &
                                      ~(uintptr_t)1023);
}

__device__ __forceinline__ constexpr int tri(int v, int u) { return v * (v + 1) / 2 + u; }

// Raise a timeout once and make every role of the CTA stop.
__device__ __forceinline__ void tc_fail(TcSmem& sm, int* status) {
    sm.abort = 1;
    dev_raise(status, MVN_ERR_TIMEOUT, 0);
}

__global__ void __launch_bounds__(TC_THREADS, 2) k_sov_tc(const TcBatch bt,
                                                          const uint64_t* __restrict__ alpha) {
    extern __shared__ uint8_t smem_raw[];
    TcSmem& sm = tc_smem(smem_raw);
    const int t = threadIdx.x;
    tc_setup(sm);
    TcPipe pp;            // producer / issuer state
    uint32_t dphase = 0;  // loads of the packed diagonal block issued (path thread 0)
    uint32_t g_all = 0;   // accumulation groups of all far GEMMs so far (path threads)
    uint8_t* Ybuf = bt.Yscratch + (int64_t)blockIdx.x * bt.ystride;
    const uint32_t lane_base = ((uint32_t)(t >> 5) * 32u) << 16;

    for (;;) {
        if (t == 0) sm.item = atomicAdd(bt.counter, 1);
        __syncthreads();
        const int it = sm.item;
        if (it >= bt.nitems || sm.abort) break;
        const SovProblem& P = (bt.probs == nullptr) ? bt.single : bt.probs[bt.items[it].x];
        const int n = P.n;
        const int nsb = (n + TC_N - 1) / TC_N;
        if (t >= TC_P) {
            // ------------------------------------------------ pipeline warps: far GEMMs 1 .. nsb-1
            if (t == TC_PRODUCER || t == TC_ISSUER) {
                for (int rb = 1; rb < nsb; ++rb) {
                    // y of super-block rb - 1 written, its buffers and diagonal block released
                    if (!tc_wait(&sm.ybar, pp.ywait & 1u, &sm.abort)) {
                        tc_fail(sm, bt.status);
                        break;
                    }
                    ++pp.ywait;
                    tc::tc_fence_after();
                    const bool ok = (t == TC_PRODUCER) ? tc_far_load(sm, pp, Ybuf, bt.Lt, rb)
                                                       : tc_far_mma(sm, pp, rb);
                    if (!ok) {
                        tc_fail(sm, bt.status);
                        break;
                    }
                }
            }
            __syncwarp();
        } else {
            // ------------------------------------------------ path threads
            const int tile = (bt.probs == nullptr) ? it : bt.items[it].y;
            const int64_t p = (int64_t)tile * TC_P + t;
            const bool valid = p < P.Ntot;
            const int64_t pg = P.p0 + p;  // index of the path in the whole lattice rule
            const int64_t q = valid ? pg / P.Ns : 0;
            const uint64_t j = valid ? (uint64_t)(pg - q * P.Ns) + 1u : 1u;
            const uint64_t* __restrict__ dq = P.delta + q * P.dstride;
            DFProd lp;
            int pf = 0;
            int next_k = (P.nprefix > 0) ? P.prefix[0] : -1;
            bool done = true;
            for (int rb = 0; rb < nsb; ++rb) {
                const int d0 = rb * TC_N;
                const int nb2 = min(TC_N, n - d0);
                {
                    const int v = d0 + t;
                    const double av = (t < nb2) ? P.a[v] : 0.0;
                    const double bv = (t < nb2) ? P.b[v] : 1.0;
                    sm.a[t] = av;
                    sm.b[t] = bv;
                    sm.af[t] = (float)av;
                    sm.bf[t] = (float)bv;
                    sm.ainf[t] = (av == -INFINITY);
                    sm.binf[t] = (bv == INFINITY);
                    sm.alpha[t] = (t < nb2) ? alpha[v] : 0u;
                    sm.escale[t] = bt.escale[v];
                }
                tc_path_sync();
                // far part of the shifts (Alg. 2 step (c) over all earlier super-blocks) -> TMEM
                // buffer 1; buffer 0 receives this super-block's y
                const uint32_t sbuf = sm.tmem + lane_base + TC_N, ybuf = sm.tmem + lane_base;
                bool fail = false;
                {
                    float s[TC_N];
                    if (rb > 0) {
                        fail = !tc_far_drain(sm, rb, g_all, s);
                        g_all += (uint32_t)tc_groups(rb);
                    } else {
#pragma unroll
                        for (int v = 0; v < TC_N; ++v) s[v] = 0.0f;
                    }
                    if (fail) {
                        tc_fail(sm, bt.status);
                    } else {
                        // packed diagonal block into the (now idle) stage area
                        if (t == 0) {
                            tc::fence_proxy_async_smem();
                            tc::mbar_arrive_expect_tx(&sm.dbar, TC_DPACK * 4);
                            tc::bulk_g2s(sm.D, bt.Dpack + (size_t)rb * TC_DPACK, TC_DPACK * 4,
                                         &sm.dbar);
                            ++dphase;
                        }
#pragma unroll
                        for (int c = 0; c < TC_N; c += 32) {
                            float h[32];
#pragma unroll
                            for (int i = 0; i < 32; ++i) h[i] = s[c + i];
                            tc::tmem_st32(sbuf + c, h);
                        }
                    }
                }
                if (t == 0 && !fail && !tc::mbar_wait(&sm.dbar, (dphase - 1) & 1u, TC_WAIT_BUDGET)) {
                    fail = true;
                    tc_fail(sm, bt.status);
                }
                if (tc_path_sync_or(fail || sm.abort)) {
                    done = false;
                    break;
                }
                // diagonal block (Alg. 3) in blocks of 16 dimensions.  For block c the shifts of
                // its dimensions start as q_i = far_i + sum_{u < 16c} L(16c + i, u) y_u (a
                // 16 x 16c mat-vec over the earlier y, read back from TMEM 16 at a time); inside
                // the block the dimensions go one at a time, q being a queue whose head is the
                // current dimension: after the elementwise step of Eq. 2 gives y_v, the later
                // dimensions of the block get L(v + p, v) y_v added (right-looking) and the queue
                // shifts by one.  One copy of the step code serves every dimension.
#pragma unroll 1
                for (int c0 = 0; c0 < nb2; c0 += 16) {
                    float qv[16];
                    tc::tmem_ld16(sbuf + c0, qv);
#pragma unroll 1
                    for (int u0 = 0; u0 < c0; u0 += 16) {
                        float yy[16];
                        tc::tmem_ld16(ybuf + u0, yy);
#pragma unroll
                        for (int i = 0; i < 16; ++i) {
                            const float* Dr = sm.D + tri(c0 + i, u0);
#pragma unroll
                            for (int k = 0; k < 16; ++k) qv[i] = fmaf(Dr[k], yy[k], qv[i]);
                        }
                    }
                    float y16[16];
#pragma unroll 1
                    for (int i = 0; i < 16; ++i) {
                        const int v = c0 + i;
                        float y = 0.0f;
                        if (v < nb2) {
                            float w, wc, dh, dl;
                            uint64_t wm;
                            int dex;
                            lattice_wf(j, sm.alpha[v], dq[d0 + v], w, wc, wm);
                            y = sov_step_f32r(sm.af[v], sm.bf[v], sm.a[v], sm.b[v], sm.ainf[v],
                                              sm.binf[v], qv[0], sm.D[tri(v, v)],
                                              sm.D[TC_RCP + v], w, wc, wm, dh, dl, dex);
                            lp.mul(dh, dl, dex);
                            while (next_k == d0 + v + 1) {
                                if (valid) P.logw_prefix[(int64_t)pf * P.Ntot + p] = lp.log_value();
                                ++pf;
                                next_k = (pf < P.nprefix) ? P.prefix[pf] : -1;
                            }
                        }
                        // later dimensions of the block (column v of the band), then shift
                        // the queues
                        float bd[16];
#pragma unroll
                        for (int c = 0; c < 4; ++c)
                            *reinterpret_cast<float4*>(bd + 4 * c) =
                                *reinterpret_cast<const float4*>(sm.D + TC_BAND + 16 * v + 4 * c);
#pragma unroll
                        for (int pp2 = 1; pp2 < 16; ++pp2)
                            if (pp2 < 16 - i) qv[pp2] = fmaf(bd[pp2], y, qv[pp2]);
#pragma unroll
                        for (int k = 0; k < 15; ++k) {
                            qv[k] = qv[k + 1];
                            y16[k] = y16[k + 1];
                        }
                        qv[15] = 0.0f;
                        y16[15] = y;
                    }
                    tc::tmem_st16(ybuf + c0, y16);
                }
                // y of this super-block -> operand buffer of the later super-blocks (read back
                // by the async proxy: fence, then release it to the pipeline thread through
                // ybar together with the TMEM buffers and the stage area)
                if (d0 + TC_N < n) {
#pragma unroll 1
                    for (int c = 0; c < TC_N; c += 32) {
                        float yy[32];
                        tc::tmem_ld32(ybuf + c, yy);
                        tc_write_y32(Ybuf, (d0 + c) / TC_KS, t, yy);
                    }
                    tc::fence_proxy_async_global();
                    tc::fence_proxy_async_smem();
                    tc::tc_fence_before();
                    tc::mbar_arrive(&sm.ybar);
                }
                tc_path_sync();  // the limits of the next super-block overwrite sm.a ..
            }
            if (done && valid && P.logw) P.logw[p] = lp.log_value();
        }
        __syncthreads();
    }
    tc_quiesce(sm, pp, dphase, bt.status);
    tc_teardown(sm);
}

// ---------------------------------------------------------------- host side

static size_t tc_smem_bytes() { return sizeof(TcSmem) + 1024; }

static int tc_grid(mvn_ctx* ctx, int nmax, int64_t ntiles) {
    // up to two CTAs per SM (shared memory ~103 KB, 256 TMEM columns each); the autotuner picks
    const int per_sm = tune_sweep(ctx, MVN_MIXED, nmax, ntiles).tc_ctas_per_sm;
    return (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, per_sm * (int64_t)ctx->sm_count));
}

static int tc_nsb(int n) { return (std::max(n, 1) + TC_N - 1) / TC_N; }

static size_t tc_factor_bytes(int nsb) {
    return ws_round(tc_lt_off(nsb, 0)) + ws_round(sizeof(int) * (size_t)nsb * TC_N) +
           ws_round(sizeof(unsigned long long) * (size_t)nsb * TC_N) +
           ws_round(sizeof(float) * (size_t)nsb * TC_N) +
           ws_round(sizeof(float) * (size_t)nsb * TC_DPACK);
}

size_t sov_tc_ws_bytes(mvn_ctx* ctx, int nprob, int nmax, int64_t ntiles) {
    const int nsb = tc_nsb(nmax);
    size_t b = ws_round(sizeof(int));
    if (nprob > 1)
        b += ws_round(sizeof(SovProblem) * nprob) + ws_round(sizeof(int2) * (size_t)ntiles);
    b += tc_factor_bytes(nsb);
    b += ws_round((size_t)tc_grid(ctx, nmax, ntiles) * nsb * 4 * 2 * TC_TILE);
    return b;
}

// Operand copies of the factor: split tiles, row scales and packed diagonal blocks.
static mvn_status tc_prepare_factor(mvn_ctx* ctx, int n, const double* L, int64_t ld, int nsb,
                                    WsCarver& wc, uint8_t*& Lt, float*& escale, float*& Dpack) {
    Lt = wc.take<uint8_t>(tc_lt_off(nsb, 0));
    int* eL = wc.take<int>((size_t)nsb * TC_N);
    unsigned long long* rowmax = wc.take<unsigned long long>((size_t)nsb * TC_N);
    escale = wc.take<float>((size_t)nsb * TC_N);
    Dpack = wc.take<float>((size_t)nsb * TC_DPACK);
    const int rows = nsb * TC_N;
    MVN_CUDA(ctx, cudaMemsetAsync(rowmax, 0, sizeof(unsigned long long) * rows, ctx->stream));
    if (n > 0) {
        k_row_max<<<dim3(nsb, (n + TC_RM_COLS - 1) / TC_RM_COLS), TC_N, 0, ctx->stream>>>(
            n, L, ld, rowmax);
        MVN_LAUNCHED(ctx);
    }
    k_row_exp<<<(rows + 127) / 128, 128, 0, ctx->stream>>>(rows, rowmax, eL, escale);
    MVN_LAUNCHED(ctx);
    if (nsb > 1) {
        k_split_L<<<dim3(4 * (nsb - 1), nsb), 128, 0, ctx->stream>>>(n, L, ld, eL, Lt);
        MVN_LAUNCHED(ctx);
    }
    k_pack_D<<<nsb, 256, 0, ctx->stream>>>(n, L, ld, Dpack);
    MVN_LAUNCHED(ctx);
    return MVN_OK;
}

// All problems of a batch share one factor L (the batched problems use its leading blocks).
mvn_status sov_run_tc(mvn_ctx* ctx, const std::vector<SovProblem>& probs_h, char* ws) {
    const int nprob = (int)probs_h.size();
    int nmax = 0;
    int64_t ntiles = 0;
    for (auto& P : probs_h) {
        nmax = std::max(nmax, P.n);
        if (P.n > 0) ntiles += (P.Ntot + TC_P - 1) / TC_P;
    }
    if (ntiles == 0) return MVN_OK;
    const int nsb = tc_nsb(nmax);
    const int grid = tc_grid(ctx, nmax, ntiles);
    WsCarver wc(ws);
    TcBatch bt;
    memset(&bt, 0, sizeof(bt));
    bt.counter = wc.take<int>(1);
    bt.nitems = (int)ntiles;
    if (nprob == 1) {
        bt.single = probs_h[0];
    } else {
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
            int64_t nt = (probs_h[pi].Ntot + TC_P - 1) / TC_P;
            for (int64_t tt = 0; tt < nt; ++tt) items.push_back(make_int2(pi, (int)tt));
        }
        MVN_CUDA(ctx, cudaMemcpyAsync(d_probs, probs_h.data(), sizeof(SovProblem) * nprob,
                                      cudaMemcpyHostToDevice, ctx->stream));
        MVN_CUDA(ctx, cudaMemcpyAsync(d_items, items.data(), sizeof(int2) * items.size(),
                                      cudaMemcpyHostToDevice, ctx->stream));
        bt.probs = d_probs;
        bt.items = d_items;
    }
    const SovProblem& P0 = probs_h[0];
    for (auto& P : probs_h)
        if (P.L != P0.L || P.ld != P0.ld)
            return mvn_fail(ctx, MVN_ERR_ARG, "tensor-core batch needs one shared factor");
    uint8_t* Lt;
    float *escale, *Dpack;
    MVN_TRY(tc_prepare_factor(ctx, nmax, P0.L, P0.ld, nsb, wc, Lt, escale, Dpack));
    bt.Lt = Lt;
    bt.escale = escale;
    bt.Dpack = Dpack;
    bt.ystride = (int64_t)nsb * 4 * 2 * TC_TILE;
    bt.Yscratch = wc.take<uint8_t>((size_t)grid * bt.ystride);
    bt.status = ctx->d_status;
    MVN_CUDA(ctx, cudaMemsetAsync(bt.counter, 0, sizeof(int), ctx->stream));
    const size_t smem = tc_smem_bytes();
    MVN_CUDA(ctx, cudaFuncSetAttribute(k_sov_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    MVN_TIMED(ctx, "k_sov_tc", (k_sov_tc<<<grid, TC_THREADS, smem, ctx->stream>>>(bt, ctx->d_alpha)));
    return MVN_OK;
}

// ---------------------------------------------------------------- GEMM self-test

// S (128 x 128, row-major) = Y (128 x K) L (128 x K)^T through exactly the operand split, tile
// layout, bulk-copy pipeline, descriptors, MMAs, TMEM drains and row scaling of the sweep's far
// GEMM: the test rows form super-block rb = ceil(K / 128) of a factor whose earlier columns are
// the K test columns.  Y rows are written by one thread per path (as the sweep does).
__global__ void k_tc_selftest_fill(int K, const double* __restrict__ L, int rb, int nf,
                                   double* __restrict__ F) {
    // F(128 rb + r, k) = L(r, k), F column-major with leading dimension nf
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < TC_N * K; e += gridDim.x * blockDim.x) {
        const int r = e % TC_N, k = e / TC_N;
        F[(TC_N * rb + r) + (int64_t)k * nf] = L[(int64_t)r * K + k];
    }
}

__global__ void k_tc_selftest_prep(int K, const double* __restrict__ Y, uint8_t* __restrict__ Ybuf) {
    const int t = threadIdx.x;
    for (int kc = 0; kc * TC_KS < K; ++kc) {
        float y[32];
#pragma unroll
        for (int v = 0; v < 32; ++v) {
            const int k = kc * TC_KS + v;
            y[v] = (k < K) ? (float)Y[(int64_t)t * K + k] : 0.0f;
        }
        tc_write_y32(Ybuf, kc, t, y);
    }
    tc::fence_proxy_async_global();
}

__global__ void __launch_bounds__(TC_THREADS, 2) k_tc_selftest(int rb,
                                                               const uint8_t* __restrict__ Ybuf,
                                                               const uint8_t* __restrict__ Lt,
                                                               const float* __restrict__ escale,
                                                               float* __restrict__ S, int* status) {
    extern __shared__ uint8_t smem_raw[];
    TcSmem& sm = tc_smem(smem_raw);
    const int t = threadIdx.x;
    tc_setup(sm);
    TcPipe pp;
    if (t < TC_P) sm.escale[t] = escale[TC_N * rb + t];
    __syncthreads();
    if (t >= TC_P) {
        if (t == TC_PRODUCER && !tc_far_load(sm, pp, Ybuf, Lt, rb)) tc_fail(sm, status);
        if (t == TC_ISSUER && !tc_far_mma(sm, pp, rb)) tc_fail(sm, status);
        __syncwarp();
    } else {
        float s[TC_N];
        if (!tc_far_drain(sm, rb, 0u, s))
            tc_fail(sm, status);
        else
            for (int v = 0; v < TC_N; ++v) S[t * TC_N + v] = s[v];
    }
    tc_quiesce(sm, pp, 0, status);
    tc_teardown(sm);
}

extern "C" mvn_status mvn_tc_selftest(mvn_ctx* ctx, int K, const double* Y, const double* L,
                                      float* S) {
    if (!ctx) return MVN_ERR_ARG;
    if (K < 1 || K > 65536 || !Y || !L || !S)
        return mvn_fail(ctx, MVN_ERR_ARG, "mvn_tc_selftest: invalid argument");
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    // factor of order n = 128 (rb + 1) whose rows 128 rb .. hold the test rows of L in columns
    // 0 .. K-1 (zero elsewhere); built densely on the device, then split like the sweep's factor
    const int rb = (K + TC_N - 1) / TC_N;
    const int nsb = rb + 1;
    const int nf = TC_N * nsb;
    const size_t fbytes = sizeof(double) * (size_t)nf * nf;
    const size_t ybytes = (size_t)nsb * 4 * 2 * TC_TILE;
    MVN_TRY(ws_reserve(ctx, ws_round(fbytes) + tc_factor_bytes(nsb) + ws_round(ybytes) + 1024));
    WsCarver wc(ctx->ws);
    double* F = wc.take<double>((size_t)nf * nf);
    MVN_CUDA(ctx, cudaMemsetAsync(F, 0, fbytes, ctx->stream));
    k_tc_selftest_fill<<<64, 256, 0, ctx->stream>>>(K, L, rb, nf, F);
    MVN_LAUNCHED(ctx);
    uint8_t* Lt;
    float *escale, *Dpack;
    MVN_TRY(tc_prepare_factor(ctx, nf, F, nf, nsb, wc, Lt, escale, Dpack));
    uint8_t* Ybuf = wc.take<uint8_t>(ybytes);
    MVN_CUDA(ctx, cudaMemsetAsync(Ybuf, 0, ybytes, ctx->stream));
    k_tc_selftest_prep<<<1, TC_P, 0, ctx->stream>>>(K, Y, Ybuf);
    MVN_LAUNCHED(ctx);
    const size_t smem = tc_smem_bytes();
    MVN_CUDA(ctx, cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    k_tc_selftest<<<1, TC_THREADS, smem, ctx->stream>>>(rb, Ybuf, Lt, escale, S, ctx->d_status);
    MVN_LAUNCHED(ctx);
    return MVN_OK;
}

// ---------------------------------------------------------------- bounded-wait self-test

// One thread waits on an mbarrier that nothing completes, with the same bounded wait as the
// tensor-core kernels; when the budget runs out it raises MVN_ERR_TIMEOUT and returns.
__global__ void k_wait_selftest(long long budget, int* status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && !tc::mbar_wait(&bar, 0, budget)) dev_raise(status, MVN_ERR_TIMEOUT, 0);
}

extern "C" mvn_status mvn_wait_selftest(mvn_ctx* ctx, int64_t budget_cycles) {
    if (!ctx) return MVN_ERR_ARG;
    if (budget_cycles < 1000 || budget_cycles > 4000000000LL)
        return mvn_fail(ctx, MVN_ERR_ARG, "budget out of [1e3, 4e9] cycles");
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    k_wait_selftest<<<1, 32, 0, ctx->stream>>>(budget_cycles, ctx->d_status);
    MVN_LAUNCHED(ctx);
    return MVN_OK;
}
