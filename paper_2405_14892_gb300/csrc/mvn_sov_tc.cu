// mvn_sov_tc.cu -- the SOV sweep with the limit-update GEMM (Alg. 2 step (c)) on the tcgen05
// tensor cores (MVN_MIXED).
//
// One CTA owns 128 paths (= the 128 TMEM lanes, one thread per path) and walks the dimensions in
// blocks of 64.  For block r the limit shift S(paths, block) = Y(paths, 0:64r) L(block, 0:64r)^T is
// an M=128, N=64, K=64r GEMM whose operands stream through shared memory with 1-D bulk copies
// (3-stage mbarrier pipeline) and whose FP32 accumulators live in tensor memory.  FP32 accuracy of
// the shift is recovered from FP16 operands by splitting each value into two FP16 slices:
//   L * 2^12 = Lh + 2^-11 Ll,  y = Yh + 2^-11 Yl,
//   S = 2^-12 (Yh Lh^T + 2^-11 (Yh Ll^T + Yl Lh^T))   (the Yl Ll^T term, 2^-22 relative, dropped)
// with the two products accumulated in two TMEM accumulators (3 MMAs per K step).  The 2^12
// scaling keeps small entries of L out of the FP16 subnormal range.  The diagonal block (Alg. 3)
// runs on the CUDA cores in FP32 with the running log-weight in FP64; each thread then writes its
// path's 64 new y values (both slices) to a per-CTA global buffer in the swizzled operand layout,
// from where later blocks stream them back.  Paths are independent: no CTA waits on another.
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
#define TC_B 64             // dimensions per block (MMA N, K chunk)
#define TC_STAGES 2
#define TC_G 4              // K chunks per TMEM accumulation group (then drained to registers)
#define TC_YT_BYTES 16384   // one slice of a 128 x 64 FP16 Y tile
#define TC_LT_BYTES 8192    // one slice of a 64 x 64 FP16 L tile
#define TC_STAGE_BYTES (2 * TC_YT_BYTES + 2 * TC_LT_BYTES)
#define TC_TMEM_COLS 256    // two accumulation buffers x (acc1 64 + acc2 64 columns)
#define TC_WAIT_BUDGET 4000000000LL  // cycles (~2 s) before a wait gives up

// ---------------------------------------------------------------- operand preparation

// Split L (FP64, column-major, lower) into FP16 tiles: Lt[slice][kc][rb] is the 64 x 64 tile of
// rows 64 rb.., columns 64 kc.. in the swizzled K-major layout.  Only kc <= rb is written; the
// strict upper part, rows >= n and columns >= n are zero.
__global__ void k_split_L(int n, const double* __restrict__ L, int64_t ld, int nrb,
                          __half* __restrict__ Lt) {
    const int x = blockIdx.x;
    int rb = (int)((sqrt(8.0 * x + 1.0) - 1.0) * 0.5);
    while ((rb + 1) * (rb + 2) / 2 <= x) ++rb;
    while (rb * (rb + 1) / 2 > x) --rb;
    const int kc = x - rb * (rb + 1) / 2;
    const size_t slice = (size_t)nrb * nrb * (TC_LT_BYTES / 2);
    __half* hi = Lt + ((size_t)kc * nrb + rb) * (TC_LT_BYTES / 2);
    __half* lo = hi + slice;
    for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
        const int r = e & 63, k = e >> 6;  // consecutive threads: consecutive rows (coalesced)
        const int i = 64 * rb + r, j = 64 * kc + k;
        double v = (i < n && j < n && j <= i) ? L[i + (int64_t)j * ld] * 4096.0 : 0.0;
        __half h = __double2half(v);
        __half l = __double2half((v - (double)__half2float(h)) * 2048.0);
        const uint32_t off = tc::sw128_off(r, k) >> 1;
        hi[off] = h;
        lo[off] = l;
    }
}

// ---------------------------------------------------------------- shared memory

// ~106 KB: two CTAs fit on one SM (157 tiles of W2's 20,000 paths are resident at once).
struct __align__(1024) TcSmem;
struct __align__(1024) TcSmem {
    uint8_t stage[TC_STAGES][TC_STAGE_BYTES];  // [Yh 16K | Yl 16K | Lh 8K | Ll 8K]
    float Ld[TC_B * (TC_B + 1) / 2];           // diagonal block, packed lower triangle
    double a[TC_B], b[TC_B];
    float af[TC_B], bf[TC_B];
    unsigned char ainf[TC_B], binf[TC_B];
    uint64_t alpha[TC_B];
    uint64_t full[TC_STAGES], empty[TC_STAGES], accf[2], fin;
    uint32_t tmem;
    int item;
    int abort;
};

static_assert(sizeof(TcSmem) <= 112 * 1024, "two CTAs per SM need <= 112 KB each");

// ---------------------------------------------------------------- GEMM pipeline (thread 0)
//
// The K chunks of all blocks form one sequence; chunk number q uses stage q % TC_STAGES, whose
// "full" barrier completes for the (q / TC_STAGES)-th time when its bulk copies land and whose
// "empty" barrier completes when the MMAs reading it are done.  Chunks are grouped by TC_G; group
// number g accumulates into TMEM buffer g % 2 and commits to accf[g % 2] when complete.  All
// parities follow from these counters, so no barrier phase is ever skipped or waited twice.
struct TcPipe {
    uint64_t q_load = 0;  // global chunk number of the next load
    uint64_t q_mma = 0;   // global chunk number of the next MMA chunk
    uint64_t g_next = 0;  // global group number of the group the next MMA chunk belongs to
    // current block
    const uint8_t* Ybuf;
    const uint8_t* Lt;
    size_t lslice;
    int nrb, rb;
    int kcs;              // chunks of the block
    int next_load, next_mma;  // within-block chunk indices
    uint64_t q_block0;    // global chunk number of the block's chunk 0
};

__device__ __forceinline__ uint32_t tc_buf_col(uint64_t g) { return (uint32_t)(g & 1u) * 128u; }

// Issue loads ahead and MMAs for the block's chunks < limit; false on a timed-out wait.
__device__ bool tc_pump(TcSmem& sm, TcPipe& pp, int limit) {
    const uint32_t idesc = tc::idesc_f16_f32(TC_P, TC_B);
    while (pp.next_mma < limit) {
        while (pp.next_load < pp.kcs && pp.next_load < pp.next_mma + TC_STAGES) {
            const uint64_t q = pp.q_load;
            const int s = (int)(q % TC_STAGES);
            if (q >= TC_STAGES) {  // the MMAs of chunk q - TC_STAGES must have left the stage
                const uint32_t par = (uint32_t)((q / TC_STAGES - 1) & 1u);
                if (!tc::mbar_wait(&sm.empty[s], par, TC_WAIT_BUDGET)) return false;
            }
            uint8_t* st = sm.stage[s];
            const int kc = pp.next_load;
            tc::mbar_arrive_expect_tx(&sm.full[s], TC_STAGE_BYTES);
            tc::bulk_g2s(st, pp.Ybuf + (size_t)kc * 2 * TC_YT_BYTES, 2 * TC_YT_BYTES, &sm.full[s]);
            const uint8_t* lt = pp.Lt + ((size_t)kc * pp.nrb + pp.rb) * TC_LT_BYTES;
            tc::bulk_g2s(st + 2 * TC_YT_BYTES, lt, TC_LT_BYTES, &sm.full[s]);
            tc::bulk_g2s(st + 2 * TC_YT_BYTES + TC_LT_BYTES, lt + pp.lslice, TC_LT_BYTES,
                         &sm.full[s]);
            ++pp.q_load;
            ++pp.next_load;
        }
        const uint64_t q = pp.q_mma;
        const int s = (int)(q % TC_STAGES);
        if (!tc::mbar_wait(&sm.full[s], (uint32_t)((q / TC_STAGES) & 1u), TC_WAIT_BUDGET))
            return false;
        tc::tc_fence_after();
        const int kc = pp.next_mma;
        const uint64_t g = pp.g_next + (uint64_t)(kc / TC_G);
        const uint32_t acc1 = sm.tmem + tc_buf_col(g), acc2 = acc1 + TC_B;
        const uint32_t base = tc::smem_u32(sm.stage[s]);
#pragma unroll
        for (int k16 = 0; k16 < 4; ++k16) {
            const uint32_t ko = k16 * 32;
            const uint64_t ah = tc::sdesc_sw128(base + ko);
            const uint64_t al = tc::sdesc_sw128(base + TC_YT_BYTES + ko);
            const uint64_t bh = tc::sdesc_sw128(base + 2 * TC_YT_BYTES + ko);
            const uint64_t bl = tc::sdesc_sw128(base + 2 * TC_YT_BYTES + TC_LT_BYTES + ko);
            const uint32_t first = (kc % TC_G == 0 && k16 == 0) ? 0u : 1u;
            tc::mma_f16(acc1, ah, bh, idesc, first);
            tc::mma_f16(acc2, ah, bl, idesc, first);
            tc::mma_f16(acc2, al, bh, idesc, 1u);
        }
        tc::mma_commit(&sm.empty[s]);
        if (kc % TC_G == TC_G - 1 || kc == pp.kcs - 1) tc::mma_commit(&sm.accf[g & 1u]);
        ++pp.q_mma;
        ++pp.next_mma;
    }
    return true;
}

// Limit shift of this thread's path for the block's 64 dimensions: the K chunks are accumulated
// in TMEM group by group (TC_G chunks each, two ping-pong buffers) and every group's partial sums
// are added into FP32 registers.  Short in-TMEM accumulation chains keep the tensor cores'
// accumulation error near that of an FP32 sum.  All threads call this; thread 0 also issues.
// Returns false if a wait timed out.
__device__ bool tc_block_shift(TcSmem& sm, TcPipe& pp, const uint8_t* Ybuf, const uint8_t* Lt,
                               int nrb, int rb, uint64_t& g_all, float (&s)[TC_B]) {
    const int t = threadIdx.x;
    const int kcs = rb;  // chunks 0 .. rb-1
    const int ng = (kcs + TC_G - 1) / TC_G;
    bool ok = true;
    if (t == 0) {
        pp.Ybuf = Ybuf;
        pp.Lt = Lt;
        pp.lslice = (size_t)nrb * nrb * TC_LT_BYTES;
        pp.nrb = nrb;
        pp.rb = rb;
        pp.kcs = kcs;
        pp.next_load = 0;
        pp.next_mma = 0;
        pp.g_next = g_all;
        ok = tc_pump(sm, pp, min(kcs, 2 * TC_G));
        if (!ok) sm.abort = 1;
    }
#pragma unroll
    for (int v = 0; v < TC_B; ++v) s[v] = 0.0f;
    const uint32_t lane_base = ((uint32_t)(t >> 5) * 32u) << 16;
    for (int g = 0; g < ng; ++g) {
        const uint64_t gg = g_all + g;
        if (!tc::mbar_wait(&sm.accf[gg & 1u], (uint32_t)((gg >> 1) & 1u), TC_WAIT_BUDGET)) {
            ok = false;
            sm.abort = 1;
        }
        tc::tc_fence_after();
        const uint32_t col = sm.tmem + lane_base + tc_buf_col(gg);
#pragma unroll
        for (int c = 0; c < TC_B; c += 16) {
            float h[16], l[16];
            tc::tmem_ld16(col + c, h);
            tc::tmem_ld16(col + TC_B + c, l);
#pragma unroll
            for (int i = 0; i < 16; ++i) s[c + i] += fmaf(l[i], 1.0f / 2048.0f, h[i]);
        }
        tc::tc_fence_before();
        __syncthreads();  // the buffer of group g is free again
        if (sm.abort) break;
        if (t == 0) {
            tc::tc_fence_after();
            if (!tc_pump(sm, pp, min(kcs, (g + 3) * TC_G))) sm.abort = 1;
        }
    }
#pragma unroll
    for (int v = 0; v < TC_B; ++v) s[v] *= (1.0f / 4096.0f);
    g_all += ng;
    return ok && !sm.abort;
}

// Write this thread's 64 new y values (two FP16 slices) as row `t` of the Y tile of chunk kc.
__device__ __forceinline__ void tc_write_y(uint8_t* __restrict__ Ybuf, int kc, int t,
                                           const float (&y)[TC_B]) {
    uint8_t* hi = Ybuf + (size_t)kc * 2 * TC_YT_BYTES;
    uint8_t* lo = hi + TC_YT_BYTES;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        __align__(16) __half h[8], l[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const float v = y[8 * c + e];
            h[e] = __float2half_rn(v);
            l[e] = __float2half_rn((v - __half2float(h[e])) * 2048.0f);
        }
        const uint32_t off = tc::sw128_off(t, 8 * c);
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
    const uint8_t* Lt;     // split factor tiles
    int nrb;               // row blocks of the split factor
    uint8_t* Yscratch;     // per-CTA Y buffers
    int64_t ystride;       // bytes per CTA buffer
    int* status;
};

__device__ __forceinline__ double tc_logprod_value(double prod, int ex) {
    return prod > 0.0 ? log(prod) + (double)ex * 0.69314718055994530942 : -INFINITY;
}

// Shared set-up of the tensor-core kernels: barriers and TMEM.
__device__ __forceinline__ void tc_setup(TcSmem& sm) {
    const int t = threadIdx.x;
    if (t == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            tc::mbar_init(&sm.full[s], 1);
            tc::mbar_init(&sm.empty[s], 1);
        }
        tc::mbar_init(&sm.accf[0], 1);
        tc::mbar_init(&sm.accf[1], 1);
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

// After an aborted (timed-out) wait: let the copies and MMAs this CTA issued finish (bounded)
// before its shared memory and tensor memory are released.
__device__ __forceinline__ void tc_quiesce(TcSmem& sm, const TcPipe& pp) {
    if (threadIdx.x != 0 || !sm.abort) return;
    for (uint64_t q = pp.q_mma; q < pp.q_load; ++q)
        tc::mbar_wait(&sm.full[q % TC_STAGES], (uint32_t)((q / TC_STAGES) & 1u), TC_WAIT_BUDGET);
    tc::mma_commit(&sm.fin);
    tc::mbar_wait(&sm.fin, 0, TC_WAIT_BUDGET);
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

__device__ __forceinline__ int tri(int v, int u) { return v * (v + 1) / 2 + u; }

__global__ void __launch_bounds__(TC_P, 2) k_sov_tc(const TcBatch bt,
                                                     const uint64_t* __restrict__ alpha) {
    extern __shared__ uint8_t smem_raw[];
    TcSmem& sm = tc_smem(smem_raw);
    const int t = threadIdx.x;
    tc_setup(sm);
    TcPipe pp;
    uint64_t g_all = 0;  // groups issued so far (uniform across threads)
    uint8_t* Ybuf = bt.Yscratch + (int64_t)blockIdx.x * bt.ystride;

    for (;;) {
        if (t == 0) sm.item = atomicAdd(bt.counter, 1);
        __syncthreads();
        const int it = sm.item;
        if (it >= bt.nitems || sm.abort) break;
        const SovProblem& P = (bt.probs == nullptr) ? bt.single : bt.probs[bt.items[it].x];
        const int tile = (bt.probs == nullptr) ? it : bt.items[it].y;
        const int n = P.n;
        const int64_t p = (int64_t)tile * TC_P + t;
        const bool valid = p < P.Ntot;
        const int64_t q = valid ? p / P.Ns : 0;
        const uint64_t j = valid ? (uint64_t)(p - q * P.Ns) + 1u : 1u;
        const uint64_t* __restrict__ dq = P.delta + q * P.dstride;
        DFProd lp;
        int pf = 0;
        int next_k = (P.nprefix > 0) ? P.prefix[0] : -1;

        for (int r0 = 0; r0 < n; r0 += TC_B) {
            const int nb = min(TC_B, n - r0);
            const int rb = r0 / TC_B;
            float s[TC_B];
            if (rb > 0) {
                if (!tc_block_shift(sm, pp, Ybuf, bt.Lt, bt.nrb, rb, g_all, s)) {
                    if (t == 0) dev_raise(bt.status, MVN_ERR_TIMEOUT, 0);
                }
            } else {
#pragma unroll
                for (int v = 0; v < TC_B; ++v) s[v] = 0.0f;
            }
            __syncthreads();
            if (sm.abort) break;
            // diagonal block operands
            for (int e = t; e < TC_B * TC_B; e += TC_P) {
                const int v = e % TC_B, u = e / TC_B;
                if (u <= v)
                    sm.Ld[tri(v, u)] =
                        (v < nb) ? (float)P.L[(r0 + v) + (int64_t)(r0 + u) * P.ld] : 0.0f;
            }
            if (t < TC_B) {
                const double av = (t < nb) ? P.a[r0 + t] : 0.0;
                const double bv = (t < nb) ? P.b[r0 + t] : 1.0;
                sm.a[t] = av;
                sm.b[t] = bv;
                sm.af[t] = (float)av;
                sm.bf[t] = (float)bv;
                sm.ainf[t] = (av == -INFINITY);
                sm.binf[t] = (bv == INFINITY);
                sm.alpha[t] = (t < nb) ? alpha[r0 + t] : 0u;
            }
            __syncthreads();
            float y[TC_B];
#pragma unroll
            for (int v = 0; v < TC_B; ++v) {
                if (v < nb) {
                    float sv = s[v];
#pragma unroll
                    for (int u = 0; u < v; ++u) sv = fmaf(sm.Ld[tri(v, u)], y[u], sv);
                    float w, wc, dh, dl;
                    uint64_t wm;
                    int dex;
                    lattice_wf(j, sm.alpha[v], dq[r0 + v], w, wc, wm);
                    y[v] = sov_step_f32p(sm.af[v], sm.bf[v], sm.a[v], sm.b[v], sm.ainf[v],
                                         sm.binf[v], sv, sm.Ld[tri(v, v)], w, wc, wm, dh, dl, dex);
                    lp.mul(dh, dl, dex);
                    while (next_k == r0 + v + 1) {
                        if (valid) P.logw_prefix[(int64_t)pf * P.Ntot + p] = lp.log_value();
                        ++pf;
                        next_k = (pf < P.nprefix) ? P.prefix[pf] : -1;
                    }
                } else {
                    y[v] = 0.0f;
                }
            }
            // y of this block -> operand buffer of the later blocks (bulk-copied back by the
            // async proxy: fence before the barrier that precedes the next loads)
            if (r0 + TC_B < n) {
                tc_write_y(Ybuf, rb, t, y);
                tc::fence_proxy_async_global();
            }
            __syncthreads();
        }
        if (valid && P.logw) P.logw[p] = lp.log_value();
        __syncthreads();
    }
    tc_quiesce(sm, pp);
    tc_teardown(sm);
}

// ---------------------------------------------------------------- host side

static size_t tc_smem_bytes() { return sizeof(TcSmem) + 1024; }

static int tc_grid(mvn_ctx* ctx, int64_t ntiles) {
    // two CTAs per SM (shared memory ~106 KB, 256 TMEM columns each)
    return (int)std::max<int64_t>(1, std::min<int64_t>(ntiles, 2 * (int64_t)ctx->sm_count));
}

size_t sov_tc_ws_bytes(mvn_ctx* ctx, int nprob, int nmax, int64_t ntiles) {
    const int nrb = (std::max(nmax, 1) + TC_B - 1) / TC_B;
    size_t b = ws_round(sizeof(int));
    if (nprob > 1)
        b += ws_round(sizeof(SovProblem) * nprob) + ws_round(sizeof(int2) * (size_t)ntiles);
    b += ws_round((size_t)2 * nrb * nrb * TC_LT_BYTES);
    b += ws_round((size_t)tc_grid(ctx, ntiles) * nrb * 2 * TC_YT_BYTES);
    return b;
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
    const int nrb = (nmax + TC_B - 1) / TC_B;
    const int grid = tc_grid(ctx, ntiles);
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
    __half* Lt = wc.take<__half>((size_t)2 * nrb * nrb * TC_LT_BYTES / 2);
    bt.Lt = reinterpret_cast<const uint8_t*>(Lt);
    bt.nrb = nrb;
    bt.ystride = (int64_t)nrb * 2 * TC_YT_BYTES;
    bt.Yscratch = wc.take<uint8_t>((size_t)grid * bt.ystride);
    bt.status = ctx->d_status;
    // split the shared factor into FP16 operand tiles (lower tiles only)
    const SovProblem& P0 = probs_h[0];
    for (auto& P : probs_h)
        if (P.L != P0.L || P.ld != P0.ld)
            return mvn_fail(ctx, MVN_ERR_ARG, "tensor-core batch needs one shared factor");
    const int64_t ltiles = (int64_t)nrb * (nrb + 1) / 2;
    k_split_L<<<(unsigned)ltiles, 256, 0, ctx->stream>>>(nmax, P0.L, P0.ld, nrb, Lt);
    MVN_LAUNCHED(ctx);
    MVN_CUDA(ctx, cudaMemsetAsync(bt.counter, 0, sizeof(int), ctx->stream));
    const size_t smem = tc_smem_bytes();
    MVN_CUDA(ctx, cudaFuncSetAttribute(k_sov_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    MVN_TIMED(ctx, "k_sov_tc", (k_sov_tc<<<grid, TC_P, smem, ctx->stream>>>(bt, ctx->d_alpha)));
    return MVN_OK;
}

// ---------------------------------------------------------------- GEMM self-test

// S (128 x 64, row-major) = Y (128 x K) L (64 x K)^T through exactly the operand split, tile
// layout, bulk-copy pipeline, descriptors, MMAs and TMEM read of the SOV kernel.
__global__ void k_tc_selftest_prep(int K, const double* __restrict__ Y,
                                   const double* __restrict__ Lr, uint8_t* __restrict__ Ybuf,
                                   __half* __restrict__ Lt, int nrb) {
    // Y rows: one thread per path; L rows: tiles (rb = kcs, kc) of a factor whose row block kcs
    // holds the test rows
    const int t = threadIdx.x;
    for (int kc = 0; kc * TC_B < K; ++kc) {
        float y[TC_B];
#pragma unroll
        for (int v = 0; v < TC_B; ++v) {
            const int k = kc * TC_B + v;
            y[v] = (k < K) ? (float)Y[(int64_t)t * K + k] : 0.0f;
        }
        tc_write_y(Ybuf, kc, t, y);
    }
    const size_t slice = (size_t)nrb * nrb * (TC_LT_BYTES / 2);
    for (int kc = 0; kc * TC_B < K; ++kc) {
        const int rbt = (K + TC_B - 1) / TC_B;
        __half* hi = Lt + ((size_t)kc * nrb + rbt) * (TC_LT_BYTES / 2);
        __half* lo = hi + slice;
        for (int e = t; e < 64 * 64; e += blockDim.x) {
            const int r = e & 63, k = e >> 6;
            const int kk = kc * TC_B + k;
            double v = (kk < K) ? Lr[(int64_t)r * K + kk] * 4096.0 : 0.0;
            __half h = __double2half(v);
            __half l = __double2half((v - (double)__half2float(h)) * 2048.0);
            const uint32_t off = tc::sw128_off(r, k) >> 1;
            hi[off] = h;
            lo[off] = l;
        }
    }
    __syncthreads();
    tc::fence_proxy_async_global();
}

__global__ void __launch_bounds__(TC_P, 2) k_tc_selftest(int K, const uint8_t* __restrict__ Ybuf,
                                                          const uint8_t* __restrict__ Lt, int nrb,
                                                          float* __restrict__ S, int* status) {
    extern __shared__ uint8_t smem_raw[];
    TcSmem& sm = tc_smem(smem_raw);
    const int t = threadIdx.x;
    tc_setup(sm);
    TcPipe pp;
    uint64_t g_all = 0;
    float s[TC_B];
    const int kcs = (K + TC_B - 1) / TC_B;
    // row block kcs of a factor whose tiles (kcs, kc) hold the test rows: the block has kcs chunks
    const bool ok = tc_block_shift(sm, pp, Ybuf, Lt, nrb, kcs, g_all, s);
    if (!ok && t == 0) dev_raise(status, MVN_ERR_TIMEOUT, 0);
    if (ok)
        for (int v = 0; v < TC_B; ++v) S[t * TC_B + v] = s[v];
    tc_quiesce(sm, pp);
    tc_teardown(sm);
}

extern "C" mvn_status mvn_tc_selftest(mvn_ctx* ctx, int K, const double* Y, const double* L,
                                      float* S) {
    if (!ctx) return MVN_ERR_ARG;
    if (K < 1 || K > 65536 || !Y || !L || !S)
        return mvn_fail(ctx, MVN_ERR_ARG, "mvn_tc_selftest: invalid argument");
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    const int kcs = (K + TC_B - 1) / TC_B;
    const int nrb = kcs + 1;
    const size_t ybytes = (size_t)kcs * 2 * TC_YT_BYTES;
    const size_t lbytes = (size_t)2 * nrb * nrb * TC_LT_BYTES;
    MVN_TRY(ws_reserve(ctx, ws_round(ybytes) + ws_round(lbytes) + 1024));
    WsCarver wc(ctx->ws);
    uint8_t* Ybuf = wc.take<uint8_t>(ybytes);
    __half* Lt = wc.take<__half>(lbytes / 2);
    k_tc_selftest_prep<<<1, TC_P, 0, ctx->stream>>>(K, Y, L, Ybuf, Lt, nrb);
    MVN_LAUNCHED(ctx);
    const size_t smem = tc_smem_bytes();
    MVN_CUDA(ctx, cudaFuncSetAttribute(k_tc_selftest, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem));
    k_tc_selftest<<<1, TC_P, smem, ctx->stream>>>(K, Ybuf, reinterpret_cast<const uint8_t*>(Lt),
                                                  nrb, S, ctx->d_status);
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
