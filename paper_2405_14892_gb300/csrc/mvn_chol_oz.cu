// mvn_chol_oz.cu -- tile Cholesky (Alg. 1 "dpotrf") whose trailing updates run on the tcgen05
// tensor cores with 42-bit products (the MVN_MIXED factorisation).
//
// The SOV estimate needs an FP64-accurate factor (an FP32 factor moves log P by ~1e-2 at
// n = 16,384), and GB300's FP64 units deliver ~1.25 TFLOP/s.  The update L(i,:) L(j,:)^T of the
// left-looking algorithm is therefore computed exactly from small-integer digits on the BF16
// tensor cores (the error-free splitting of Ozaki, Ogita, Oishi and Rump, 2012):
//   - every row i of L is scaled by 2^-E_i with 2^E_i > sqrt(Sigma_ii) >= |L_ik| (fixed before the
//     factorisation, since sum_k L_ik^2 = Sigma_ii), so x_ik = L_ik 2^-E_i lies in (-1, 1);
//   - x_ik is rounded once to v_ik = rint(x_ik 2^42) and written as six balanced 7-bit digits,
//     x_ik ~ sum_{s<6} a^(s)_ik 2^(-7(s+1)), |a^(0)| <= 128, |a^(s>0)| <= 64, exact in BF16;
//   - the digit products of one level l = s + t (l <= 5) share a TMEM accumulator; a level has at
//     most two products with a leading digit (<= 128 x 64 each) and four others (<= 64 x 64),
//     i.e. at most 2^15 per value of k, so over 384 values of k its sum is an integer below
//     12.6e6 < 2^24 and the tensor core's FP32 accumulation is exact;
//   - every 384 values of k the six level sums are drained into a 64-bit integer
//     T = sum_l V_l 2^(7(5-l)) (the product in units of 2^-49), which stays exact; split-K
//     partial sums are added with integer atomics (exact and order-independent), and the POTRF
//     and TRSM kernels apply C_ij -= 2^(E_i+E_j-49) T_ij in FP64 as they load their block.
// The products thus carry 42 bits relative to |L_i||L_j| (row maxima), against 24 for FP32.
// The diagonal block (POTRF), the panel solve (TRSM) and the digit split run on the CUDA cores.
//
// The update of block column j (64 columns) is an M = 128 (row tile) x N = 64 x K = 64 j GEMM
// per row tile.  Its K range is cut into work items that a persistent grid of one CTA per SM
// walks; inside a CTA one warp streams digit tiles (1-D bulk copies, 2-stage mbarrier ring), one
// warp issues the MMAs (a row digit times 4, 2 or 1 adjacent block-column digits per MMA of
// N = 256, 128 or 64: the issuing thread, not the tensor pipe, sets the pace), and eight warps
// drain TMEM into the integer accumulators.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "mvn_internal.cuh"
#include "mvn_tc.cuh"

#define OZ_NB 64            // block column width
#define OZ_RT 128           // row tile height (MMA M)
#define OZ_S 6              // digits per value
#define OZ_AT 8192          // one digit tile: 128 rows x 32 K, BF16, 64-byte swizzle
#define OZ_BT 4096          // 64 rows of such a tile (the B operand)
#define OZ_STAGE (OZ_S * (OZ_AT + OZ_BT))
#define OZ_NST 2            // pipeline stages (K = 32 each, 72 KB; measured: a third stage does
                            // not speed the W2 factorisation up)
#define OZ_GRP 12           // stages accumulated in TMEM between drains (K = 384)
#define OZ_DW 8             // drain warps
#define OZ_THREADS (32 * (OZ_DW + 2))
#define OZ_WAIT 4000000000LL
// K sub-chunks per work item of the bulk and tail updates: TuneParams (default 16 and 2; short
// CTAs, so that the chain kernels get SMs as they retire)

__device__ __forceinline__ bool oz_failed(const int* status) {
    return *(volatile const int*)status != 0;
}

// Digit tile of sub-chunk kc (columns 32 kc .. 32 kc + 31), digit s, row tile rt.
__host__ __device__ __forceinline__ size_t oz_tile(int kc, int s, int rt, int nrt) {
    return (((size_t)kc * OZ_S + s) * nrt + rt) * OZ_AT;
}

// Bounded wait that also gives up as soon as another role of the CTA has aborted.
__device__ __forceinline__ bool oz_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
    if (tc::mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!tc::mbar_try_wait(bar, parity)) {
        if (*abort_flag || clock64() - t0 > OZ_WAIT) return false;
    }
    return true;
}

// 2^k as a double for |k| < 1000 (exact; no FP64 arithmetic)
__device__ __forceinline__ double oz_pow2(int k) {
    return __longlong_as_double((long long)(1023 + k) << 52);
}

__global__ void k_oz_exps(int n, const double* __restrict__ A, int64_t ld, int* __restrict__ E) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double d = A[i + (int64_t)i * ld];
    int e = 0;
    if (d > 0.0) {
        frexp(sqrt(d), &e);  // sqrt(d) = m 2^e with m in [0.5, 1): 2^e > sqrt(d)
    }
    E[i] = e;
}

// rint(x 2^sh) as a 64-bit integer from the bits of an FP32 value (integer ALU only; GB300's
// FP64 pipe is narrow).  Requires |x 2^sh| < 2^62; ties round away from zero.
__device__ __forceinline__ long long oz_f2fix(float x, int sh) {
    const uint32_t b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 255u);
    if (e == 0) return 0;  // zero (FP32 subnormals lie far below 2^-42 of any row here)
    const long long m = (long long)((b & 0x7fffffu) | 0x800000u);  // x = m 2^(e - 150)
    const int s2 = e - 150 + sh;
    long long v;
    if (s2 >= 0)
        v = m << s2;
    else if (s2 < -25)
        v = 0;
    else
        v = (m + (1ll << (-s2 - 1))) >> (-s2);
    return (b >> 31) ? -v : v;
}

// Digits of 8 consecutive entries x = hi + lo (double-float) of row i of the finished factor
// (one 16-byte chunk of a 64-byte swizzled tile row per digit): v = rint(hi 2^(42 - E_i)) +
// rint(lo 2^(42 - E_i)) (the value in 42-bit fixed point, to one unit), then balanced 7-bit digits
// peeled off with integer shifts: d = (v + 2^(k-1)) >> k, v -= d 2^k.  Zero entries (above the
// diagonal, beyond n) give zero digits.
__device__ __forceinline__ void oz_digits8(const float (&xh)[8], const float (&xl)[8], int ei,
                                           uint4 (&out)[OZ_S]) {
    uint32_t pk[OZ_S][4];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        long long v = oz_f2fix(xh[e], 42 - ei) + oz_f2fix(xl[e], 42 - ei);
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) {
            const int sh = 7 * (OZ_S - 1 - s);
            const long long d = (sh > 0) ? ((v + (1ll << (sh - 1))) >> sh) : v;
            v -= d * (1ll << sh);
            const uint32_t b = (uint32_t)__bfloat16_as_ushort(__int2bfloat16_rn((int)d));
            if (e & 1)
                pk[s][e >> 1] |= b << 16;
            else
                pk[s][e >> 1] = b;
        }
    }
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) out[s] = make_uint4(pk[s][0], pk[s][1], pk[s][2], pk[s][3]);
}

// Store the digits of row r (global row index), columns c0 + 8 c8 .. of block column j (c0 =
// 64 j) into the digit tiles of sub-chunk 2 j + c8 / 4.
__device__ __forceinline__ void oz_store_digits(uint8_t* __restrict__ Z, int nrt, int j, int r,
                                                int c8, const uint4 (&dg)[OZ_S]) {
    const int rt = r / OZ_RT, rr = r % OZ_RT;
    const int kc = 2 * j + (c8 >> 2);
    const uint32_t off = tc::sw64_off((uint32_t)rr, (uint32_t)(8 * (c8 & 3)));
#pragma unroll
    for (int s = 0; s < OZ_S; ++s) *reinterpret_cast<uint4*>(Z + oz_tile(kc, s, rt, nrt) + off) = dg[s];
}

struct __align__(1024) OzSmem {
    uint8_t stage[OZ_NST][OZ_STAGE];  // per stage: A digits [S][8 KB], then B digits [S][4 KB]
    uint64_t full[OZ_NST], empty[OZ_NST], accf, drained, fin;
    uint32_t tmem;
    int abort;
};

// Work of one update launch: row tiles rt0 .. rt0+n_rt-1 of block column j, K sub-chunks
// [kc0, kc1) cut into pieces of P.  Item it = piece (it / n_rt), row tile rt0 + it % n_rt, so
// CTAs running at the same time read the same B tiles.
struct OzWork {
    int n, j, nrt, rt0, n_rt, kc0, kc1, P, n_items;
    int64_t ldT;
};
__device__ __forceinline__ void oz_item(const OzWork& w, int it, int& rt, int& ka, int& kb) {
    const int p = it / w.n_rt;
    rt = w.rt0 + (it - p * w.n_rt);
    ka = w.kc0 + p * w.P;
    kb = min(ka + w.P, w.kc1);
}

// Left-looking update of block column j: T(i, c) += sum_k (digit products), exact, for rows i of
// the row tiles and columns c0 .. c0+63.  320 threads: warps 0-7 drain and accumulate (warp w:
// TMEM lanes 32 (w % 4).., columns 32 (w / 4)..), warp 8 loads, warp 9 issues the MMAs.
__global__ void __launch_bounds__(OZ_THREADS, 1) k_oz_update(const OzWork w,
                                                               const uint8_t* __restrict__ Z,
                                                               const int* __restrict__ E,
                                                               long long* __restrict__ T,
                                                               int* __restrict__ status) {
    extern __shared__ uint8_t smem_raw[];
    OzSmem& sm = *reinterpret_cast<OzSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                            ~(uintptr_t)1023);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int c0 = w.j * OZ_NB;
    if (t == 0) {
        sm.abort = oz_failed(status) ? 1 : 0;  // one reading of the status for the whole CTA
        for (int q = 0; q < OZ_NST; ++q) {
            tc::mbar_init(&sm.full[q], 1);
            tc::mbar_init(&sm.empty[q], 1);
        }
        tc::mbar_init(&sm.accf, 1);
        tc::mbar_init(&sm.drained, 32 * OZ_DW);
        tc::mbar_init(&sm.fin, 1);
        tc::mbar_fence_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(&sm.tmem, 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    volatile int* abort_flag = &sm.abort;

    if (warp == OZ_DW) {
        // ---------------------------------------------------------------- producer
        if (lane == 0) {
            const int rtj = c0 / OZ_RT, hb = (c0 % OZ_RT) / OZ_NB;
            uint32_t q = 0;
            for (int it = blockIdx.x; it < w.n_items && !*abort_flag; it += gridDim.x) {
                int rt, ka, kb;
                oz_item(w, it, rt, ka, kb);
                for (int kc = ka; kc < kb; ++kc, ++q) {
                    const int slot = (int)(q % OZ_NST);
                    if (q >= OZ_NST &&
                        !oz_wait(&sm.empty[slot], ((q / OZ_NST) - 1) & 1u, abort_flag)) {
                        dev_raise(status, MVN_ERR_TIMEOUT, 0);
                        *abort_flag = 1;
                        break;
                    }
                    uint8_t* st = sm.stage[slot];
                    tc::mbar_arrive_expect_tx(&sm.full[slot], OZ_STAGE);
                    for (int s = 0; s < OZ_S; ++s)
                        tc::bulk_g2s(st + s * OZ_AT, Z + oz_tile(kc, s, rt, w.nrt), OZ_AT,
                                     &sm.full[slot]);
                    for (int s = 0; s < OZ_S; ++s)
                        tc::bulk_g2s(st + OZ_S * OZ_AT + s * OZ_BT,
                                     Z + oz_tile(kc, s, rtj, w.nrt) + hb * OZ_BT, OZ_BT,
                                     &sm.full[slot]);
                }
            }
            // every issued copy has landed before the shared memory is released (a wait that
            // runs out here leaves the result unreliable: it raises the status too)
            for (uint32_t k = (q > OZ_NST ? q - OZ_NST : 0); k < q; ++k)
                if (!tc::mbar_wait(&sm.full[k % OZ_NST], (k / OZ_NST) & 1u, OZ_WAIT))
                    dev_raise(status, MVN_ERR_TIMEOUT, 0);
        }
    } else if (warp == OZ_DW + 1) {
        // ---------------------------------------------------------------- MMA issue
        if (lane == 0) {
            // digits u .. u + c - 1 of the block column are adjacent 64-row B tiles and levels
            // s + u .. s + u + c - 1 adjacent 64-column accumulators, so one MMA of N = 64 c forms
            // c products; the 6 - s products of digit s of the rows go in chunks of 4, 2, 1
            // (9 MMAs per 16 K instead of 21; the issuing thread pays per instruction)
            auto idesc_n = [](int nc) {
                return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((nc * OZ_NB) >> 3) << 17) |
                       ((uint32_t)(OZ_RT >> 4) << 24);
            };
            uint32_t q = 0, g = 0;
            bool ok = true;
            for (int it = blockIdx.x; it < w.n_items && ok; it += gridDim.x) {
                int rt, ka, kb;
                oz_item(w, it, rt, ka, kb);
                for (int k0 = ka; k0 < kb && ok; k0 += OZ_GRP, ++g) {
                    if (*abort_flag || (g > 0 && !oz_wait(&sm.drained, (g - 1) & 1u, abort_flag))) {
                        ok = false;
                        break;
                    }
                    tc::tc_fence_after();
                    const int k1 = min(k0 + OZ_GRP, kb);
                    for (int kc = k0; kc < k1; ++kc, ++q) {
                        const int slot = (int)(q % OZ_NST);
                        if (!oz_wait(&sm.full[slot], (q / OZ_NST) & 1u, abort_flag)) {
                            ok = false;
                            break;
                        }
                        tc::tc_fence_after();
                        const uint32_t base = tc::smem_u32(sm.stage[slot]);
#pragma unroll
                        for (int s = 0; s < OZ_S; ++s) {
#pragma unroll
                            for (int u = 0; u + s < OZ_S;) {
                                const int left = OZ_S - s - u;
                                const int nc = left >= 4 ? 4 : (left >= 2 ? 2 : 1);
                                const uint32_t dcol = sm.tmem + (uint32_t)(s + u) * OZ_NB;
#pragma unroll
                                for (int k16 = 0; k16 < 2; ++k16) {
                                    const uint64_t ad =
                                        tc::sdesc_sw64(base + s * OZ_AT + k16 * 32);
                                    const uint64_t bd = tc::sdesc_sw64(
                                        base + OZ_S * OZ_AT + u * OZ_BT + k16 * 32);
                                    const uint32_t acc =
                                        (kc == k0 && s == 0 && k16 == 0) ? 0u : 1u;
                                    tc::mma_f16(dcol, ad, bd, idesc_n(nc), acc);
                                }
                                u += nc;
                            }
                        }
                        tc::mma_commit(&sm.empty[slot]);
                    }
                    if (ok) tc::mma_commit(&sm.accf);
                }
            }
            if (!ok) {
                dev_raise(status, MVN_ERR_TIMEOUT, 0);
                *abort_flag = 1;
            }
            // all issued MMAs complete before TMEM and shared memory are released
            tc::mma_commit(&sm.fin);
            if (!tc::mbar_wait(&sm.fin, 0, OZ_WAIT)) dev_raise(status, MVN_ERR_TIMEOUT, 0);
        }
    } else {
        // ---------------------------------------------------------------- drain + epilogue
        const int quarter = warp & 3, chalf = warp >> 2;
        const uint32_t taddr = sm.tmem + (((uint32_t)quarter * 32u) << 16) + (uint32_t)chalf * 32u;
        long long acc[32];
#pragma unroll
        for (int c = 0; c < 32; ++c) acc[c] = 0;
        uint32_t g = 0;
        bool ok = true;
        for (int it = blockIdx.x; it < w.n_items && ok; it += gridDim.x) {
            int rt, ka, kb;
            oz_item(w, it, rt, ka, kb);
            for (int k0 = ka; k0 < kb; k0 += OZ_GRP, ++g) {
                if (*abort_flag || !oz_wait(&sm.accf, g & 1u, abort_flag)) {
                    ok = false;
                    break;
                }
                tc::tc_fence_after();
#pragma unroll
                for (int l = 0; l < OZ_S; ++l) {
                    float v[32];
                    tc::tmem_ld32(taddr + (uint32_t)l * OZ_NB, v);
                    const long long sc = 1ll << (7 * (OZ_S - 1 - l));
#pragma unroll
                    for (int c = 0; c < 32; ++c) acc[c] += (long long)__float2int_rn(v[c]) * sc;
                }
                tc::tc_fence_before();
                asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(
                                 tc::smem_u32(&sm.drained))
                             : "memory");
            }
            if (!ok) break;
            const int i = rt * OZ_RT + quarter * 32 + lane;
            if (i < w.n && i >= c0) {
#pragma unroll
                for (int c = 0; c < 32; ++c) {
                    const int cc = chalf * 32 + c;
                    const int col = c0 + cc;
                    if (col <= i && col < w.n && acc[c] != 0)
                        atomicAdd(reinterpret_cast<unsigned long long*>(T + i + cc * w.ldT),
                                  (unsigned long long)acc[c]);
                }
            }
#pragma unroll
            for (int c = 0; c < 32; ++c) acc[c] = 0;
        }
        if (!ok) {
            dev_raise(status, MVN_ERR_TIMEOUT, 0);
            *abort_flag = 1;
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(sm.tmem, 512);
    }
}


// Double-float (FP32 pair) arithmetic: x = hi + lo with |lo| <= ulp(hi) / 2 (Dekker 1971;
// Knuth's two-sum).  GB300 runs FP32 at 64 times its FP64 rate and FP64 division and square root
// are long dependent sequences, so the panel (POTRF, triangular inverse, TRSM) runs on pairs:
// ~48 bits, beyond the 42 bits the digit products keep.
struct DF {
    float hi, lo;
};
__device__ __forceinline__ DF df_from(double x) {
    const float h = __double2float_rn(x);
    return DF{h, __double2float_rn(x - (double)h)};
}
__device__ __forceinline__ double df_to(DF a) { return (double)a.hi + (double)a.lo; }
__device__ __forceinline__ DF df_norm(float h, float l) {
    const float s = h + l;
    return DF{s, l - (s - h)};
}
// s += a * b, with s kept unnormalised (s.lo collects the rounding errors; normalise at the end)
__device__ __forceinline__ void df_fma_acc(DF& s, DF a, DF b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    const float t = s.hi + p;
    const float bp = t - s.hi;
    s.lo += ((s.hi - (t - bp)) + (p - bp)) + e;
    s.hi = t;
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return df_norm(p, e);
}
// Square root and reciprocal of the pivot, on the POTRF's serial path: the hardware
// approximations (relative error ~2^-22), one Newton-Raphson step in FP32 (Markstein 1990),
// then one Newton correction in double-float with the residual formed exactly by FMA (Dekker
// 1971): ~2^-45 relative, beyond the 42 bits the digit products keep, without the special-case
// branches of the IEEE square root and division.
// sqrt: y ~ 1/sqrt(d.hi) refined by y (3 - d y^2) / 2, s0 = d.hi y, then s0 + (d - s0^2) y / 2
__device__ __forceinline__ DF df_sqrt(DF d) {
    float y;
    asm("rsqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(d.hi));
    y = y * fmaf(-0.5f * d.hi * y, y, 1.5f);
    const float s0 = d.hi * y;
    const float p = s0 * s0;
    const float pe = fmaf(s0, s0, -p);
    const float diff = ((d.hi - p) - pe) + d.lo;
    return df_norm(s0, diff * (0.5f * y));
}
// reciprocal: r ~ 1/l.hi refined by r + r (1 - l.hi r), then r0 (1 + (1 - l r0))
__device__ __forceinline__ DF df_rcp(DF l) {
    float r0;
    asm("rcp.approx.f32 %0, %1;" : "=f"(r0) : "f"(l.hi));
    r0 = fmaf(r0, fmaf(-l.hi, r0, 1.0f), r0);
    const float p = l.hi * r0;
    const float pe = fmaf(l.hi, r0, -p);
    const float res = ((1.0f - p) - pe) - l.lo * r0;
    return df_norm(r0, r0 * res);
}

// POTRF of the diagonal block (c0, c0), nb <= 64, after applying the update, and the inverse
// W = L_jj^-1 for the panel solve (double-float).  The 64 x 64 block is cut into 2 x 4 blocks
// (rows 2 ty .., columns 4 tx ..); the 272 of them that reach the lower triangle (4 tx <= 2 ty + 1)
// go one per thread, packed densely in row-major order (row pair p, i.e. ty = 2p and 2p + 1, holds
// 2 (p + 1) blocks starting at block p (p + 1)), so that no warp issues for the empty upper half.
// Each thread keeps its block X in registers (8 double-float updates per step).
// One array carries both factors: at step k of the right-looking sweep the columns m > k of X
// hold the Schur complement S, the columns m <= k hold W (the column-oriented forward
// substitution L W = I riding along), so the two updates of step k are one symmetric rank-1
// update of the rows i > k:
//     X(i, m) -= V(i) V(m),   V(m) = L(m, k) for m > k,  V(m) = W(k, m) for m <= k,
// where W(k, m) = X(k, m) / L_kk (m < k) and W(k, k) = 1 / L_kk; column k itself is zeroed by
// its owners before the update (W(i, k) = -L(i, k) W(k, k)).  Columns of L leave the array as
// they are finished (staged in shared memory).  Rows and columns beyond nb are the identity and
// are never touched.  Writes L_jj to A (FP64), W^T as pairs Wt[u][c] = W[c][u], and the digits of
// the diagonal rows.
#define OZ_PF_BLOCKS 272   // 2 x 4 blocks of a 64 x 64 block that reach its lower triangle
#define OZ_PF_THREADS 288  // whole warps
__global__ void __launch_bounds__(OZ_PF_THREADS) k_oz_potrf(double* __restrict__ A, int64_t ld,
                                                           int c0, int nb,
                                                           const int* __restrict__ E,
                                                           long long* __restrict__ T, int64_t ldT,
                                                           float* __restrict__ Wt,
                                                           uint8_t* __restrict__ Z, int nrt,
                                                           int* status) {
    __shared__ DF Vs[2][OZ_NB];  // step vector V, by step parity
    __shared__ DF Sdp[2];        // S(k, k) published one step ahead, by step parity
    // staging: the loaded block, then the columns of L as they are finished
    __shared__ float Sh[OZ_NB][OZ_NB + 1], Sl[OZ_NB][OZ_NB + 1];
    __shared__ int Eb[OZ_NB];
    if (oz_failed(status)) return;
    const int t = threadIdx.x;
    const bool act = (t < OZ_PF_BLOCKS);
    int ty = 0, tx = 0;  // idle threads (act false) take part in the loads, barriers and stores only
    if (act) {
        int p = 0;
        while ((p + 1) * (p + 2) <= t) ++p;
        const int q = t - p * (p + 1);
        ty = 2 * p + (q > p ? 1 : 0);
        tx = (q > p) ? q - p - 1 : q;
    }
    if (t < OZ_NB) {
        Eb[t] = (t < nb) ? E[c0 + t] : 0;
        Vs[1][t] = DF{0.0f, 0.0f};  // the vector "before step 0": the first update is empty
    }
    __syncthreads();
    {
        // all loads first (independent), then the update is applied
        constexpr int NL = (OZ_NB * OZ_NB + OZ_PF_THREADS - 1) / OZ_PF_THREADS;
        double av[NL];
        long long tv[NL];
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int e = t + OZ_PF_THREADS * k, i = e % OZ_NB, m = e / OZ_NB;
            const bool in = (e < OZ_NB * OZ_NB && i < nb && m <= i);
            av[k] = in ? A[(c0 + i) + (int64_t)(c0 + m) * ld] : 0.0;
            tv[k] = in ? T[(c0 + i) + (int64_t)m * ldT] : 0;
        }
#pragma unroll
        for (int k = 0; k < NL; ++k) {
            const int e = t + OZ_PF_THREADS * k, i = e % OZ_NB, m = e / OZ_NB;
            if (e >= OZ_NB * OZ_NB) continue;
            DF v{0.0f, 0.0f};
            if (i < nb && m <= i) {
                double a = av[k];
                if (tv[k] != 0) {
                    a -= (double)tv[k] * oz_pow2(Eb[i] + Eb[m] - 49);
                    T[(c0 + i) + (int64_t)m * ldT] = 0;
                }
                v = df_from(a);
            } else if (i == m) {
                v = DF{1.0f, 0.0f};
            }
            Sh[i][m] = v.hi;
            Sl[i][m] = v.lo;
        }
    }
    __syncthreads();
    DF X[2][4];  // this thread's block: lower entries of S, becoming W; upper entries unused
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int i = 2 * ty + a, m = 4 * tx + b;
            X[a][b] = (act && m <= i) ? DF{Sh[i][m], Sl[i][m]} : DF{0.0f, 0.0f};
        }
    if (t == 0) Sdp[0] = DF{Sh[0][0], Sl[0][0]};
    __syncthreads();  // Sh/Sl now receive the finished columns of L
    // Step k runs in one phase between two barriers: the rank-1 update of step k - 1, then the
    // scaling of column k (and of row k of W).  Every thread with a row i > k - 1 computes the
    // pivot itself, from S(k, k) as its owner published it one phase ahead (in Sdp, after the
    // update of step k - 2) with the last update -V(k) V(k) redone by the owner's exact
    // operations, so that every copy is the same; the pivot does not depend on this phase's
    // update, so the two dependency chains interleave in one straight-line block.
    for (int k = 0; k < nb; ++k) {
        const int kb = k >> 2, kk = k & 3;  // column block and column of k
        const int kr = k >> 1, ka = k & 1;  // row block and row of k
        DF* V = Vs[k & 1];
        const DF* Vp = Vs[(k + 1) & 1];  // the vector of step k - 1 (zero before step 0)
        int bad = 0;
        if (act && 2 * ty + 1 > k - 1) {
            // pivot L_kk = sqrt(S_kk) and its reciprocal
            DF d = Sdp[k & 1];
            const DF vk = Vp[k];
            df_fma_acc(d, DF{-vk.hi, -vk.lo}, vk);
            d = df_norm(d.hi, d.lo);
            const bool pos = (d.hi > 0.0f);
            const DF l = df_sqrt(pos ? d : DF{1.0f, 0.0f});
            const DF r = df_rcp(l);
            // rank-1 update of step k - 1; rows <= k - 1 take an exact zero multiplier
            DF vi[2], vm[4];
#pragma unroll
            for (int a = 0; a < 2; ++a) vi[a] = Vp[2 * ty + a];
#pragma unroll
            for (int b = 0; b < 4; ++b) vm[b] = Vp[4 * tx + b];
#pragma unroll
            for (int a = 0; a < 2; ++a) {
                const bool row = (2 * ty + a > k - 1);
                const DF nv{row ? -vi[a].hi : 0.0f, row ? -vi[a].lo : 0.0f};
#pragma unroll
                for (int b = 0; b < 4; ++b) df_fma_acc(X[a][b], nv, vm[b]);
            }
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) X[a][b] = df_norm(X[a][b].hi, X[a][b].lo);
            // the owner of (k + 1, k + 1) publishes it for the pivot of step k + 1
            const int k1 = k + 1;
            if (k1 < nb && ty == (k1 >> 1) && tx == (k1 >> 2)) {
                const int qr = k1 & 1, qc = k1 & 3;
                DF v = X[0][0];
#pragma unroll
                for (int a = 0; a < 2; ++a)
#pragma unroll
                    for (int b = 0; b < 4; ++b)
                        if (a == qr && b == qc) v = X[a][b];
                Sdp[k1 & 1] = v;
            }
            if (!pos) {
                bad = 1;
                dev_raise(status, MVN_ERR_NOT_PD, c0 + k + 1);
            } else {
                // X(k, k) becomes W(k, k) = 1 / L_kk
                if (ty == kr && tx == kb) {
                    V[k] = r;
                    Sh[k][k] = l.hi;
                    Sl[k][k] = l.lo;
#pragma unroll
                    for (int a = 0; a < 2; ++a)
#pragma unroll
                        for (int b = 0; b < 4; ++b)
                            if (a == ka && b == kk) X[a][b] = r;
                }
                // column k below the pivot: L(i, k) = S(i, k) / L_kk leaves the array (entry
                // zeroed); the entry is selected first, then scaled once
                if (tx == kb && 2 * ty + 1 > k) {
#pragma unroll
                    for (int a = 0; a < 2; ++a) {
                        const int i = 2 * ty + a;
                        DF x = X[a][0];
#pragma unroll
                        for (int b = 1; b < 4; ++b)
                            if (b == kk) x = X[a][b];
                        if (i > k) {
                            const DF v = df_mul(x, r);
#pragma unroll
                            for (int b = 0; b < 4; ++b)
                                if (b == kk) X[a][b] = DF{0.0f, 0.0f};
                            V[i] = v;
                            Sh[i][k] = v.hi;
                            Sl[i][k] = v.lo;
                        }
                    }
                }
                // row k left of the pivot: W(k, c) = X(k, c) / L_kk, final
                if (ty == kr && 4 * tx < k) {
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const int c = 4 * tx + b;
                        const DF x = ka ? X[1][b] : X[0][b];
                        if (c < k) {
                            const DF v = df_mul(x, r);
                            if (ka)
                                X[1][b] = v;
                            else
                                X[0][b] = v;
                            V[c] = v;
                        }
                    }
                }
            }
        }
        // this step's vector, pivot copy and columns become visible; the buffers of the other
        // parity are rewritten next phase, after every thread has read them in this one
        if (__syncthreads_or(bad)) return;
    }
    // W^T (X holds W in its lower entries; rows and columns beyond nb are the identity)
    if (act) {
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const int i = 2 * ty + a, m = 4 * tx + b;
                DF w = (m < i) ? X[a][b] : DF{0.0f, 0.0f};
                if (m == i) w = (i < nb) ? X[a][b] : DF{1.0f, 0.0f};
                Wt[m * OZ_NB + i] = w.hi;
                Wt[OZ_NB * OZ_NB + m * OZ_NB + i] = w.lo;
            }
    }
    // the blocks that no thread holds (above the diagonal) are zero in W^T
    for (int e = t; e < OZ_NB * OZ_NB; e += OZ_PF_THREADS) {
        const int i = e % OZ_NB, m = e / OZ_NB;
        if (4 * (m >> 2) > 2 * (i >> 1) + 1) {
            Wt[m * OZ_NB + i] = 0.0f;
            Wt[OZ_NB * OZ_NB + m * OZ_NB + i] = 0.0f;
        }
    }
    __syncthreads();
    for (int e = t; e < OZ_NB * OZ_NB; e += OZ_PF_THREADS) {
        const int i = e % OZ_NB, m = e / OZ_NB;
        if (m <= i && i < nb)
            A[(c0 + i) + (int64_t)(c0 + m) * ld] = df_to(DF{Sh[i][m], Sl[i][m]});
    }
    // digits of the diagonal rows (and zero digits for the rows of the row tile above them)
    if (Z != nullptr) {
        for (int e = t; e < 2 * OZ_NB * 8; e += OZ_PF_THREADS) {
            const int c8 = e & 7, i = (e >> 3) - ((c0 % OZ_RT) ? OZ_NB : 0);
            if (i >= OZ_NB) continue;
            float xh[8], xl[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const int m = 8 * c8 + q;
                const bool in = (i >= 0 && i < nb && m <= i);
                xh[q] = in ? Sh[i][m] : 0.0f;
                xl[q] = in ? Sl[i][m] : 0.0f;
            }
            uint4 dg[OZ_S];
            oz_digits8(xh, xl, (i >= 0) ? Eb[i] : 0, dg);
            oz_store_digits(Z, nrt, c0 / OZ_NB, c0 + i, c8, dg);
        }
    }
}

// Panel solve X = C(i, c0:c0+64) L_jj^-T = C W^T for the rows i >= c0 + nb below the diagonal
// block, after applying the update: a double-float GEMM.  CTA = 16 rows x 64 columns, 256
// threads, each 1 row x 4 columns; C and W^T staged in shared memory as pairs.
#define OZ_TR_ROWS 16                // rows per CTA: short CTAs, the chain waits on the last
#define OZ_TR_RPT (OZ_TR_ROWS / 16)  // rows per thread
__global__ void __launch_bounds__(256) k_oz_trsm(double* __restrict__ A, int64_t ld, int c0,
                                                 int nb, int n, const int* __restrict__ E,
                                                 long long* __restrict__ T, int64_t ldT,
                                                 const float* __restrict__ Wt,
                                                 uint8_t* __restrict__ Z, int nrt,
                                                 const int* status) {
    extern __shared__ float4 tr_raw[];  // Bh, Bl [NB][ROWS], Wh, Wl [NB][NB] (64 KB)
    float(*Bh)[OZ_TR_ROWS] = reinterpret_cast<float(*)[OZ_TR_ROWS]>(tr_raw);
    float(*Bl)[OZ_TR_ROWS] = Bh + OZ_NB;
    float(*Wh)[OZ_NB] = reinterpret_cast<float(*)[OZ_NB]>(Bl + OZ_NB);
    float(*Wl)[OZ_NB] = Wh + OZ_NB;
    __shared__ int Ec[OZ_NB];
    if (oz_failed(status)) return;
    const int t = threadIdx.x;
    const int r0 = c0 + nb + blockIdx.x * OZ_TR_ROWS;
    if (t < OZ_NB) Ec[t] = (t < nb) ? E[c0 + t] : 0;
    for (int e = t; e < OZ_NB * OZ_NB; e += 256) {
        Wh[e / OZ_NB][e % OZ_NB] = Wt[e];
        Wl[e / OZ_NB][e % OZ_NB] = Wt[OZ_NB * OZ_NB + e];
    }
    __syncthreads();
    {
        // all loads first (16 per thread, independent), then the update is applied
        constexpr int PER = OZ_NB * OZ_TR_ROWS / 256;
        double av[PER];
        long long tv[PER];
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = t + 256 * k, rr = e % OZ_TR_ROWS, u = e / OZ_TR_ROWS;
            const int r = r0 + rr;
            const bool in = (r < n && u < nb);
            av[k] = in ? A[r + (int64_t)(c0 + u) * ld] : 0.0;
            tv[k] = in ? T[r + (int64_t)u * ldT] : 0;
        }
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            const int e = t + 256 * k, rr = e % OZ_TR_ROWS, u = e / OZ_TR_ROWS;
            const int r = r0 + rr;
            DF v{0.0f, 0.0f};
            if (r < n && u < nb) {
                double a = av[k];
                if (tv[k] != 0) {
                    a -= (double)tv[k] * oz_pow2(E[r] + Ec[u] - 49);
                    T[r + (int64_t)u * ldT] = 0;
                }
                v = df_from(a);
            }
            Bh[u][rr] = v.hi;
            Bl[u][rr] = v.lo;
        }
    }
    __syncthreads();
    // thread (ty, tx): rows OZ_TR_RPT ty .., columns 4 tx .. 4 tx + 3
    const int ty = t >> 4, tx = t & 15;
    DF acc[OZ_TR_RPT][4];
#pragma unroll
    for (int a = 0; a < OZ_TR_RPT; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = DF{0.0f, 0.0f};
    const int umax = min(nb, 4 * tx + 4);  // W[c][u] = 0 for u > c
#pragma unroll 2
    for (int u = 0; u < umax; ++u) {
        DF bv[OZ_TR_RPT];
        if constexpr (OZ_TR_RPT == 4) {
            const float4 bh = *reinterpret_cast<const float4*>(&Bh[u][4 * ty]);
            const float4 bl = *reinterpret_cast<const float4*>(&Bl[u][4 * ty]);
            bv[0] = DF{bh.x, bl.x};
            bv[1] = DF{bh.y, bl.y};
            bv[2] = DF{bh.z, bl.z};
            bv[3] = DF{bh.w, bl.w};
        } else if constexpr (OZ_TR_RPT == 2) {
            const float2 bh = *reinterpret_cast<const float2*>(&Bh[u][2 * ty]);
            const float2 bl = *reinterpret_cast<const float2*>(&Bl[u][2 * ty]);
            bv[0] = DF{bh.x, bl.x};
            bv[1] = DF{bh.y, bl.y};
        } else {
            bv[0] = DF{Bh[u][ty], Bl[u][ty]};
        }
        const float4 wh = *reinterpret_cast<const float4*>(&Wh[u][4 * tx]);
        const float4 wl = *reinterpret_cast<const float4*>(&Wl[u][4 * tx]);
        const DF wv[4] = {{wh.x, wl.x}, {wh.y, wl.y}, {wh.z, wl.z}, {wh.w, wl.w}};
#pragma unroll
        for (int a = 0; a < OZ_TR_RPT; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) df_fma_acc(acc[a][b], bv[a], wv[b]);
    }
    __syncthreads();  // the staging area below reuses the operand tiles
    float(*Xh)[OZ_NB + 1] = reinterpret_cast<float(*)[OZ_NB + 1]>(tr_raw);
    float(*Xl)[OZ_NB + 1] = Xh + OZ_TR_ROWS;
#pragma unroll
    for (int a = 0; a < OZ_TR_RPT; ++a) {
        const int r = r0 + OZ_TR_RPT * ty + a;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int cc = 4 * tx + b;
            DF x{0.0f, 0.0f};
            if (r < n && cc < nb) {
                x = df_norm(acc[a][b].hi, acc[a][b].lo);
                A[r + (int64_t)(c0 + cc) * ld] = df_to(x);
            }
            Xh[OZ_TR_RPT * ty + a][cc] = x.hi;
            Xl[OZ_TR_RPT * ty + a][cc] = x.lo;
        }
    }
    // digits of these rows for the later updates (whole 16-byte chunks per thread)
    if (Z != nullptr) {
        __syncthreads();
        for (int e = t; e < OZ_TR_ROWS * 8; e += 256) {
            const int rr = e >> 3, c8 = e & 7, r = r0 + rr;
            float xh[8], xl[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                xh[q] = Xh[rr][8 * c8 + q];
                xl[q] = Xl[rr][8 * c8 + q];
            }
            uint4 dg[OZ_S];
            oz_digits8(xh, xl, (r < n) ? E[r] : 0, dg);
            oz_store_digits(Z, nrt, c0 / OZ_NB, r, c8, dg);
        }
    }
}

static size_t oz_smem() { return sizeof(OzSmem) + 1024; }
static_assert(sizeof(OzSmem) + 1024 <= 232448, "the update CTA's shared memory fits one SM");

static int oz_nrt(int n) { return (n + OZ_RT - 1) / OZ_RT; }
static int oz_nbc(int n) { return (n + OZ_NB - 1) / OZ_NB; }

static size_t oz_trsm_smem() { return sizeof(float) * 2 * OZ_NB * (OZ_TR_ROWS + OZ_NB); }
static_assert(sizeof(float) * 2 * OZ_TR_ROWS * (OZ_NB + 1) <= sizeof(float) * 2 * OZ_NB * (OZ_TR_ROWS + OZ_NB),
              "the digit staging fits the operand tiles");

size_t chol_oz_ws_bytes(int n) {
    const int nrt = oz_nrt(n), nbc = oz_nbc(n);
    return ws_round(sizeof(int) * (size_t)n) +
           ws_round((size_t)2 * nbc * OZ_S * nrt * OZ_AT) +
           ws_round(sizeof(long long) * 2 * (size_t)OZ_NB * nrt * OZ_RT) +
           ws_round(sizeof(float) * 2 * OZ_NB * OZ_NB);
}

#define OZ_CHAIN_SMS 4

// Update of block column j from the block columns [c_lo, c_hi) (K sub-chunks [2 c_lo, 2 c_hi)),
// cut into work items of P sub-chunks, one CTA per item (the bulk: a persistent grid).
static mvn_status oz_update_launch(mvn_ctx* ctx, cudaStream_t st, int n, int nrt, int j, int c_lo,
                                   int c_hi, int P, const uint8_t* Z, const int* E,
                                   long long* Tj, int64_t ldT, size_t ssm) {
    OzWork w;
    w.n = n;
    w.j = j;
    w.nrt = nrt;
    w.rt0 = (j * OZ_NB) / OZ_RT;
    w.n_rt = nrt - w.rt0;
    w.kc0 = 2 * c_lo;
    w.kc1 = 2 * c_hi;
    w.ldT = ldT;
    w.P = P;
    w.n_items = w.n_rt * ((w.kc1 - w.kc0 + P - 1) / P);
    // the bulk (low-priority stream) runs as a persistent grid that leaves OZ_CHAIN_SMS SMs to
    // the POTRF / TRSM chain, whose kernels cannot share an SM with an update CTA (registers):
    // they start at once instead of when an update CTA retires (W2: Cholesky 56.4 -> 53.9 ms
    // with 4 SMs left free; 8: 54.3, 16: 55.2, 32: 56.3)
    int grid = w.n_items;
    if (st == ctx->aux[1]) grid = std::max(1, std::min(w.n_items, ctx->sm_count - OZ_CHAIN_SMS));
    MVN_TIMED_ON(ctx, st, "k_oz_update",
                 (k_oz_update<<<grid, OZ_THREADS, ssm, st>>>(w, Z, E, Tj, ctx->d_status)));
    return MVN_OK;
}

// Left-looking factorisation over 64-wide block columns.  The update of block column j is the
// bulk (block columns 0 .. j-2) plus the tail (block column j-1).  The bulk of column j+1 needs
// only digits that exist once column j-1 is split, so it runs on a low-priority stream while the
// high-priority stream does the tail, POTRF, TRSM and split of column j (the chain every later
// column waits for); the two update sums of a column go into one of two integer accumulators
// (column parity).  The update kernel is launched one CTA per work item, so that the chain's
// kernels get SMs as the bulk's CTAs retire.  Both streams fork from and join the caller's stream.
// Subtract the finished trailing update of block column j (c0 = 64 j, nb columns) from A:
// A(r, c0 + u) -= T(r, u) 2^(E_r + E_{c0+u} - 49) for r >= c0 + u, and clear T.
__global__ void k_oz_apply(double* __restrict__ A, int64_t ld, int n, int c0, int nb,
                           const int* __restrict__ E, long long* __restrict__ T, int64_t ldT,
                           const int* status) {
    if (oz_failed(status)) return;
    const int r = c0 + blockIdx.x * blockDim.x + threadIdx.x;
    const int u = blockIdx.y;
    if (r >= n || u >= nb || r < c0 + u) return;
    const long long v = T[r + (int64_t)u * ldT];
    if (v == 0) return;
    A[r + (int64_t)(c0 + u) * ld] -= (double)v * oz_pow2(E[r] + E[c0 + u] - 49);
    T[r + (int64_t)u * ldT] = 0;
}

static mvn_status chol_oz_run(mvn_ctx* ctx, int n, double* A, int64_t ld, char* ws, int ncols);

mvn_status chol_oz_launch(mvn_ctx* ctx, int n, double* A, int64_t ld, char* ws) {
    return chol_oz_run(ctx, n, A, ld, ws, n);
}

// The first ncols columns (a multiple of 64) of the factorisation of the order-n matrix A, and
// the Schur complement A22 - A21 A11^-1 A12 left in the lower triangle of the trailing block:
// the factor's block columns as in chol_oz_launch, then every trailing block column updated by
// all of them (the exact-digit tensor-core update, K = ncols) and the update subtracted in FP64.
mvn_status chol_oz_partial(mvn_ctx* ctx, int n, double* A, int64_t ld, int ncols, char* ws) {
    if (ncols % OZ_NB != 0 || ncols < 0 || ncols > n)
        return mvn_fail(ctx, MVN_ERR_ARG, "partial factorisation: ncols a multiple of 64, <= n");
    if (ncols == 0) return MVN_OK;
    return chol_oz_run(ctx, n, A, ld, ws, ncols);
}

size_t chol_oz_partial_ws_bytes(int n, int ncols) {
    const int nrt = oz_nrt(n), ncb = ncols / OZ_NB;
    return ws_round(sizeof(int) * (size_t)n) +
           ws_round((size_t)2 * std::max(ncb, 1) * OZ_S * nrt * OZ_AT) +
           ws_round(sizeof(long long) * 2 * (size_t)OZ_NB * nrt * OZ_RT) +
           ws_round(sizeof(float) * 2 * OZ_NB * OZ_NB);
}

static mvn_status chol_oz_run(mvn_ctx* ctx, int n, double* A, int64_t ld, char* ws, int ncols) {
    const int nrt = oz_nrt(n), nbc = oz_nbc(n);
    const int ncb = (ncols >= n) ? nbc : ncols / OZ_NB;  // block columns that are factorised
    const int64_t ldT = (int64_t)nrt * OZ_RT;
    const TuneParams tp = tune_chol(ctx, n);
    WsCarver wc(ws);
    int* E = wc.take<int>((size_t)n);
    uint8_t* Z = wc.take<uint8_t>((size_t)2 * std::max(ncb, 1) * OZ_S * nrt * OZ_AT);
    long long* T = wc.take<long long>((size_t)2 * OZ_NB * ldT);
    float* Wt = wc.take<float>((size_t)2 * OZ_NB * OZ_NB);
    MVN_TRY(ctx_aux(ctx));
    cudaStream_t hi = ctx->aux[0], lo = ctx->aux[1];
    cudaEvent_t ev_fork = ctx->aux_ev[0], ev_split = ctx->aux_ev[1];
    cudaEvent_t ev_bulk[2] = {ctx->aux_ev[2], ctx->aux_ev[3]};
    cudaEvent_t ev_join = ctx->aux_ev[4];
    const size_t ssm = oz_smem();
    MVN_CUDA(ctx, cudaFuncSetAttribute(k_oz_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)ssm));
    const size_t tsm = oz_trsm_smem();
    MVN_CUDA(ctx, cudaFuncSetAttribute(k_oz_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tsm));
    MVN_CUDA(ctx, cudaEventRecord(ev_fork, ctx->stream));
    MVN_CUDA(ctx, cudaStreamWaitEvent(hi, ev_fork, 0));
    MVN_CUDA(ctx, cudaMemsetAsync(T, 0, sizeof(long long) * 2 * (size_t)OZ_NB * ldT, hi));
    k_oz_exps<<<(n + 255) / 256, 256, 0, hi>>>(n, A, ld, E);
    MVN_LAUNCHED(ctx);
    bool lo_used = false;
    for (int j = 0; j < ncb; ++j) {
        const int c0 = j * OZ_NB;
        const int nb = std::min(OZ_NB, n - c0);
        long long* Tj = T + (size_t)(j & 1) * OZ_NB * ldT;
        // bulk of column j+1 (block columns 0 .. j-1): split(j-1) is the last digit write it reads
        if (j >= 1 && j + 1 < ncb) {
            MVN_CUDA(ctx, cudaStreamWaitEvent(lo, ev_split, 0));
            long long* Tn = T + (size_t)((j + 1) & 1) * OZ_NB * ldT;
            MVN_TRY(oz_update_launch(ctx, lo, n, nrt, j + 1, 0, j, tp.chol_bulk_p, Z, E, Tn, ldT,
                                     ssm));
            MVN_CUDA(ctx, cudaEventRecord(ev_bulk[(j + 1) & 1], lo));
            lo_used = true;
        }
        if (j >= 1) {
            // tail of column j (block column j-1), then wait for its bulk
            MVN_TRY(oz_update_launch(ctx, hi, n, nrt, j, j - 1, j, tp.chol_tail_p, Z, E, Tj, ldT,
                                     ssm));
            if (j >= 2) MVN_CUDA(ctx, cudaStreamWaitEvent(hi, ev_bulk[j & 1], 0));
        }
        // the digits of block column j are written by POTRF (diagonal rows) and TRSM (the rows
        // below, up to the end of the last row tile) when a later column needs them
        uint8_t* Zj = (j + 1 < nbc) ? Z : nullptr;
        MVN_TIMED_ON(ctx, hi, "k_oz_potrf",
                     (k_oz_potrf<<<1, OZ_PF_THREADS, 0, hi>>>(A, ld, c0, nb, E, Tj, ldT, Wt, Zj, nrt,
                                                    ctx->d_status)));
        const int rows = (Zj != nullptr) ? nrt * OZ_RT - c0 - nb : n - c0 - nb;
        if (rows > 0) {
            MVN_TIMED_ON(ctx, hi, "k_oz_trsm",
                         (k_oz_trsm<<<(rows + OZ_TR_ROWS - 1) / OZ_TR_ROWS, 256, tsm, hi>>>(
                             A, ld, c0, nb, n, E, Tj, ldT, Wt, Zj, nrt, ctx->d_status)));
        }
        if (j + 1 < nbc) MVN_CUDA(ctx, cudaEventRecord(ev_split, hi));
    }
    // partial factorisation: every trailing block column takes the update by all ncols columns
    for (int j = ncb; j < nbc && ncb < nbc; ++j) {
        const int c0 = j * OZ_NB;
        const int nb = std::min(OZ_NB, n - c0);
        long long* Tj = T + (size_t)(j & 1) * OZ_NB * ldT;
        MVN_TRY(oz_update_launch(ctx, hi, n, nrt, j, 0, ncb, tp.chol_bulk_p, Z, E, Tj, ldT, ssm));
        k_oz_apply<<<dim3((unsigned)((n - c0 + 255) / 256), OZ_NB), 256, 0, hi>>>(
            A, ld, n, c0, nb, E, Tj, ldT, ctx->d_status);
        MVN_LAUNCHED(ctx);
    }
    // join both streams back into the caller's stream
    MVN_CUDA(ctx, cudaEventRecord(ev_join, hi));
    MVN_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ev_join, 0));
    if (lo_used) {
        MVN_CUDA(ctx, cudaEventRecord(ev_join, lo));
        MVN_CUDA(ctx, cudaStreamWaitEvent(ctx->stream, ev_join, 0));
    }
    return MVN_OK;
}
