// mvn_chol_oz.cu -- tile Cholesky (Alg. 1 "dpotrf") whose trailing updates run on the tcgen05
// tensor cores with FP64-class accuracy (the MVN_MIXED factorisation).
//
// The SOV estimate needs an FP64-accurate factor (an FP32 factor moves log P by ~1e-2 at
// n = 16,384), and GB300's FP64 units deliver ~1.25 TFLOP/s.  The update L(i,:) L(j,:)^T of the
// left-looking algorithm is therefore computed exactly from small-integer digits on the BF16
// tensor cores (the error-free splitting of Ozaki, Ogita, Oishi and Rump, 2012):
//   - every row i of L is scaled by 2^-E_i with 2^E_i > sqrt(Sigma_ii) >= |L_ik| (fixed before the
//     factorisation, since sum_k L_ik^2 = Sigma_ii), so x_ik = L_ik 2^-E_i lies in (-1, 1);
//   - x_ik = sum_{s<S} a_ik^(s) 2^(-7(s+1)) + O(2^(-7S)) with integer digits |a^(s)| <= 128,
//     exact in BF16;
//   - over a 128-wide K chunk, sum_k a^(s)_ik a^(t)_jk is an integer below 2^24 even when the
//     up to 6 digit pairs of one level s+t share an accumulator, so the tensor core's FP32
//     accumulation (which truncates) is exact;
//   - each chunk's 6 level accumulators are drained into double-float (FP32 pair) registers, and
//     at the end C_ij -= 2^(E_i+E_j) * acc in FP64.
// With S = 6 digits the products carry 43 bits relative to |L_i||L_j| (row maxima), against 24
// for FP32.  The diagonal block (POTRF), the panel solve (TRSM) and the digit split run in FP64.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "mvn_internal.cuh"
#include "mvn_tc.cuh"

#define OZ_NB 128           // block column width = K chunk
#define OZ_S 6              // digit slices per value
#define OZ_TILE 16384       // one 128-row x 64-column BF16 tile (128-byte swizzle)
#define OZ_HALF 8192        // rows 0-63 or 64-127 of such a tile
#define OZ_WAIT 4000000000LL

__device__ __forceinline__ bool oz_failed(const int* status) {
    return *(volatile const int*)status != 0;
}

// E_i with 2^E_i > sqrt(A_ii)
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

// Digits of the finished block column j (columns c0 .. c0+127, rows >= c0) into the slice tiles
// Z[((j*S + s)*nt + rt)*2 + ks].  One CTA per row tile rt >= j.  x = L_ik 2^-E_i is rounded once
// to 42-bit fixed point v = rint(x 2^42) (the same value as six successive 7-bit roundings), and
// the balanced digits are peeled off with integer shifts: d = (v + 2^(k-1)) >> k, v -= d 2^k.
__global__ void k_oz_split(int n, const double* __restrict__ A, int64_t ld,
                           const int* __restrict__ E, int j, int nt, uint8_t* __restrict__ Z) {
    const int rt = j + blockIdx.x;
    const int c0 = j * OZ_NB;
    for (int e = threadIdx.x; e < OZ_NB * OZ_NB; e += blockDim.x) {
        const int r = e % OZ_NB, k = e / OZ_NB;  // consecutive threads: consecutive rows
        const int i = rt * OZ_NB + r, col = c0 + k;
        long long v = 0;
        if (i < n && col < n && col <= i) v = llrint(ldexp(A[i + (int64_t)col * ld], 42 - E[i]));
        const int ks = k >> 6, kk = k & 63;
        const uint32_t off = tc::sw128_off(r, kk);
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) {
            const int sh = 7 * (OZ_S - 1 - s);
            const long long d = (sh > 0) ? ((v + (1ll << (sh - 1))) >> sh) : v;
            v -= d * (1ll << sh);
            uint8_t* tile = Z + ((((size_t)j * OZ_S + s) * nt + rt) * 2 + ks) * OZ_TILE;
            *reinterpret_cast<__nv_bfloat16*>(tile + off) = __int2bfloat16_rn((int)d);
        }
    }
}

struct __align__(1024) OzSmem {
    uint8_t a[OZ_S][OZ_TILE];  // A digits: 128 rows x 64 K per slice
    uint8_t b[OZ_S][OZ_HALF];  // B digits: 64 rows x 64 K per slice
    int Ej[64];
    uint64_t full, mdone;
    uint32_t tmem;
    int abort;
};

__device__ __forceinline__ void df_add(float& hi, float& lo, float x) {
    const float s = hi + x;
    const float bb = s - hi;
    const float err = (hi - (s - bb)) + (x - bb);
    hi = s;
    lo += err;
}

// Left-looking update of block column j: output tile = row tile (j + blockIdx.x), columns
// c0 + 64*blockIdx.y .. +63, from the digit tiles of chunks 0 .. j-1.  128 threads (row = thread).
__global__ void __launch_bounds__(128, 1) k_oz_update(int n, double* __restrict__ A, int64_t ld,
                                                       const int* __restrict__ E, int j, int nt,
                                                       const uint8_t* __restrict__ Z,
                                                       int* __restrict__ status) {
    extern __shared__ uint8_t smem_raw[];
    OzSmem& sm = *reinterpret_cast<OzSmem*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                            ~(uintptr_t)1023);
    if (oz_failed(status)) return;
    const int t = threadIdx.x, warp = t >> 5;
    const int rt = j + blockIdx.x, half = blockIdx.y;
    const int c0 = j * OZ_NB;
    if (t == 0) {
        tc::mbar_init(&sm.full, 1);
        tc::mbar_init(&sm.mdone, 1);
        tc::mbar_fence_init();
        sm.abort = 0;
    }
    if (t < 64) {
        const int col = c0 + 64 * half + t;
        sm.Ej[t] = (col < n) ? E[col] : 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(&sm.tmem, 512);
        tc::tmem_relinquish();
    }
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
    const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(64 >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);  // BF16 x BF16 -> F32, M=128, N=64
    float hi[64], lo[64];
#pragma unroll
    for (int c = 0; c < 64; ++c) {
        hi[c] = 0.0f;
        lo[c] = 0.0f;
    }
    uint32_t par = 0;
    const uint32_t lane_base = ((uint32_t)warp * 32u) << 16;
    for (int c = 0; c < j && !sm.abort; ++c) {
        for (int ks = 0; ks < 2; ++ks) {
            if (t == 0) {
                tc::mbar_arrive_expect_tx(&sm.full, OZ_S * (OZ_TILE + OZ_HALF));
                for (int s = 0; s < OZ_S; ++s) {
                    const uint8_t* za = Z + ((((size_t)c * OZ_S + s) * nt + rt) * 2 + ks) * OZ_TILE;
                    const uint8_t* zb =
                        Z + ((((size_t)c * OZ_S + s) * nt + j) * 2 + ks) * OZ_TILE + half * OZ_HALF;
                    tc::bulk_g2s(sm.a[s], za, OZ_TILE, &sm.full);
                    tc::bulk_g2s(sm.b[s], zb, OZ_HALF, &sm.full);
                }
                if (!tc::mbar_wait(&sm.full, par, OZ_WAIT)) {
                    dev_raise(status, MVN_ERR_TIMEOUT, 0);
                    sm.abort = 1;
                } else {
                    tc::tc_fence_after();
#pragma unroll 1
                    for (int s = 0; s < OZ_S; ++s) {
#pragma unroll 1
                        for (int u = 0; u + s < OZ_S; ++u) {
                            const uint32_t lev = (uint32_t)(s + u);
                            const uint32_t dcol = sm.tmem + lev * 64u;
#pragma unroll
                            for (int k16 = 0; k16 < 4; ++k16) {
                                const uint64_t ad = tc::sdesc_sw128(tc::smem_u32(sm.a[s]) + k16 * 32);
                                const uint64_t bd = tc::sdesc_sw128(tc::smem_u32(sm.b[u]) + k16 * 32);
                                const uint32_t acc = (ks == 0 && k16 == 0 && s == 0) ? 0u : 1u;
                                tc::mma_f16(dcol, ad, bd, idesc, acc);
                            }
                        }
                    }
                    tc::mma_commit(&sm.mdone);
                }
            }
            __syncthreads();
            if (sm.abort) break;
            // the stage is reused by the next K half / chunk: wait for the MMAs (bounded)
            if (!tc::mbar_wait(&sm.mdone, par, OZ_WAIT)) {
                if (t == 0) dev_raise(status, MVN_ERR_TIMEOUT, 0);
                sm.abort = 1;
            }
            par ^= 1u;
            tc::tc_fence_after();
            __syncthreads();
            if (sm.abort) break;
        }
        if (sm.abort) break;
        // drain the 6 exact level sums of this chunk into the double-float accumulators
#pragma unroll 1
        for (int lev = 0; lev < OZ_S; ++lev) {
            const float sc = exp2f(-7.0f * (float)(lev + 2));
#pragma unroll
            for (int cc = 0; cc < 64; cc += 16) {
                float v[16];
                tc::tmem_ld16(sm.tmem + lane_base + (uint32_t)lev * 64u + cc, v);
#pragma unroll
                for (int q = 0; q < 16; ++q) df_add(hi[cc + q], lo[cc + q], v[q] * sc);
            }
        }
        tc::tc_fence_before();
        __syncthreads();
    }
    // C_ij -= 2^(E_i + E_j) (hi + lo), lower part only
    const int i = rt * OZ_NB + t;
    if (!sm.abort && i < n) {
        const int Ei = E[i];
#pragma unroll
        for (int c = 0; c < 64; ++c) {
            const int col = c0 + 64 * half + c;
            if (col < n && col <= i) {
                const double v = ldexp((double)hi[c] + (double)lo[c], Ei + sm.Ej[c]);
                A[i + (int64_t)col * ld] -= v;
            }
        }
    }
    tc::tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc::tc_fence_after();
        tc::tmem_dealloc(sm.tmem, 512);
    }
}

// POTRF of the diagonal block (c0, c0), nb <= 128, in shared memory (FP64).  256 threads as a
// 16 x 16 grid over the trailing triangle (no integer division in the inner loops).
__global__ void __launch_bounds__(256) k_oz_potrf(double* __restrict__ A, int64_t ld, int c0,
                                                  int nb, int* status) {
    extern __shared__ double Ts[];  // nb x (nb + 1)
    __shared__ int bad;
    if (oz_failed(status)) return;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4;
    const int sd = nb + 1;
    if (t == 0) bad = 0;
    for (int jj = ty; jj < nb; jj += 16)
        for (int i = jj + tx; i < nb; i += 16) Ts[i * sd + jj] = A[(c0 + i) + (int64_t)(c0 + jj) * ld];
    __syncthreads();
    for (int jj = 0; jj < nb; ++jj) {
        if (t == 0) {
            const double d = Ts[jj * sd + jj];
            if (!(d > 0.0)) {
                dev_raise(status, MVN_ERR_NOT_PD, c0 + jj + 1);
                bad = 1;
            } else {
                Ts[jj * sd + jj] = sqrt(d);
            }
        }
        __syncthreads();
        if (bad) return;
        const double rl = 1.0 / Ts[jj * sd + jj];
        for (int i = jj + 1 + t; i < nb; i += 256) Ts[i * sd + jj] *= rl;
        __syncthreads();
        for (int i = jj + 1 + ty; i < nb; i += 16) {
            const double li = Ts[i * sd + jj];
            for (int c = jj + 1 + tx; c <= i; c += 16) Ts[i * sd + c] -= li * Ts[c * sd + jj];
        }
        __syncthreads();
    }
    for (int jj = ty; jj < nb; jj += 16)
        for (int i = jj + tx; i < nb; i += 16) A[(c0 + i) + (int64_t)(c0 + jj) * ld] = Ts[i * sd + jj];
}

// TRSM of the rows below the diagonal block: X L_jj^T = A(i, c0:c0+nb) for i >= c0 + nb, in two
// 64-column halves (x in registers; the first half is also kept in shared memory, one column
// per thread, for the second half's right-hand side).  One thread per row.
__global__ void __launch_bounds__(128) k_oz_trsm(double* __restrict__ A, int64_t ld, int c0,
                                                 int nb, int n, const int* status) {
    extern __shared__ double Ls[];  // nb x (nb + 1), then x1[64][128]
    if (oz_failed(status)) return;
    const int t = threadIdx.x;
    const int sd = nb + 1;
    double* x1s = Ls + nb * sd;
    for (int e = t; e < nb * nb; e += 128) {
        const int i = e % nb, k = e / nb;
        Ls[i * sd + k] = (i >= k) ? A[(c0 + i) + (int64_t)(c0 + k) * ld] : 0.0;
    }
    __syncthreads();
    const int r = c0 + nb + blockIdx.x * 128 + t;
    if (r >= n) return;
    double x[64];
    const int h0 = min(64, nb);
#pragma unroll
    for (int c = 0; c < 64; ++c) x[c] = (c < h0) ? A[r + (int64_t)(c0 + c) * ld] : 0.0;
#pragma unroll
    for (int c = 0; c < 64; ++c) {
        if (c < h0) {
            double s = x[c];
#pragma unroll
            for (int u = 0; u < c; ++u) s -= x[u] * Ls[c * sd + u];
            x[c] = s / Ls[c * sd + c];
            A[r + (int64_t)(c0 + c) * ld] = x[c];
            x1s[c * 128 + t] = x[c];
        }
    }
    if (nb <= 64) return;
    const int h1 = nb - 64;
#pragma unroll
    for (int c = 0; c < 64; ++c) x[c] = (c < h1) ? A[r + (int64_t)(c0 + 64 + c) * ld] : 0.0;
    for (int u = 0; u < 64; ++u) {
        const double xu = x1s[u * 128 + t];
#pragma unroll
        for (int c = 0; c < 64; ++c)
            if (c < h1) x[c] -= xu * Ls[(64 + c) * sd + u];
    }
#pragma unroll
    for (int c = 0; c < 64; ++c) {
        if (c < h1) {
            double s = x[c];
#pragma unroll
            for (int u = 0; u < c; ++u) s -= x[u] * Ls[(64 + c) * sd + 64 + u];
            x[c] = s / Ls[(64 + c) * sd + 64 + c];
            A[r + (int64_t)(c0 + 64 + c) * ld] = x[c];
        }
    }
}

static size_t oz_smem() { return sizeof(OzSmem) + 1024; }

size_t chol_oz_ws_bytes(int n) {
    const int nt = (n + OZ_NB - 1) / OZ_NB;
    return ws_round(sizeof(int) * (size_t)n) +
           ws_round((size_t)nt * OZ_S * nt * 2 * OZ_TILE);
}

mvn_status chol_oz_launch(mvn_ctx* ctx, int n, double* A, int64_t ld, char* ws) {
    const int nt = (n + OZ_NB - 1) / OZ_NB;
    WsCarver wc(ws);
    int* E = wc.take<int>((size_t)n);
    uint8_t* Z = wc.take<uint8_t>((size_t)nt * OZ_S * nt * 2 * OZ_TILE);
    k_oz_exps<<<(n + 255) / 256, 256, 0, ctx->stream>>>(n, A, ld, E);
    MVN_LAUNCHED(ctx);
    const size_t ssm = oz_smem();
    MVN_CUDA(ctx, cudaFuncSetAttribute(k_oz_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)ssm));
    const size_t dsm = sizeof(double) * OZ_NB * (OZ_NB + 1);
    MVN_CUDA(ctx, cudaFuncSetAttribute(k_oz_potrf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)dsm));
    const size_t tsm = dsm + sizeof(double) * 64 * 128;
    MVN_CUDA(ctx, cudaFuncSetAttribute(k_oz_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)tsm));
    for (int j = 0; j < nt; ++j) {
        const int c0 = j * OZ_NB;
        const int nb = std::min(OZ_NB, n - c0);
        if (j > 0) {
            MVN_TIMED(ctx, "k_oz_update",
                      (k_oz_update<<<dim3(nt - j, (nb + 63) / 64), 128, ssm, ctx->stream>>>(
                          n, A, ld, E, j, nt, Z, ctx->d_status)));
        }
        k_oz_potrf<<<1, 256, dsm, ctx->stream>>>(A, ld, c0, nb, ctx->d_status);
        MVN_LAUNCHED(ctx);
        const int rows = n - c0 - nb;
        if (rows > 0) {
            k_oz_trsm<<<(rows + 127) / 128, 128, tsm, ctx->stream>>>(A, ld, c0, nb, n,
                                                                      ctx->d_status);
            MVN_LAUNCHED(ctx);
        }
        if (j + 1 < nt) {
            k_oz_split<<<nt - j, 256, 0, ctx->stream>>>(n, A, ld, E, j, nt, Z);
            MVN_LAUNCHED(ctx);
        }
    }
    return MVN_OK;
}
