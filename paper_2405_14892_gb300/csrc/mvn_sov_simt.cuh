// mvn_sov_simt.cuh -- the CUDA-core tile sweep of the SOV estimator (Eqs. 2-3, Algs. 2-3),
// shared by the forward entry points and the adjoint.
#pragma once
#include "mvn_sov.cuh"
#include "mvn_sov_step.cuh"

#define SOV_P 128

// ---------------------------------------------------------------- tile sweep

template <int B, typename T>
struct SovSmem {
    T Lk[B][B];       // GEMM operand: Lk[kk][v] = L(r0+v, k0+kk)
    T Ld[B][B + 1];   // diagonal block: Ld[v][u] = L(r0+v, r0+u), u <= v
    double a[B], b[B];
    uint64_t alpha[B];
};

// Sweep one tile of 128 paths of problem P through all n dimensions.
// T = working type of the limit GEMM and of the stored y (double: FP64 path; float: mixed).
template <int B, typename T, bool ELEM64>
__device__ void sov_tile(const SovProblem& P, int tile, const uint64_t* __restrict__ alpha,
                         T* __restrict__ Ycta, SovSmem<B, T>& sm) {
    const int t = threadIdx.x;
    const int n = P.n;
    const int64_t p = (int64_t)tile * SOV_P + t;
    const bool valid = p < P.Ntot;
    const int64_t pg = P.p0 + p;  // index of the path in the whole lattice rule
    const int64_t q = valid ? pg / P.Ns : 0;
    const uint64_t j = valid ? (uint64_t)(pg - q * P.Ns) + 1u : 1u;
    const uint64_t* __restrict__ dq = P.delta + q * P.dstride;
    const double* __restrict__ L = P.L;
    const int64_t ld = P.ld;
    LogProd lp;
    int pf = 0;
    int next_k = (P.nprefix > 0) ? P.prefix[0] : -1;

    for (int r0 = 0; r0 < n; r0 += B) {
        const int nb = min(B, n - r0);
        T acc[B];
#pragma unroll
        for (int v = 0; v < B; ++v) acc[v] = (T)0;
        // limit shift from earlier blocks: acc[v] = sum_{k < r0} L(r0+v, k) y_k  (Alg. 2 (c))
        for (int k0 = 0; k0 < r0; k0 += B) {
            __syncthreads();
            for (int e = t; e < B * B; e += SOV_P) {
                const int v = e % B, kk = e / B;
                const int row = r0 + v;
                sm.Lk[kk][v] = (row < n) ? (T)L[row + (int64_t)(k0 + kk) * ld] : (T)0;
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < B; ++kk) {
                const T yk = Ycta[(int64_t)(k0 + kk) * SOV_P + t];
#pragma unroll
                for (int v = 0; v < B; ++v) acc[v] = fma(sm.Lk[kk][v], yk, acc[v]);
            }
        }
        // diagonal block (Alg. 3)
        __syncthreads();
        for (int e = t; e < B * B; e += SOV_P) {
            const int v = e % B, u = e / B;
            sm.Ld[v][u] = (v < nb && u <= v) ? (T)L[(r0 + v) + (int64_t)(r0 + u) * ld] : (T)0;
        }
        if (t < B) {
            sm.a[t] = (t < nb) ? P.a[r0 + t] : 0.0;
            sm.b[t] = (t < nb) ? P.b[r0 + t] : 1.0;
            sm.alpha[t] = (t < nb) ? alpha[r0 + t] : 0u;
        }
        __syncthreads();
        T y[B];
#pragma unroll
        for (int v = 0; v < B; ++v) {
            if (v < nb) {
                T s = acc[v];
#pragma unroll
                for (int u = 0; u < v; ++u) s = fma(sm.Ld[v][u], y[u], s);
                const double w = lattice_w(j, sm.alpha[v], dq[r0 + v]);
                double delta;
                if constexpr (ELEM64) {
                    y[v] = (T)sov_step_f64(sm.a[v], sm.b[v], (double)s, (double)sm.Ld[v][v], w,
                                           delta);
                } else {
                    y[v] = (T)sov_step_f32(sm.a[v], sm.b[v], (float)s, (float)sm.Ld[v][v], w,
                                           delta);
                }
                lp.mul(delta);
                if (valid) Ycta[(int64_t)(r0 + v) * SOV_P + t] = y[v];
                while (next_k == r0 + v + 1) {
                    if (valid) P.logw_prefix[(int64_t)pf * P.Ntot + p] = lp.log_value();
                    ++pf;
                    next_k = (pf < P.nprefix) ? P.prefix[pf] : -1;
                }
            } else {
                y[v] = (T)0;
            }
        }
    }
    if (valid && P.logw) P.logw[p] = lp.log_value();
}

struct SovBatch {
    SovProblem single;               // used when probs == nullptr (item it -> tile it)
    const SovProblem* probs;         // batched: problem table
    const int2* items;               // batched: (problem, tile), longest problems first
    int nitems;
    int* counter;                    // work-queue head (zeroed before the launch)
    int y_per_tile;                  // 1: Y of tile `it` kept at Yscratch + it * ystride (adjoint)
};

template <int B, typename T, bool ELEM64>
__global__ void __launch_bounds__(SOV_P) k_sov_simt(const SovBatch batch,
                                                    const uint64_t* __restrict__ alpha,
                                                    T* __restrict__ Yscratch, int64_t ystride) {
    __shared__ SovSmem<B, T> sm;
    __shared__ int s_item;
    T* Ycta = Yscratch + (int64_t)blockIdx.x * ystride;
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = atomicAdd(batch.counter, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= batch.nitems) break;
        if (batch.probs == nullptr) {
            T* Yt = batch.y_per_tile ? Yscratch + (int64_t)it * ystride : Ycta;
            sov_tile<B, T, ELEM64>(batch.single, it, alpha, Yt, sm);
        } else {
            const int2 item = batch.items[it];
            sov_tile<B, T, ELEM64>(batch.probs[item.x], item.y, alpha, Ycta, sm);
        }
    }
}

