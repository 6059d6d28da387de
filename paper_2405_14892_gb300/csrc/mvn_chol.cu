// mvn_chol.cu -- tile Cholesky factorisation Sigma = L L^T in FP64 (Alg. 1, "dpotrf"),
// right-looking over 64-wide panels: POTRF of the diagonal tile (one CTA, in shared memory),
// TRSM of the panel below it (one thread per row), SYRK/GEMM update of the trailing lower
// triangle (64 x 64 output tiles).  A non-positive pivot raises MVN_ERR_NOT_PD with the
// LAPACK-style 1-based column in the device status word; later kernels then return at once.
#include <math.h>

#include "mvn_internal.cuh"

#define CH_NB 64

// tensor-core factorisation with 42-bit products (mvn_chol_oz.cu)
size_t chol_oz_ws_bytes(int n);
mvn_status chol_oz_launch(mvn_ctx* ctx, int n, double* A, int64_t ld, char* ws);

__device__ __forceinline__ bool dev_failed(const int* status) {
    return *(volatile const int*)status != 0;
}

// POTRF of the nb x nb diagonal tile at (k0, k0), nb <= 64.  256 threads.
__global__ void __launch_bounds__(256) k_potrf(double* __restrict__ A, int64_t ld, int k0, int nb,
                                               int* status) {
    __shared__ double T[CH_NB][CH_NB + 1];  // T[i][j], i >= j
    __shared__ int bad;
    if (dev_failed(status)) return;
    const int t = threadIdx.x;
    if (t == 0) bad = 0;
    for (int e = t; e < nb * nb; e += 256) {
        int i = e % nb, j = e / nb;
        if (i >= j) T[i][j] = A[(k0 + i) + (int64_t)(k0 + j) * ld];
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
        if (t == 0) {
            double d = T[j][j];
            if (!(d > 0.0)) {
                if (!bad) dev_raise(status, MVN_ERR_NOT_PD, k0 + j + 1);
                bad = 1;
                T[j][j] = NAN;
            } else {
                T[j][j] = sqrt(d);
            }
        }
        __syncthreads();
        if (bad) break;
        const double ljj = T[j][j];
        for (int i = j + 1 + t; i < nb; i += 256) T[i][j] /= ljj;
        __syncthreads();
        // trailing update of the tile: T[i][c] -= T[i][j] T[c][j], j < c <= i
        const int m = nb - j - 1;
        for (int e = t; e < m * m; e += 256) {
            int i = j + 1 + e % m, c = j + 1 + e / m;
            if (c <= i) T[i][c] -= T[i][j] * T[c][j];
        }
        __syncthreads();
    }
    if (bad) return;
    for (int e = t; e < nb * nb; e += 256) {
        int i = e % nb, j = e / nb;
        if (i >= j) A[(k0 + i) + (int64_t)(k0 + j) * ld] = T[i][j];
    }
}

// TRSM: rows r0 <= i < n of the panel A(i, k0:k0+nb) <- A(i, k0:k0+nb) L_kk^-T (forward
// substitution per row: x_j = (a_j - sum_{l<j} x_l L_jl) / L_jj).  One thread per row.
__global__ void __launch_bounds__(128) k_trsm(double* __restrict__ A, int64_t ld, int k0, int nb,
                                              int r0, int n, const int* status) {
    __shared__ double Lk[CH_NB][CH_NB + 1];
    if (dev_failed(status)) return;
    const int t = threadIdx.x;
    for (int e = t; e < nb * nb; e += 128) {
        int i = e % nb, j = e / nb;
        Lk[i][j] = (i >= j) ? A[(k0 + i) + (int64_t)(k0 + j) * ld] : 0.0;
    }
    __syncthreads();
    const int i = r0 + blockIdx.x * 128 + t;
    if (i >= n) return;
    double x[CH_NB];
#pragma unroll
    for (int j = 0; j < CH_NB; ++j) {
        if (j < nb) {
            double s = A[i + (int64_t)(k0 + j) * ld];
#pragma unroll
            for (int l = 0; l < j; ++l) s -= x[l] * Lk[j][l];
            x[j] = s / Lk[j][j];
            A[i + (int64_t)(k0 + j) * ld] = x[j];
        } else {
            x[j] = 0.0;
        }
    }
}

// Trailing update: for lower tile pairs (ti >= tj) of the region starting at c0,
//   C(ti, tj) -= A(ti-rows, k0:k0+nb) A(tj-rows, k0:k0+nb)^T.   256 threads, 4x4 per thread.
__global__ void __launch_bounds__(256) k_syrk(double* __restrict__ A, int64_t ld, int k0, int nb,
                                              int c0, int n, const int* status) {
    __shared__ double Ai[CH_NB][CH_NB];  // Ai[kk][r]
    __shared__ double Aj[CH_NB][CH_NB];  // Aj[kk][c]
    if (dev_failed(status)) return;
    // tile pair from the linear block index
    const int x = blockIdx.x;
    int ti = (int)((sqrt(8.0 * x + 1.0) - 1.0) * 0.5);
    while ((ti + 1) * (ti + 2) / 2 <= x) ++ti;
    while (ti * (ti + 1) / 2 > x) --ti;
    const int tj = x - ti * (ti + 1) / 2;
    const int R0 = c0 + ti * CH_NB, C0 = c0 + tj * CH_NB;
    const int t = threadIdx.x;
    for (int e = t; e < nb * CH_NB; e += 256) {
        int r = e % CH_NB, kk = e / CH_NB;
        Ai[kk][r] = (R0 + r < n) ? A[(R0 + r) + (int64_t)(k0 + kk) * ld] : 0.0;
        Aj[kk][r] = (C0 + r < n) ? A[(C0 + r) + (int64_t)(k0 + kk) * ld] : 0.0;
    }
    __syncthreads();
    const int tx = t & 15, ty = t >> 4;
    double acc[4][4] = {};
    for (int kk = 0; kk < nb; ++kk) {
        double a[4], b[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) a[u] = Ai[kk][tx + 16 * u];
#pragma unroll
        for (int v = 0; v < 4; ++v) b[v] = Aj[kk][ty + 16 * v];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int c = C0 + ty + 16 * v;
        if (c >= n) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int r = R0 + tx + 16 * u;
            if (r >= n || r < c) continue;
            A[r + (int64_t)c * ld] -= acc[u][v];
        }
    }
}

// The first `ncols` steps of the right-looking factorisation of the order-n matrix A: columns
// 0..ncols-1 become the factor's, and the trailing block A(ncols:, ncols:) is left holding the
// Schur complement A22 - A21 A11^-1 A12 (lower triangle).  ncols = n is the full factorisation.
mvn_status chol_f64_partial(mvn_ctx* ctx, int n, double* A, int64_t ld, int ncols) {
    for (int k0 = 0; k0 < ncols; k0 += CH_NB) {
        const int nb = (ncols - k0 < CH_NB) ? ncols - k0 : CH_NB;
        k_potrf<<<1, 256, 0, ctx->stream>>>(A, ld, k0, nb, ctx->d_status);
        MVN_LAUNCHED(ctx);
        const int r0 = k0 + nb;
        if (r0 >= n) break;
        const int rows = n - r0;
        k_trsm<<<(rows + 127) / 128, 128, 0, ctx->stream>>>(A, ld, k0, nb, r0, n, ctx->d_status);
        MVN_LAUNCHED(ctx);
        const int T = (rows + CH_NB - 1) / CH_NB;
        const int64_t tiles = (int64_t)T * (T + 1) / 2;
        MVN_TIMED(ctx, "k_syrk",
                  (k_syrk<<<(unsigned)tiles, 256, 0, ctx->stream>>>(A, ld, k0, nb, r0, n,
                                                                   ctx->d_status)));
    }
    return MVN_OK;
}

mvn_status chol_f64_launch(mvn_ctx* ctx, int n, double* A, int64_t ld) {
    return chol_f64_partial(ctx, n, A, ld, n);
}

extern "C" mvn_status mvn_cholesky(mvn_ctx* ctx, int n, double* A, int64_t ld, int tile,
                                   mvn_prec prec, int* info) {
    if (!ctx) return MVN_ERR_ARG;
    if (tile < 0) return mvn_fail(ctx, MVN_ERR_ARG, "negative tile size");  // panel width is fixed at 64
    if (n < 0 || n > (1 << 21) || ld < (n > 0 ? n : 1) || (n > 0 && !A))
        return mvn_fail(ctx, MVN_ERR_ARG, "mvn_cholesky: invalid argument");
    if (prec != MVN_FP64 && prec != MVN_MIXED && prec != MVN_MIXED_SIMT)
        return mvn_fail(ctx, MVN_ERR_ARG, "unknown precision");
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    if (info) *info = 0;
    if (n > 0) {
        if (prec == MVN_MIXED) {
            MVN_TRY(ws_reserve(ctx, chol_oz_ws_bytes(n) + 1024));
            MVN_TRY(chol_oz_launch(ctx, n, A, ld, (char*)ctx->ws));
        } else {
            MVN_TRY(chol_f64_launch(ctx, n, A, ld));
        }
    }
    if (info) return mvn_sync(ctx, info);
    return MVN_OK;
}
