// mvn_tlr.cu -- tile low-rank (TLR) compression of the covariance and TLR Cholesky (Sec. III-E;
// Alg. 1 "pmvn_init" / "dpotrf" on TLR tiles), FP64.
//
// Compression of a batch of dense m x m tiles A (randomised range finder, Halko, Martinsson and
// Tropp 2011, with one power iteration), each step a batched kernel:
//   Y = A Omega (Omega Gaussian, m x r, r = max_rank + 8 <= m);  Q = orth(Y)
//   Y = A (A^T Q);  Q = orth(Y)
//   X = A^T Q (m x r);  X G = V Sigma (one-sided Jacobi SVD, FP64: rotations of column pairs
//   until the columns are orthogonal; sigma_l = the column norms, resolved relative to
//   themselves)
//   sigma_l sorted descending;  k = #{sigma_l > acc} capped at max_rank
//   U = Q G_k diag(sigma_k),  V = V_k  (so A ~= Q X^T = U V^T).
// orth(Y) is shifted Cholesky QR applied three times (Gram matrix + small shift, Cholesky,
// triangular inverse, Y R^-1): stable for rank-deficient sketches, whose surplus directions only
// add rows of negligible norm to B.
// TLR Cholesky, left-looking over tile columns k (as HiCMA's, with the low-rank updates of a tile
// accumulated densely and truncated once at the tile's accuracy):
//   D_kk -= sum_{l<k} U_kl (V_kl^T V_kl) U_kl^T;  L_kk = chol(D_kk)
//   A_ik  = U_ik V_ik^T - sum_{l<k} (U_il (V_il^T V_kl)) U_kl^T;  A_ik ~= U' V'^T;
//   L_ik  = U' (L_kk^-1 V')^T.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "mvn_internal.cuh"

mvn_status chol_f64_launch(mvn_ctx* ctx, int n, double* A, int64_t ld);

#include "mvn_tlr.cuh"

// ---------------------------------------------------------------- batched FP64 GEMM

// C(i,j) = alpha sum_l A(i,l) B(l,j) + beta C(i,j); A(i,l) = A[i*sar + l*sac],
// B(l,j) = B[l*sbr + j*sbc], C(i,j) = C[i + j*ldc]; beta = 0 does not read C.
struct GItem {
    const double* A;
    const double* B;
    double* C;
    int m, n, k;
    int64_t sar, sac, sbr, sbc, ldc;
    double alpha, beta;
};

__global__ void __launch_bounds__(256) k_bgemm(const GItem* __restrict__ items) {
    __shared__ double As[16][64 + 1];
    __shared__ double Bs[16][64 + 1];
    const GItem it = items[blockIdx.z];
    const int I0 = blockIdx.x * 64, J0 = blockIdx.y * 64;
    if (I0 >= it.m || J0 >= it.n) return;
    const int t = threadIdx.x, tx = t & 15, ty = t >> 4, w2 = (t >> 5) * 2;
    // FP64 is the scarce unit on this GPU, so no FMA is spent on padding: the row groups
    // (16 u ..), the column groups of this warp (16 v + w2 ..) and the K steps beyond the item's
    // sizes are skipped (uniform across the CTA or the warp; the skipped products were zeros)
    const int mrem = it.m - I0, nrem = it.n - J0;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < it.k; k0 += 16) {
        __syncthreads();
        for (int e = t; e < 16 * 64; e += 256) {
            const int i = e % 64, l = e / 64;
            const int gi = I0 + i, gl = k0 + l, gj = J0 + i;
            As[l][i] = (gi < it.m && gl < it.k) ? it.A[gi * it.sar + gl * it.sac] : 0.0;
            Bs[l][i] = (gj < it.n && gl < it.k) ? it.B[gl * it.sbr + gj * it.sbc] : 0.0;
        }
        __syncthreads();
        if (w2 >= nrem) continue;  // no column of this warp is in range
        const int kl = min(16, it.k - k0);
#pragma unroll
        for (int l = 0; l < 16; ++l) {
            if (l >= kl) break;
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = As[l][tx + 16 * u];
#pragma unroll
            for (int v = 0; v < 4; ++v) b[v] = Bs[l][ty + 16 * v];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (16 * u >= mrem) break;
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    if (16 * v + w2 >= nrem) break;
                    acc[u][v] = fma(a[u], b[v], acc[u][v]);
                }
            }
        }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int j = J0 + ty + 16 * v;
        if (j >= it.n) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = I0 + tx + 16 * u;
            if (i >= it.m) continue;
            double* c = it.C + i + (int64_t)j * it.ldc;
            *c = (it.beta == 0.0) ? it.alpha * acc[u][v] : fma(it.alpha, acc[u][v], it.beta * *c);
        }
    }
}

// Batched GEMM launcher: items are copied into a workspace slot (pageable copy: staged before
// the call returns).
static mvn_status bgemm(mvn_ctx* ctx, const std::vector<GItem>& items, GItem* d_items) {
    if (items.empty()) return MVN_OK;
    int mm = 0, nn = 0;
    for (auto& it : items) {
        mm = std::max(mm, it.m);
        nn = std::max(nn, it.n);
    }
    if (mm == 0 || nn == 0) return MVN_OK;
    MVN_CUDA(ctx, cudaMemcpyAsync(d_items, items.data(), sizeof(GItem) * items.size(),
                                  cudaMemcpyHostToDevice, ctx->stream));
    for (size_t z0 = 0; z0 < items.size(); z0 += 65535) {
        const unsigned nz = (unsigned)std::min<size_t>(65535, items.size() - z0);
        MVN_TIMED(ctx, "k_bgemm",
                  (k_bgemm<<<dim3((mm + 63) / 64, (nn + 63) / 64, nz), 256, 0, ctx->stream>>>(
                      d_items + z0)));
    }
    return MVN_OK;
}

static GItem gi(const double* A, int64_t sar, int64_t sac, const double* B, int64_t sbr,
                int64_t sbc, double* C, int64_t ldc, int m, int n, int k, double alpha,
                double beta) {
    GItem g;
    g.A = A;
    g.B = B;
    g.C = C;
    g.m = m;
    g.n = n;
    g.k = k;
    g.sar = sar;
    g.sac = sac;
    g.sbr = sbr;
    g.sbc = sbc;
    g.ldc = ldc;
    g.alpha = alpha;
    g.beta = beta;
    return g;
}

// ---------------------------------------------------------------- small dense kernels

// Omega (m x r, ld m): standard normals by Box-Muller of SplitMix64 counter outputs.
__global__ void k_gauss(int m, int r, uint64_t seed, double* __restrict__ Om) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)m * r) return;
    const uint64_t x1 = splitmix64_at(seed, 2 * (uint64_t)e);
    const uint64_t x2 = splitmix64_at(seed, 2 * (uint64_t)e + 1);
    const double u1 = ((double)(x1 >> 11) + 0.5) * 0x1p-53;
    const double u2 = ((double)(x2 >> 11) + 0.5) * 0x1p-53;
    Om[e] = sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// Per item (one CTA): G (r x r, ld r) <- inverse of the Cholesky factor of G + shift I, upper
// triangular R^-1 with G + shift I = R^T R, written to Rinv (r x r, ld r, strict lower = 0).
// shift = 1e-14 * (r + 1) * max_i G_ii keeps the factorisation of a rank-deficient Gram defined.
__global__ void __launch_bounds__(256) k_chol_inv(int r, double* const* __restrict__ Gs,
                                                  double* const* __restrict__ Rs) {
    double* G = Gs[blockIdx.x];
    double* R = Rs[blockIdx.x];
    const int t = threadIdx.x;
    __shared__ double shift;
    if (t == 0) {
        double mx = 0.0;
        for (int i = 0; i < r; ++i) mx = fmax(mx, G[i + (int64_t)i * r]);
        shift = 1e-14 * (r + 1) * mx + 1e-300;
    }
    __syncthreads();
    for (int i = t; i < r; i += 256) G[i + (int64_t)i * r] += shift;
    __syncthreads();
    // in place lower Cholesky G = L L^T (column loop)
    for (int j = 0; j < r; ++j) {
        __shared__ double ljj;
        if (t == 0) {
            const double d = G[j + (int64_t)j * r];
            ljj = sqrt(fmax(d, 1e-300));
            G[j + (int64_t)j * r] = ljj;
        }
        __syncthreads();
        for (int i = j + 1 + t; i < r; i += 256) G[i + (int64_t)j * r] /= ljj;
        __syncthreads();
        const int mrem = r - j - 1;
        for (int e = t; e < mrem * mrem; e += 256) {
            const int i = j + 1 + e % mrem, c = j + 1 + e / mrem;
            if (c <= i) G[i + (int64_t)c * r] -= G[i + (int64_t)j * r] * G[c + (int64_t)j * r];
        }
        __syncthreads();
    }
    // Linv (lower) column by column: L X = I; then R^-1 = (L^-1)^T (upper)
    for (int c = t; c < r; c += 256) {
        for (int i = 0; i < r; ++i) R[i + (int64_t)c * r] = 0.0;  // column c of R^-1
    }
    __syncthreads();
    for (int c = t; c < r; c += 256) {
        // x = L^-1 e_c (entries i >= c): x_i = (delta_ic - sum_{c<=l<i} L_il x_l) / L_ii
        for (int i = c; i < r; ++i) {
            double s = (i == c) ? 1.0 : 0.0;
            for (int l = c; l < i; ++l) s -= G[i + (int64_t)l * r] * R[c + (int64_t)l * r];
            R[c + (int64_t)i * r] = s / G[i + (int64_t)i * r];  // R^-1(c, i) = Linv(i, c)
        }
    }
}

// deterministic block sum of one value per thread (256 threads)
__device__ double block_sum256(double v, double* red) {
    const int t = threadIdx.x;
    red[t] = v;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (t < w) red[t] += red[t + w];
        __syncthreads();
    }
    const double s = red[0];
    __syncthreads();
    return s;
}

// One-sided (Hestenes) Jacobi SVD of X = A^T Q (m x r, ld m) per item, in place: plane rotations
// of column pairs make the columns mutually orthogonal, X <- X G with G (r x r) accumulated in W.
// Then X = V Sigma with sigma_j = ||X_j||, and A ~= Q X^T = (Q G) Sigma V^T.  Unlike an eigen-
// decomposition of B B^T it never forms a Gram matrix, so each singular value is resolved
// relative to itself (Demmel and Veselic 1992), not to sigma_1^2: the truncation at sigma ~ acc
// is decided on accurate values.  Pairs follow the round-robin (circle) order, each round's
// r/2 disjoint pairs spread over the block's warps (one warp per pair: three dot products over
// the m rows, then the rotation of the two columns of X and of W).  Columns whose norm stays
// below acc / 100 are left out of the rotations (the truncation drops them).  lam[j] = sigma_j^2 and
// order = the columns by descending sigma.  Rutishauser's rotation:
//   zeta = (beta - alpha) / (2 gamma), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
//   c = 1 / sqrt(1 + t^2), s = c t;  X_i <- c X_i - s X_j,  X_j <- s X_i + c X_j.
template <int CH>  // CH > 0: each lane keeps its CH rows of the pair in registers (m <= 32 CH)
__global__ void __launch_bounds__(256) k_jacobi1(int m, int r, double* const* __restrict__ Xs,
                                                 double* const* __restrict__ Ws,
                                                 double* const* __restrict__ lams,
                                                 int* const* __restrict__ orders,
                                                 int max_sweeps, double floor2) {
    __shared__ int s_rot;
    double* X = Xs[blockIdx.x];
    double* W = Ws[blockIdx.x];
    double* lam = lams[blockIdx.x];
    int* order = orders[blockIdx.x];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5, nw = blockDim.x >> 5;
    for (int e = t; e < r * r; e += blockDim.x) W[e] = ((e % r) == (e / r)) ? 1.0 : 0.0;
    const int rp = (r + 1) & ~1;  // even player count (player r is a dummy when r is odd)
    for (int sweep = 0; sweep < max_sweeps; ++sweep) {
        if (t == 0) s_rot = 0;
        __syncthreads();
        for (int round = 0; round < rp - 1; ++round) {
            for (int pi = warp; pi < rp / 2; pi += nw) {
                int i, j;
                if (pi == 0) {
                    i = round;
                    j = rp - 1;
                } else {
                    i = (round + pi) % (rp - 1);
                    j = (round - pi + (rp - 1)) % (rp - 1);
                }
                if (i > j) {
                    const int x = i;
                    i = j;
                    j = x;
                }
                if (j >= r) continue;  // the dummy player
                double* xi = X + (int64_t)i * m;
                double* xj = X + (int64_t)j * m;
                double al = 0.0, be = 0.0, ga = 0.0;
                double ra[CH > 0 ? CH : 1], rb[CH > 0 ? CH : 1];
                if constexpr (CH > 0) {
#pragma unroll
                    for (int q = 0; q < CH; ++q) {
                        const int u = lane + 32 * q;
                        ra[q] = (u < m) ? xi[u] : 0.0;
                        rb[q] = (u < m) ? xj[u] : 0.0;
                    }
#pragma unroll
                    for (int q = 0; q < CH; ++q) {
                        al = fma(ra[q], ra[q], al);
                        be = fma(rb[q], rb[q], be);
                        ga = fma(ra[q], rb[q], ga);
                    }
                } else {
                    for (int u = lane; u < m; u += 32) {
                        const double a = xi[u], b = xj[u];
                        al = fma(a, a, al);
                        be = fma(b, b, be);
                        ga = fma(a, b, ga);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    al += __shfl_xor_sync(0xffffffffu, al, o);
                    be += __shfl_xor_sync(0xffffffffu, be, o);
                    ga += __shfl_xor_sync(0xffffffffu, ga, o);
                }
                // converged pair; or a column below floor2 = (acc / 100)^2 in squared norm, which
                // the truncation drops: rotating with it would move the other column by at most
                // floor2 / its norm (far below acc), and its own direction is never used
                if (!(fabs(ga) > 2.2e-16 * sqrt(al * be)) || ga == 0.0 || fmin(al, be) < floor2)
                    continue;
                const double zeta = (be - al) / (2.0 * ga);
                const double tt = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / sqrt(1.0 + tt * tt), sn = c * tt;
                if constexpr (CH > 0) {
#pragma unroll
                    for (int q = 0; q < CH; ++q) {
                        const int u = lane + 32 * q;
                        if (u < m) {
                            xi[u] = c * ra[q] - sn * rb[q];
                            xj[u] = sn * ra[q] + c * rb[q];
                        }
                    }
                } else {
                    for (int u = lane; u < m; u += 32) {
                        const double a = xi[u], b = xj[u];
                        xi[u] = c * a - sn * b;
                        xj[u] = sn * a + c * b;
                    }
                }
                double* wi = W + (int64_t)i * r;
                double* wj = W + (int64_t)j * r;
                for (int u = lane; u < r; u += 32) {
                    const double a = wi[u], b = wj[u];
                    wi[u] = c * a - sn * b;
                    wj[u] = sn * a + c * b;
                }
                if (lane == 0) s_rot = 1;
            }
            __syncthreads();
        }
        if (!s_rot) break;
        __syncthreads();
    }
    // sigma_j^2 = ||X_j||^2, then the order by descending value (stable)
    for (int jj = warp; jj < r; jj += nw) {
        const double* xj = X + (int64_t)jj * m;
        double a = 0.0;
        for (int u = lane; u < m; u += 32) a = fma(xj[u], xj[u], a);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) lam[jj] = a;
    }
    __syncthreads();
    for (int jj = t; jj < r; jj += blockDim.x) {
        int rankpos = 0;
        for (int k = 0; k < r; ++k)
            rankpos += (lam[k] > lam[jj]) || (lam[k] == lam[jj] && k < jj);
        order[rankpos] = jj;
    }
}

// After k_jacobi1: WU(:, q) = G(:, order_q) sigma_q and WV(order_q, q) = 1 / sigma_q (a selection
// matrix, r x kmax, ld r) for q < k, zero columns for q >= k, k = #{sigma > acc} capped at kmax;
// then U = Q WU and V = X WV = the rotated columns scaled to unit norm.
__global__ void k_select1(int r, int kmax, double acc, double* const* __restrict__ Ws,
                          double* const* __restrict__ lams, int* const* __restrict__ orders,
                          double* const* __restrict__ WUs, double* const* __restrict__ WVs,
                          int* __restrict__ rank_out, int* __restrict__ capped) {
    const double* W = Ws[blockIdx.x];
    const double* lam = lams[blockIdx.x];
    const int* order = orders[blockIdx.x];
    double* WU = WUs[blockIdx.x];
    double* WV = WVs[blockIdx.x];
    __shared__ int ks;
    if (threadIdx.x == 0) {
        int k = 0;
        while (k < r && lam[order[k]] > 0.0 && sqrt(lam[order[k]]) > acc) ++k;
        if (k > kmax) {
            atomicAdd(capped, 1);
            k = kmax;
        }
        ks = k;
        rank_out[blockIdx.x] = k;
    }
    __syncthreads();
    const int k = ks;
    for (int e = threadIdx.x; e < r * kmax; e += blockDim.x) {
        const int i = e % r, q = e / r;
        double u = 0.0, v = 0.0;
        if (q < k) {
            const double sg = sqrt(lam[order[q]]);
            u = W[i + (int64_t)order[q] * r] * sg;
            v = (i == order[q]) ? 1.0 / sg : 0.0;
        }
        WU[e] = u;
        WV[e] = v;
    }
}

// Copy the lower triangle tiles of A into dense m x m scratch tiles (zero outside [0, n), identity
// on the diagonal of padded rows of diagonal tiles).  One block per (tile, column).
__global__ void k_copy_tile(int n, int m, const double* __restrict__ A, int64_t ld, int ti, int tj,
                            double* __restrict__ out) {
    const int c = blockIdx.x;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        const int i = ti * m + r, j = tj * m + c;
        double v = 0.0;
        if (i < n && j < n) v = (i >= j) ? A[i + (int64_t)j * ld] : A[j + (int64_t)i * ld];
        else if (i == j) v = 1.0;
        out[r + (int64_t)c * m] = v;
    }
}

// V(rows r0..r0+63, :) <- L_bb^-1 V(rows, :) for every item (64-row diagonal block of L_kk in
// shared memory, one thread per column of one item).
__global__ void k_trsm_block(int m, int kmax, const double* __restrict__ Lkk, int r0,
                             double* const* __restrict__ Vs, int nitems) {
    __shared__ double Lb[64][65];
    for (int e = threadIdx.x; e < 64 * 64; e += blockDim.x) {
        const int i = e % 64, k = e / 64;
        Lb[i][k] = (i >= k) ? Lkk[(r0 + i) + (int64_t)(r0 + k) * m] : 0.0;
    }
    __syncthreads();
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const int item = g / kmax, col = g % kmax;
    if (item >= nitems) return;
    double* V = Vs[item] + (int64_t)col * m + r0;
    double x[64];
#pragma unroll
    for (int i = 0; i < 64; ++i) {
        double s = V[i];
#pragma unroll
        for (int k = 0; k < i; ++k) s -= Lb[i][k] * x[k];
        x[i] = s / Lb[i][i];
    }
#pragma unroll
    for (int i = 0; i < 64; ++i) V[i] = x[i];
}

// ---------------------------------------------------------------- compression pipeline

struct CompWs {
    int m, r, kmax, T;
    double *Om, *Y, *Q, *Z, *B, *G, *R, *W, *WU, *WV, *lam;
    int *order, *rank, *capped, *rk;
    double **pG, **pR, **pW, **pWU, **pWV, **plam, **pB;
    int** porder;
    GItem* items;
};

static size_t comp_ws_bytes(int m, int r, int kmax, int T) {
    const size_t mr = (size_t)m * r, rr = (size_t)r * r;
    return ws_round(sizeof(double) * mr) + 4 * ws_round(sizeof(double) * mr * T) +
           3 * ws_round(sizeof(double) * rr * T) + 2 * ws_round(sizeof(double) * (size_t)r * kmax * T) +
           ws_round(sizeof(double) * (size_t)r * T) + 2 * ws_round(sizeof(int) * (size_t)r * T) +
           ws_round(sizeof(int) * (size_t)T) + ws_round(sizeof(int)) + 8 * ws_round(sizeof(void*) * T) +
           ws_round(sizeof(GItem) * (size_t)T * 4) + 8 * 256;
}

static CompWs comp_ws_carve(WsCarver& wc, int m, int r, int kmax, int T) {
    CompWs c;
    c.m = m;
    c.r = r;
    c.kmax = kmax;
    c.T = T;
    const size_t mr = (size_t)m * r, rr = (size_t)r * r;
    c.Om = wc.take<double>(mr);
    c.Y = wc.take<double>(mr * T);
    c.Q = wc.take<double>(mr * T);
    c.Z = wc.take<double>(mr * T);
    c.B = wc.take<double>(mr * T);
    c.G = wc.take<double>(rr * T);
    c.R = wc.take<double>(rr * T);
    c.W = wc.take<double>(rr * T);
    c.WU = wc.take<double>((size_t)r * kmax * T);
    c.WV = wc.take<double>((size_t)r * kmax * T);
    c.lam = wc.take<double>((size_t)r * T);
    c.order = wc.take<int>((size_t)r * T);
    c.rk = wc.take<int>((size_t)r * T);
    c.rank = wc.take<int>((size_t)T);
    c.capped = wc.take<int>(1);
    c.pG = wc.take<double*>(T);
    c.pR = wc.take<double*>(T);
    c.pW = wc.take<double*>(T);
    c.pWU = wc.take<double*>(T);
    c.pWV = wc.take<double*>(T);
    c.plam = wc.take<double*>(T);
    c.porder = wc.take<int*>(T);
    c.pB = wc.take<double*>(T);
    c.items = wc.take<GItem>((size_t)T * 4);
    return c;
}

// Q = orth(Y) for every item (three passes of shifted Cholesky QR); Y is overwritten.
static mvn_status comp_orth(mvn_ctx* ctx, CompWs& c, int T, double* Y, double* Q, int r) {
    const int m = c.m;
    const size_t mr = (size_t)m * r, rr = (size_t)r * r;
    double* src = Y;
    double* dst = Q;
    for (int pass = 0; pass < 3; ++pass) {
        std::vector<GItem> it;
        for (int t = 0; t < T; ++t)
            it.push_back(gi(src + t * mr, m, 1, src + t * mr, 1, m, c.G + t * rr, r, r, r, m, 1.0, 0.0));
        MVN_TRY(bgemm(ctx, it, c.items));
        MVN_TIMED(ctx, "k_chol_inv", (k_chol_inv<<<T, 256, 0, ctx->stream>>>(r, c.pG, c.pR)));
        it.clear();
        for (int t = 0; t < T; ++t)
            it.push_back(gi(src + t * mr, 1, m, c.R + t * rr, 1, r, dst + t * mr, m, m, r, r, 1.0, 0.0));
        MVN_TRY(bgemm(ctx, it, c.items));
        std::swap(src, dst);
    }
    // three passes: the result is in src (== Y after an odd number of swaps) -> copy to Q
    if (src != Q)
        MVN_CUDA(ctx, cudaMemcpyAsync(Q, src, sizeof(double) * mr * T, cudaMemcpyDeviceToDevice,
                                      ctx->stream));
    return MVN_OK;
}

// Compress T dense m x m tiles (A[t], ld m) into U[t], V[t] (m x kmax, ld m); ranks -> rank_out[t]
// (device), capped tiles counted into *capped_out (device).
static mvn_status comp_run(mvn_ctx* ctx, CompWs& c, int T, const std::vector<const double*>& A,
                           const std::vector<double*>& U, const std::vector<double*>& V,
                           double acc, uint64_t seed, int* rank_out, int r) {
    const int m = c.m, kmax = c.kmax;
    const size_t mr = (size_t)m * r, rr = (size_t)r * r;
    {
        std::vector<double*> pG(T), pR(T), pW(T), pWU(T), pWV(T), plam(T), pB(T);
        std::vector<int*> pord(T);
        for (int t = 0; t < T; ++t) {
            pG[t] = c.G + t * rr;
            pR[t] = c.R + t * rr;
            pW[t] = c.W + t * rr;
            pWU[t] = c.WU + (size_t)t * r * kmax;
            pWV[t] = c.WV + (size_t)t * r * kmax;
            plam[t] = c.lam + (size_t)t * r;
            pord[t] = c.order + (size_t)t * r;
            pB[t] = c.B + t * mr;
        }
        MVN_CUDA(ctx, cudaMemcpyAsync(c.pB, pB.data(), sizeof(void*) * T, cudaMemcpyHostToDevice, ctx->stream));
        MVN_CUDA(ctx, cudaMemcpyAsync(c.pG, pG.data(), sizeof(void*) * T, cudaMemcpyHostToDevice, ctx->stream));
        MVN_CUDA(ctx, cudaMemcpyAsync(c.pR, pR.data(), sizeof(void*) * T, cudaMemcpyHostToDevice, ctx->stream));
        MVN_CUDA(ctx, cudaMemcpyAsync(c.pW, pW.data(), sizeof(void*) * T, cudaMemcpyHostToDevice, ctx->stream));
        MVN_CUDA(ctx, cudaMemcpyAsync(c.pWU, pWU.data(), sizeof(void*) * T, cudaMemcpyHostToDevice, ctx->stream));
        MVN_CUDA(ctx, cudaMemcpyAsync(c.pWV, pWV.data(), sizeof(void*) * T, cudaMemcpyHostToDevice, ctx->stream));
        MVN_CUDA(ctx, cudaMemcpyAsync(c.plam, plam.data(), sizeof(void*) * T, cudaMemcpyHostToDevice, ctx->stream));
        MVN_CUDA(ctx, cudaMemcpyAsync(c.porder, pord.data(), sizeof(void*) * T, cudaMemcpyHostToDevice, ctx->stream));
    }
    k_gauss<<<(unsigned)((mr + 255) / 256), 256, 0, ctx->stream>>>(m, r, seed, c.Om);
    MVN_LAUNCHED(ctx);
    std::vector<GItem> it;
    // Y = A Omega
    for (int t = 0; t < T; ++t) it.push_back(gi(A[t], 1, m, c.Om, 1, m, c.Y + t * mr, m, m, r, m, 1.0, 0.0));
    MVN_TRY(bgemm(ctx, it, c.items));
    MVN_TRY(comp_orth(ctx, c, T, c.Y, c.Q, r));
    // one power iteration: Z = A^T Q, Q' = orth(Z), Y = A Q', Q = orth(Y)
    it.clear();
    for (int t = 0; t < T; ++t) it.push_back(gi(A[t], m, 1, c.Q + t * mr, 1, m, c.Z + t * mr, m, m, r, m, 1.0, 0.0));
    MVN_TRY(bgemm(ctx, it, c.items));
    MVN_TRY(comp_orth(ctx, c, T, c.Z, c.Q, r));
    it.clear();
    for (int t = 0; t < T; ++t) it.push_back(gi(A[t], 1, m, c.Q + t * mr, 1, m, c.Y + t * mr, m, m, r, m, 1.0, 0.0));
    MVN_TRY(bgemm(ctx, it, c.items));
    MVN_TRY(comp_orth(ctx, c, T, c.Y, c.Q, r));
    // X = A^T Q (m x r, ld m), the transpose of B = Q^T A; its one-sided Jacobi SVD gives
    // A ~= (Q G) Sigma V^T with V the rotated, normalised columns of X
    it.clear();
    for (int t = 0; t < T; ++t) it.push_back(gi(A[t], m, 1, c.Q + t * mr, 1, m, c.B + t * mr, m, m, r, m, 1.0, 0.0));
    MVN_TRY(bgemm(ctx, it, c.items));
    const double floor2 = (0.01 * acc) * (0.01 * acc);
    if (m <= 256) {
        MVN_TIMED(ctx, "k_jacobi1", (k_jacobi1<8><<<T, 256, 0, ctx->stream>>>(
                                        m, r, c.pB, c.pW, c.plam, c.porder, 40, floor2)));
    } else if (m <= 512) {
        MVN_TIMED(ctx, "k_jacobi1", (k_jacobi1<16><<<T, 256, 0, ctx->stream>>>(
                                        m, r, c.pB, c.pW, c.plam, c.porder, 40, floor2)));
    } else if (m <= 1024) {
        MVN_TIMED(ctx, "k_jacobi1", (k_jacobi1<32><<<T, 256, 0, ctx->stream>>>(
                                        m, r, c.pB, c.pW, c.plam, c.porder, 40, floor2)));
    } else {
        MVN_TIMED(ctx, "k_jacobi1", (k_jacobi1<0><<<T, 256, 0, ctx->stream>>>(
                                        m, r, c.pB, c.pW, c.plam, c.porder, 40, floor2)));
    }
    k_select1<<<T, 256, 0, ctx->stream>>>(r, kmax, acc, c.pW, c.plam, c.porder, c.pWU, c.pWV,
                                          rank_out, c.capped);
    MVN_LAUNCHED(ctx);
    // U = Q WU (m x kmax);  V = X WV (m x kmax)
    it.clear();
    for (int t = 0; t < T; ++t) it.push_back(gi(c.Q + t * mr, 1, m, c.WU + (size_t)t * r * kmax, 1, r, U[t], m, m, kmax, r, 1.0, 0.0));
    MVN_TRY(bgemm(ctx, it, c.items));
    it.clear();
    for (int t = 0; t < T; ++t) it.push_back(gi(c.B + t * mr, 1, m, c.WV + (size_t)t * r * kmax, 1, r, V[t], m, m, kmax, r, 1.0, 0.0));
    MVN_TRY(bgemm(ctx, it, c.items));
    return MVN_OK;
}

// Adaptive sketch size: every tile starts with r = 32 columns; a tile whose detected rank
// reaches r - 8 (the sketch may have missed singular values above acc) is compressed again with
// twice the columns, up to max_rank + 8.  ranks_h receives the final ranks (host), rank_dev the
// same on the device.  Synchronises once per round.
static mvn_status comp_adaptive(mvn_ctx* ctx, CompWs& c, int T, const std::vector<const double*>& A,
                                const std::vector<double*>& U, const std::vector<double*>& V,
                                double acc, uint64_t seed, int* rank_dev, int* ranks_h) {
    const int rmax = c.r;
    int r = std::min(rmax, 32);
    std::vector<int> todo(T);
    for (int t = 0; t < T; ++t) todo[t] = t;
    int* rk = c.rk;  // per-round ranks
    for (int round = 0; !todo.empty(); ++round) {
        const int Tn = (int)todo.size();
        std::vector<const double*> Ar(Tn);
        std::vector<double*> Ur(Tn), Vr(Tn);
        for (int t = 0; t < Tn; ++t) {
            Ar[t] = A[todo[t]];
            Ur[t] = U[todo[t]];
            Vr[t] = V[todo[t]];
        }
        MVN_TRY(comp_run(ctx, c, Tn, Ar, Ur, Vr, acc, seed + 7919u * round, rk, r));
        std::vector<int> got(Tn);
        MVN_CUDA(ctx, cudaMemcpyAsync(got.data(), rk, sizeof(int) * Tn, cudaMemcpyDeviceToHost,
                                      ctx->stream));
        MVN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
        std::vector<int> next;
        for (int t = 0; t < Tn; ++t) {
            ranks_h[todo[t]] = got[t];
            if (got[t] >= r - 8 && r < rmax) next.push_back(todo[t]);
        }
        todo.swap(next);
        r = std::min(rmax, 2 * r);
    }
    MVN_CUDA(ctx, cudaMemcpyAsync(rank_dev, ranks_h, sizeof(int) * T, cudaMemcpyHostToDevice,
                                  ctx->stream));
    MVN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    return MVN_OK;
}

// ---------------------------------------------------------------- ABI

static int tlr_chunk(int m, int r, int kmax) {
    const double per = (4.0 * m * r + 3.0 * r * r + 2.0 * r * kmax + (double)m * m) * 8.0;
    return (int)std::max(1.0, std::min(1024.0, 24e9 / per));
}

extern "C" mvn_status mvn_tlr_compress(mvn_ctx* ctx, int n, const double* Sigma, int64_t ld,
                                       int tile, double acc, int max_rank, mvn_tlr** out,
                                       int* max_rank_hit) {
    if (!ctx) return MVN_ERR_ARG;
    if (out) *out = nullptr;
    if (!out || n < 1 || !Sigma || ld < n || tile < 64 || tile % 64 != 0 || tile > 4096 ||
        !(acc >= 0.0) || max_rank < 1 || max_rank > tile)
        return mvn_fail(ctx, MVN_ERR_ARG,
                        "mvn_tlr_compress: invalid argument (tile a multiple of 64, 1 <= max_rank <= tile)");
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    mvn_tlr* T = new mvn_tlr();
    T->ctx = ctx;
    T->n = n;
    T->m = tile;
    T->nt = (n + tile - 1) / tile;
    T->npad = T->nt * tile;
    T->kmax = max_rank;
    T->acc = acc;
    const int m = tile, nt = T->nt;
    const int64_t ntri = (int64_t)nt * (nt - 1) / 2;
    if (cudaMalloc(&T->D, sizeof(double) * (size_t)m * m * nt) != cudaSuccess ||
        cudaMalloc(&T->U, sizeof(double) * (size_t)m * max_rank * std::max<int64_t>(ntri, 1)) != cudaSuccess ||
        cudaMalloc(&T->V, sizeof(double) * (size_t)m * max_rank * std::max<int64_t>(ntri, 1)) != cudaSuccess ||
        cudaMalloc(&T->rank, sizeof(int) * std::max<int64_t>(ntri, 1)) != cudaSuccess) {
        cudaGetLastError();
        mvn_tlr_free(T);
        return mvn_fail(ctx, MVN_ERR_OOM, "mvn_tlr_compress: allocation failed");
    }
    // diagonal tiles
    for (int i = 0; i < nt; ++i) {
        k_copy_tile<<<m, 256, 0, ctx->stream>>>(n, m, Sigma, ld, i, i, T->D + (size_t)i * m * m);
        MVN_LAUNCHED(ctx);
    }
    int capped = 0;
    T->rank_h.assign((size_t)ntri, 0);
    if (ntri > 0) {
        const int r = std::min(m, max_rank + 8);
        const int chunk = tlr_chunk(m, r, max_rank);
        const size_t need = comp_ws_bytes(m, r, max_rank, chunk) +
                            ws_round(sizeof(double) * (size_t)m * m * chunk) + 4096;
        MVN_TRY(ws_reserve(ctx, need));
        WsCarver wc(ctx->ws);
        double* Ad = wc.take<double>((size_t)m * m * chunk);
        CompWs c = comp_ws_carve(wc, m, r, max_rank, chunk);
        MVN_CUDA(ctx, cudaMemsetAsync(c.capped, 0, sizeof(int), ctx->stream));
        std::vector<std::pair<int, int>> tiles;
        for (int j = 0; j < nt; ++j)
            for (int i = j + 1; i < nt; ++i) tiles.push_back({i, j});
        for (size_t t0 = 0; t0 < tiles.size(); t0 += chunk) {
            const int Tn = (int)std::min<size_t>(chunk, tiles.size() - t0);
            std::vector<const double*> A(Tn);
            std::vector<double*> U(Tn), V(Tn);
            for (int t = 0; t < Tn; ++t) {
                const int i = tiles[t0 + t].first, j = tiles[t0 + t].second;
                double* dst = Ad + (size_t)t * m * m;
                k_copy_tile<<<m, 256, 0, ctx->stream>>>(n, m, Sigma, ld, i, j, dst);
                MVN_LAUNCHED(ctx);
                A[t] = dst;
                const int64_t idx = tri_index(i, j, nt);
                U[t] = T->U + (size_t)idx * m * max_rank;
                V[t] = T->V + (size_t)idx * m * max_rank;
            }
            // tiles are enumerated in column order, so the ranks land at tri_index order
            MVN_TRY(comp_adaptive(ctx, c, Tn, A, U, V, acc, 0x5EEDull + t0, T->rank + t0,
                                  T->rank_h.data() + t0));
        }
        MVN_CUDA(ctx, cudaMemcpyAsync(&capped, c.capped, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    }
    MVN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    T->capped = capped;
    if (max_rank_hit) *max_rank_hit = capped;
    *out = T;
    return MVN_OK;
}

extern "C" mvn_status mvn_tlr_cholesky(mvn_ctx* ctx, mvn_tlr* T, int* info) {
    if (!ctx || !T || T->factored) return mvn_fail(ctx, MVN_ERR_ARG, "mvn_tlr_cholesky: invalid object");
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    if (info) *info = 0;
    const int m = T->m, nt = T->nt, kmax = T->kmax;
    const size_t mk = (size_t)m * kmax, kk = (size_t)kmax * kmax, mm = (size_t)m * m;
    const int r = std::min(m, kmax + 8);
    const int chunk = std::min(std::max(nt - 1, 1), tlr_chunk(m, r, kmax));
    const size_t need = comp_ws_bytes(m, r, kmax, chunk) + ws_round(sizeof(double) * mm * chunk) +
                        ws_round(sizeof(double) * kk * nt) + ws_round(sizeof(double) * mk * nt) +
                        ws_round(sizeof(GItem) * (size_t)nt) + ws_round(sizeof(double*) * nt) + 8192;
    MVN_TRY(ws_reserve(ctx, need));
    WsCarver wc(ctx->ws);
    double* Ad = wc.take<double>(mm * chunk);
    double* X = wc.take<double>(kk * nt);
    double* Yb = wc.take<double>(mk * nt);
    GItem* items2 = wc.take<GItem>((size_t)nt);
    double** pV = wc.take<double*>(nt);
    CompWs c = comp_ws_carve(wc, m, r, kmax, chunk);
    MVN_CUDA(ctx, cudaMemsetAsync(c.capped, 0, sizeof(int), ctx->stream));
    auto Ut = [&](int i, int j) { return T->U + (size_t)tri_index(i, j, nt) * mk; };
    auto Vt = [&](int i, int j) { return T->V + (size_t)tri_index(i, j, nt) * mk; };
    auto rk = [&](int i, int j) { return T->rank_h[(size_t)tri_index(i, j, nt)]; };
    for (int k = 0; k < nt; ++k) {
        double* Dk = T->D + (size_t)k * mm;
        // D_kk -= sum_{l<k} U_kl (V_kl^T V_kl) U_kl^T   (GEMM sizes follow the actual ranks)
        if (k > 0) {
            std::vector<GItem> it;
            for (int l = 0; l < k; ++l)
                if (rk(k, l))
                    it.push_back(gi(Vt(k, l), m, 1, Vt(k, l), 1, m, X + (size_t)l * kk, kmax,
                                    rk(k, l), rk(k, l), m, 1.0, 0.0));
            MVN_TRY(bgemm(ctx, it, items2));
            it.clear();
            for (int l = 0; l < k; ++l)
                if (rk(k, l))
                    it.push_back(gi(Ut(k, l), 1, m, X + (size_t)l * kk, 1, kmax, Yb + (size_t)l * mk,
                                    m, m, rk(k, l), rk(k, l), 1.0, 0.0));
            MVN_TRY(bgemm(ctx, it, items2));
            for (int l = 0; l < k; ++l) {
                if (!rk(k, l)) continue;
                it.clear();
                it.push_back(gi(Yb + (size_t)l * mk, 1, m, Ut(k, l), m, 1, Dk, m, m, m, rk(k, l), -1.0, 1.0));
                MVN_TRY(bgemm(ctx, it, items2));
            }
        }
        MVN_TRY(chol_f64_launch(ctx, m, Dk, m));
        // off-diagonal tiles of column k, in chunks
        for (int i0 = k + 1; i0 < nt; i0 += chunk) {
            const int Tn = std::min(chunk, nt - i0);
            std::vector<GItem> it;
            for (int t = 0; t < Tn; ++t)  // A_ik = U_ik V_ik^T
                it.push_back(gi(Ut(i0 + t, k), 1, m, Vt(i0 + t, k), m, 1, Ad + (size_t)t * mm, m, m, m,
                                rk(i0 + t, k), 1.0, 0.0));
            MVN_TRY(bgemm(ctx, it, c.items));
            for (int l = 0; l < k; ++l) {
                if (!rk(k, l)) continue;
                it.clear();
                for (int t = 0; t < Tn; ++t)  // X_il = V_il^T V_kl
                    if (rk(i0 + t, l))
                        it.push_back(gi(Vt(i0 + t, l), m, 1, Vt(k, l), 1, m, X + (size_t)t * kk, kmax,
                                        rk(i0 + t, l), rk(k, l), m, 1.0, 0.0));
                MVN_TRY(bgemm(ctx, it, c.items));
                it.clear();
                for (int t = 0; t < Tn; ++t)  // Y_il = U_il X_il
                    if (rk(i0 + t, l))
                        it.push_back(gi(Ut(i0 + t, l), 1, m, X + (size_t)t * kk, 1, kmax,
                                        Yb + (size_t)t * mk, m, m, rk(k, l), rk(i0 + t, l), 1.0, 0.0));
                MVN_TRY(bgemm(ctx, it, c.items));
                it.clear();
                for (int t = 0; t < Tn; ++t)  // A_ik -= Y_il U_kl^T
                    if (rk(i0 + t, l))
                        it.push_back(gi(Yb + (size_t)t * mk, 1, m, Ut(k, l), m, 1, Ad + (size_t)t * mm,
                                        m, m, m, rk(k, l), -1.0, 1.0));
                MVN_TRY(bgemm(ctx, it, c.items));
            }
            std::vector<const double*> A(Tn);
            std::vector<double*> U(Tn), V(Tn);
            std::vector<double*> pv(Tn);
            for (int t = 0; t < Tn; ++t) {
                A[t] = Ad + (size_t)t * mm;
                U[t] = Ut(i0 + t, k);
                V[t] = Vt(i0 + t, k);
                pv[t] = V[t];
            }
            const int64_t idx0 = tri_index(i0, k, nt);  // the chunk's tiles are consecutive
            MVN_TRY(comp_adaptive(ctx, c, Tn, A, U, V, T->acc, 0xC0FFEEull + (uint64_t)k * 4096 + i0,
                                  T->rank + idx0, T->rank_h.data() + idx0));
            int rmaxc = 0;
            for (int t = 0; t < Tn; ++t) rmaxc = std::max(rmaxc, rk(i0 + t, k));
            if (rmaxc == 0) continue;
            // V_ik <- L_kk^-1 V_ik, blocked by 64 rows (columns up to the chunk's largest rank)
            MVN_CUDA(ctx, cudaMemcpyAsync(pV, pv.data(), sizeof(double*) * Tn, cudaMemcpyHostToDevice, ctx->stream));
            for (int r0 = 0; r0 < m; r0 += 64) {
                if (r0 > 0) {
                    it.clear();
                    for (int t = 0; t < Tn; ++t)
                        if (rk(i0 + t, k))
                            it.push_back(gi(Dk + r0, 1, m, V[t], 1, m, V[t] + r0, m, 64, rk(i0 + t, k),
                                            r0, -1.0, 1.0));
                    MVN_TRY(bgemm(ctx, it, c.items));
                }
                const int threads = Tn * kmax;
                MVN_TIMED(ctx, "k_trsm_block",
                          (k_trsm_block<<<(threads + 127) / 128, 128, 0, ctx->stream>>>(
                              m, kmax, Dk, r0, pV, Tn)));
            }
        }
    }
    MVN_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    T->factored = true;
    int inf = 0;
    mvn_status st = mvn_sync(ctx, &inf);
    if (info) *info = inf;
    return st;
}

// L (n x n, ld): diagonal tiles' lower parts and U V^T below; the strict upper part untouched.
__global__ void k_diag_out(int n, int m, const double* __restrict__ D, int ti, double* __restrict__ L,
                           int64_t ld) {
    const int c = blockIdx.x;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
        const int i = ti * m + r, j = ti * m + c;
        if (i < n && j < n && r >= c) L[i + (int64_t)j * ld] = D[r + (int64_t)c * m];
    }
}

extern "C" mvn_status mvn_tlr_to_dense(mvn_ctx* ctx, const mvn_tlr* T, double* L, int64_t ld) {
    if (!ctx || !T || !L || ld < T->n) return mvn_fail(ctx, MVN_ERR_ARG, "mvn_tlr_to_dense: invalid argument");
    MVN_CUDA(ctx, cudaSetDevice(ctx->device));
    const int m = T->m, nt = T->nt, n = T->n, kmax = T->kmax;
    for (int i = 0; i < nt; ++i) {
        k_diag_out<<<m, 256, 0, ctx->stream>>>(n, m, T->D + (size_t)i * m * m, i, L, ld);
        MVN_LAUNCHED(ctx);
    }
    const int64_t ntri = (int64_t)nt * (nt - 1) / 2;
    if (ntri == 0) return MVN_OK;
    MVN_TRY(ws_reserve(ctx, ws_round(sizeof(GItem) * (size_t)ntri) + 1024));
    std::vector<GItem> it;
    for (int j = 0; j < nt; ++j)
        for (int i = j + 1; i < nt; ++i) {
            const int64_t idx = tri_index(i, j, nt);
            const int rows = std::min(m, n - i * m), cols = std::min(m, n - j * m);
            it.push_back(gi(T->U + (size_t)idx * m * kmax, 1, m, T->V + (size_t)idx * m * kmax, m, 1,
                            L + (int64_t)i * m + (int64_t)j * m * ld, ld, rows, cols,
                            T->rank_h[(size_t)idx], 1.0, 0.0));
        }
    return bgemm(ctx, it, (GItem*)ctx->ws);
}

extern "C" mvn_status mvn_tlr_ranks(const mvn_tlr* T, int* ranks) {
    if (!T || !ranks) return MVN_ERR_ARG;
    std::copy(T->rank_h.begin(), T->rank_h.end(), ranks);
    return MVN_OK;
}

extern "C" mvn_status mvn_tlr_free(mvn_tlr* T) {
    if (!T) return MVN_ERR_ARG;
    if (T->ctx) cudaStreamSynchronize(T->ctx->stream);
    if (T->D) cudaFree(T->D);
    if (T->U) cudaFree(T->U);
    if (T->V) cudaFree(T->V);
    if (T->rank) cudaFree(T->rank);
    delete T;
    return MVN_OK;
}
