// mvn_sov.cuh -- internal SOV problem description shared by the sweep kernels.
#pragma once
#include <vector>

#include "mvn_internal.cuh"

// One MVN problem P(a <= X <= b), X ~ N(0, L L^T), on the shifted lattice rule.
struct SovProblem {
    int n;
    int M;                   // shifts
    int64_t Ns;              // points per shift
    int64_t Ntot;            // paths of this problem (M * Ns, or a shard's count)
    const double* a;         // n
    const double* b;         // n
    const double* L;         // lower factor, column-major
    int64_t ld;
    const uint64_t* delta;   // shifts, delta[q * dstride + i]
    int64_t dstride;         // row stride of the shift table (>= n)
    double* logw;            // Ntot per-path log-weights (output)
    int nprefix;             // optional prefix recording (Alg. 1 loop)
    const int* prefix;       // sorted prefix lengths in 1..n (device)
    double* logw_prefix;     // [t * Ntot + p]
    int64_t p0 = 0;          // lattice index of the first path (a shard of the rule: local path
                             // p is path p0 + p of the whole rule; 0 for a whole problem)
};

mvn_status check_qmc(mvn_ctx* ctx, const mvn_qmc* qmc);
mvn_status check_problem_host(mvn_ctx* ctx, int n, const double* a, const double* b,
                              const double* L, int64_t ld);
// Enqueue a device check of the limits (a_i <= b_i, no NaN); a violation raises MVN_ERR_ARG
// in the device status word (reported by mvn_sync).
mvn_status check_limits_device(mvn_ctx* ctx, int n, const double* a, const double* b);

// Bytes of workspace the CUDA-core sweep needs for `nprob` problems of max dimension nmax
// and `ntiles` path tiles in total.
size_t sov_simt_ws_bytes(mvn_ctx* ctx, int nprob, int nmax, int64_t ntiles, mvn_prec prec);
// Run the sweep for a list of problems (host descriptors with device pointers).  `ws` must hold
// sov_simt_ws_bytes(...) bytes.  A single problem needs no host-to-device copy (asynchronous).
mvn_status sov_run_simt(mvn_ctx* ctx, const std::vector<SovProblem>& probs, mvn_prec prec,
                        char* ws);

// Tensor-core sweep (mvn_sov_tc.cu): all problems must share one factor.
size_t sov_tc_ws_bytes(mvn_ctx* ctx, int nprob, int nmax, int64_t ntiles);
mvn_status sov_run_tc(mvn_ctx* ctx, const std::vector<SovProblem>& probs, char* ws);

// Dispatch between the tensor-core sweep (MVN_MIXED) and the CUDA-core sweep.
size_t sov_any_ws_bytes(mvn_ctx* ctx, int nprob, int nmax, int64_t ntiles, mvn_prec prec);
mvn_status sov_run_any(mvn_ctx* ctx, const std::vector<SovProblem>& probs, mvn_prec prec,
                       char* ws);
