// mvn_tlr.cuh -- the tile low-rank object (Sec. III-E) shared by the TLR kernels and the
// low-rank sweep (not part of the ABI).
#pragma once
#include <stdint.h>

#include <vector>

#include "mvn_internal.cuh"

struct mvn_tlr {
    mvn_ctx* ctx = nullptr;
    int n = 0, npad = 0, m = 0, nt = 0, kmax = 0;
    double acc = 0.0;
    double* D = nullptr;  // nt diagonal tiles, m x m (ld m)
    double* U = nullptr;  // ntri tiles, m x kmax (ld m), columns >= rank are zero
    double* V = nullptr;
    int* rank = nullptr;  // device, ntri
    std::vector<int> rank_h;
    int capped = 0;
    bool factored = false;
};

static inline int64_t tri_index(int i, int j, int nt) {  // i > j, column order
    return (int64_t)j * nt - (int64_t)j * (j + 1) / 2 + (i - j - 1);
}

