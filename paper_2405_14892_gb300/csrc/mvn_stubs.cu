// mvn_stubs.cu -- entry points declared in mvn.h whose kernels are not built yet.
#include "mvn_internal.cuh"

extern "C" mvn_status mvn_tlr_compress(mvn_ctx* ctx, int, const double*, int64_t, int, double,
                                       int, mvn_tlr** out, int*) {
    if (out) *out = nullptr;
    return mvn_fail(ctx, MVN_ERR_NOT_IMPLEMENTED, "mvn_tlr_compress: not implemented");
}
extern "C" mvn_status mvn_tlr_cholesky(mvn_ctx* ctx, mvn_tlr*, int*) {
    return mvn_fail(ctx, MVN_ERR_NOT_IMPLEMENTED, "mvn_tlr_cholesky: not implemented");
}
extern "C" mvn_status mvn_tlr_to_dense(mvn_ctx* ctx, const mvn_tlr*, double*, int64_t) {
    return mvn_fail(ctx, MVN_ERR_NOT_IMPLEMENTED, "mvn_tlr_to_dense: not implemented");
}
extern "C" mvn_status mvn_tlr_ranks(const mvn_tlr*, int*) { return MVN_ERR_NOT_IMPLEMENTED; }
extern "C" mvn_status mvn_tlr_free(mvn_tlr*) { return MVN_OK; }
