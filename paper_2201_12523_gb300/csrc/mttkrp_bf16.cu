// MTTKRP and CP-model kernels for __nv_bfloat16 factors.
#include "mttkrp_kernels.cuh"

namespace blco {

cudaError_t launch_mttkrp_bf16(const StoreView &sv, const FactorSet &fs, int R, int mode, const HotRows &hot,
                          float *out, const OutCopies &oc, bool compensated, cudaStream_t s) {
    return mttkrp_as<__nv_bfloat16>(sv, fs, R, mode, hot, out, oc, compensated, s);
}

cudaError_t launch_cp_fwd_bf16(const StoreView &sv, const FactorSet &fs, int R, float *xhat, int64_t xorigin,
                          cudaStream_t s) {
    return cp_fwd_as<__nv_bfloat16>(sv, fs, R, xhat, xorigin, s);
}

}  // namespace blco
