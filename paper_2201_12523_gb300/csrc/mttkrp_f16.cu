// MTTKRP and CP-model kernels for __half factors.
#include "mttkrp_kernels.cuh"

namespace blco {

cudaError_t launch_mttkrp_f16(const StoreView &sv, const FactorSet &fs, int R, int mode, const HotRows &hot,
                          float *out, const OutCopies &oc, bool compensated, cudaStream_t s) {
    return mttkrp_as<__half>(sv, fs, R, mode, hot, out, oc, compensated, s);
}

cudaError_t launch_cp_fwd_f16(const StoreView &sv, const FactorSet &fs, int R, float *xhat, int64_t xorigin,
                          cudaStream_t s) {
    return cp_fwd_as<__half>(sv, fs, R, xhat, xorigin, s);
}

}  // namespace blco
