// MTTKRP and CP-model kernels for float factors.
#include "mttkrp_kernels.cuh"

namespace blco {

cudaError_t launch_mttkrp_f32(const StoreView &sv, const FactorSet &fs, int R, int mode, const HotRows &hot,
                          float *out, const OutCopies &oc, cudaStream_t s) {
    return mttkrp_as<float>(sv, fs, R, mode, hot, out, oc, false, s);
}

cudaError_t launch_cp_fwd_f32(const StoreView &sv, const FactorSet &fs, int R, float *xhat, int64_t xorigin,
                          cudaStream_t s) {
    return cp_fwd_as<float>(sv, fs, R, xhat, xorigin, s);
}

}  // namespace blco
