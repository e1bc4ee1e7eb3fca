// Dispatch of the MTTKRP and CP-model launches by factor type (the kernels
// live in mttkrp_kernels.cuh, instantiated per type in mttkrp_f32.cu,
// mttkrp_bf16.cu and mttkrp_f16.cu).
#include "mttkrp_kernels.cuh"

namespace blco {

bool rank_supported(int R) { return R == 8 || R == 16 || R == 32 || R == 64 || R == 128; }

int warp_tier_capacity(int R) { return rank_supported(R) ? warp_tier_rows(R) : 0; }

cudaError_t launch_mttkrp(const StoreView &sv, const FactorSet &fs, blco_dtype fdt, int R, int mode,
                          const HotRows &hot, float *out, bool compensated, cudaStream_t s) {
    switch (fdt) {
        case BLCO_F32: return launch_mttkrp_f32(sv, fs, R, mode, hot, out, s);
        case BLCO_BF16: return launch_mttkrp_bf16(sv, fs, R, mode, hot, out, compensated, s);
        case BLCO_F16: return launch_mttkrp_f16(sv, fs, R, mode, hot, out, compensated, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_cp_fwd(const StoreView &sv, const FactorSet &fs, blco_dtype fdt, int R, float *xhat,
                          int64_t xorigin, cudaStream_t s) {
    switch (fdt) {
        case BLCO_F32: return launch_cp_fwd_f32(sv, fs, R, xhat, xorigin, s);
        case BLCO_BF16: return launch_cp_fwd_bf16(sv, fs, R, xhat, xorigin, s);
        case BLCO_F16: return launch_cp_fwd_f16(sv, fs, R, xhat, xorigin, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace blco
