// Dispatch of the MTTKRP and CP-model launches by factor type (the kernels
// live in mttkrp_kernels.cuh, instantiated per type in mttkrp_f32.cu,
// mttkrp_bf16.cu and mttkrp_f16.cu).
#include "mttkrp_kernels.cuh"

namespace blco {

bool rank_supported(int R) { return R == 8 || R == 16 || R == 32 || R == 64 || R == 128; }

int warp_tier_capacity(int R) { return rank_supported(R) ? warp_tier_rows(R) : 0; }

cudaError_t launch_mttkrp(const StoreView &sv, const FactorSet &fs, blco_dtype fdt, int R, int mode,
                          const HotRows &hot, float *out, const OutCopies &oc, bool compensated, cudaStream_t s) {
    switch (fdt) {
        case BLCO_F32: return launch_mttkrp_f32(sv, fs, R, mode, hot, out, oc, s);
        case BLCO_BF16: return launch_mttkrp_bf16(sv, fs, R, mode, hot, out, oc, compensated, s);
        case BLCO_F16: return launch_mttkrp_f16(sv, fs, R, mode, hot, out, oc, compensated, s);
    }
    return cudaErrorInvalidValue;
}

// A short mode's output receives most of a launch's reductions on few rows;
// private copies spread them. Measured on GB300: at R = 64 (16 rows per warp
// on chip, 16 vector reductions per nonzero) a 1024-row mode ran 18% faster
// with one copy per SM and 21% faster with 16 copies (less L2 taken from the
// factor-row gathers); at R = 32 (32 rows on chip) 256- and 2048-row modes
// gained nothing with 16, 32 or 152 copies. So: 16 copies from R = 64, while
// they fit in 48 MB and the mode is not held on chip entirely (the per-warp
// copies cover modes of at most 1024 / R rows).
int output_copies(int64_t I, int R) {
    constexpr int kCopies = 16;
    const int64_t bytes = I * (int64_t)R * (int64_t)sizeof(float);
    if (R < 64 || I <= warp_tier_capacity(R) || bytes * kCopies > ((int64_t)48 << 20)) return 1;
    return kCopies;
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
