// Internal declarations shared by the translation units of libblco.so.
// (Not installed; the public interface is include/blco.h.)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "blco.h"

namespace blco {

constexpr int MAXN = BLCO_MAX_MODES;
constexpr uint32_t kNoRow = 0xFFFFFFFFu;  // never a valid index: I_n < 2^32

// ---------------------------------------------------------------------------
// Layout of the store (Sections 4.1-4.2), computed on the host at build time.
// ---------------------------------------------------------------------------
struct Layout {
    int N = 0;
    int64_t dims[MAXN] = {};
    int bits[MAXN] = {};      // b_n = ceil(log2 I_n)
    int B = 0;                // sum of b_n
    int line = 64;            // encoding line length L
    int kbits[MAXN] = {};     // bits of mode n above the line (block key bits)
    int width[MAXN] = {};     // in-block field width w_n = b_n - k_n
    int shift[MAXN] = {};     // in-block field offset (mode 0 lowest)
    int boff[MAXN] = {};      // offset of mode n's block bits in the packed block key
    uint8_t keypos[MAXN][32] = {};  // ALTO key position of (mode n, level l)
};

// Fills everything but dims/N/line from dims/N/line. Returns false if the
// shape is unsupported (B > 128 or more than 64 block-key bits).
bool plan_layout(Layout &L, std::string &why);

// View of (part of) a store for one kernel launch.
struct StoreView {
    const uint64_t *keys;   // in-block keys; keys[p - key_origin] for store position p
    int64_t key_origin;
    const float *vals;      // values (or an upstream gradient) in store order
    int64_t val_origin;
    const double *vals64;   // float64 values in store order (stores built with them)
    int64_t begin, end;     // store positions processed by this launch
    const uint32_t *tile_block;  // block that holds store position 32 * t
    const int64_t *bstart;       // nblocks + 1 block offsets
    const uint32_t *bbase;       // nblocks x MAXN: block high bits << field width
    int single_block;            // 1: one block with zero high bits (no lookups)
    int N;
    int64_t dims[MAXN];
    int shift[MAXN];
    uint64_t mask[MAXN];
};

struct FactorSet {
    const void *ptr[MAXN];
};

// Hot output rows of one mode (accumulated in shared memory).
struct HotRows {
    const uint32_t *rows;  // row ids by decreasing count (device)
    int count;             // rows available
    int dense;             // 1 = every row of the mode is accumulated on chip (slot == row)
};

// Private copies of a short mode's output: CTA b of a launch reduces into
// copy b % n (n == 1: into the output itself); the copies are summed into the
// output afterwards (launch_sum_copies).
struct OutCopies {
    int n = 1;
    int64_t stride = 0;  // floats between copies (I_mode * R)
};

// ----------------------------------------------------------------- kernels
// mttkrp.cu (dispatch by factor type). With 16-bit factors `compensated`
// selects Kahan-compensated run sums; float32 factors always sum plainly.
cudaError_t launch_mttkrp(const StoreView &sv, const FactorSet &fs, blco_dtype fdt, int R, int mode,
                          const HotRows &hot, float *out, const OutCopies &oc, bool compensated, cudaStream_t s);
int output_copies(int64_t I, int R);  // private output copies worth keeping for a mode (1 = none)
cudaError_t launch_cp_fwd(const StoreView &sv, const FactorSet &fs, blco_dtype fdt, int R,
                          float *xhat, int64_t xhat_origin, cudaStream_t s);
// mttkrp_f32.cu, mttkrp_bf16.cu, mttkrp_f16.cu (one factor type each)
cudaError_t launch_mttkrp_f32(const StoreView &sv, const FactorSet &fs, int R, int mode, const HotRows &hot,
                              float *out, const OutCopies &oc, cudaStream_t s);
cudaError_t launch_mttkrp_bf16(const StoreView &sv, const FactorSet &fs, int R, int mode, const HotRows &hot,
                               float *out, const OutCopies &oc, bool compensated, cudaStream_t s);
cudaError_t launch_mttkrp_f16(const StoreView &sv, const FactorSet &fs, int R, int mode, const HotRows &hot,
                              float *out, const OutCopies &oc, bool compensated, cudaStream_t s);
cudaError_t launch_cp_fwd_f32(const StoreView &sv, const FactorSet &fs, int R, float *xhat, int64_t xorigin,
                              cudaStream_t s);
cudaError_t launch_cp_fwd_bf16(const StoreView &sv, const FactorSet &fs, int R, float *xhat, int64_t xorigin,
                               cudaStream_t s);
cudaError_t launch_cp_fwd_f16(const StoreView &sv, const FactorSet &fs, int R, float *xhat, int64_t xorigin,
                              cudaStream_t s);
bool rank_supported(int R);
// All-mode MTTKRP in one pass (mttkrp_fused.cu): outs[n] for every mode with
// outs[n] != NULL; hot: per-mode hot rows. fused_supported tells whether the
// store's shape and the rank allow it (5 modes, every I_n <= 2^24,
// R = 16, 32 or 64).
bool fused_supported(const StoreView &sv, int R);
cudaError_t launch_mttkrp_fused(const StoreView &sv, const FactorSet &fs, blco_dtype fdt, int R, const HotRows *hot,
                                float *const *outs, cudaStream_t s);
// mttkrp_f64.cu: float64 values, factors and output
cudaError_t launch_mttkrp_f64(const StoreView &sv, const double *const *factors, int R, int mode, const HotRows &hot,
                              double *out, cudaStream_t s);
bool rank_supported_f64(int R);
int warp_tier_capacity_f64(int R);  // rows per launch accumulated on chip at rank R (float64)
int warp_tier_capacity(int R);  // rows per launch accumulated on chip (per-warp copies) at rank R

// build.cu
struct BuildOut {
    uint64_t *keys = nullptr;   // device, nnz (padded to a multiple of 32)
    float *vals = nullptr;      // device
    uint32_t *perm = nullptr;   // device
    std::vector<int64_t> bstart;
    std::vector<uint32_t> bhigh;  // nblocks x N
    int64_t first_bad = -1;       // first coordinate row out of range
};
// Runs linearize / sort / re-encode / block on the device. coords and vals
// are device pointers. Temporary memory via cudaMallocAsync on s.
cudaError_t build_store(const Layout &L, const uint32_t *coords, const float *vals, int64_t nnz,
                        int64_t cap, BuildOut &out, cudaStream_t s, std::string &why);
// dst[j] = src[perm[j]] for j < nnz (float64 values into store order)
cudaError_t gather_f64(const double *src, const uint32_t *perm, int64_t nnz, double *dst, cudaStream_t s);
cudaError_t build_tile_block(const int64_t *d_bstart, int64_t nblocks, int64_t nnz,
                             uint32_t *tile_block, cudaStream_t s);
// Per-mode index histogram of the store's nonzeros (counts: I_n uint32).
cudaError_t mode_histogram(const StoreView &sv, int mode, uint32_t *counts, cudaStream_t s);
// The `k` rows with the largest counts (ties: lower row id), sorted by row id.
cudaError_t top_rows(const uint32_t *counts, int64_t I, int k, uint32_t *rows_out, cudaStream_t s);

// dense.cu
cudaError_t launch_zero(float *p, int64_t n, cudaStream_t s);
cudaError_t launch_sum_copies(const float *copies, int ncopies, int64_t n, float *out, cudaStream_t s);
cudaError_t launch_convert(const float *src, void *dst, blco_dtype dt, int64_t n, cudaStream_t s);
cudaError_t launch_gram(const void *A, blco_dtype fdt, int64_t I, int R, double *G, cudaStream_t s);
cudaError_t launch_cpals_update(const double *const *grams, int N, int mode, int R, const float *M,
                                int64_t I, float *A, double *lambda, double *G_out, int32_t *info,
                                cudaStream_t s);
cudaError_t launch_cpals_fit(double normX2, const double *const *grams, int N, int R,
                             const double *lambda, const float *M, const float *A, int64_t I,
                             double *fit, cudaStream_t s);
cudaError_t launch_cpals_update_noalloc(const double *const *grams, int N, int mode, int R, const float *M,
                                        int64_t I, float *A, double *lambda, double *G_out, int32_t *info,
                                        cudaStream_t s);
int cpals_update_noalloc_max_rank();
cudaError_t launch_norm2(const float *v, int64_t n, double *out, cudaStream_t s);      // *out = sum v^2
cudaError_t launch_norm2_acc(const float *v, int64_t n, double *out, cudaStream_t s);  // *out += sum v^2

int sm_count();

}  // namespace blco
