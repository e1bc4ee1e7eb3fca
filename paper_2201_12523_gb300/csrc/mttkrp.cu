// Sparse MTTKRP (Eq. 1, Fig. 3) and the CP model at the nonzeros over a
// BLCO store, for sm_103a.
//
// One warp owns a tile of 32 consecutive nonzeros of the store:
//   1. each lane loads one nonzero's key and value (streaming loads) and
//      de-linearizes it by shift and mask (Section 4.1, Fig. 6b), adding the
//      block's high bits from the block table (Section 4.2);
//   2. the warp groups lanes with equal target row i_n with __match_any_sync
//      and orders the 32 nonzeros so that each group is contiguous (a
//      counting sort by group leader, done with one warp scan) -- this takes
//      the place of the paper's per-tile histogram + prefix-sum reordering
//      (Section 5.1, processing phase);
//   3. lanes are re-assigned across the rank: G = R*sizeof(T)/16 lanes per
//      nonzero, each lane loading 16 bytes of every gathered factor row, so
//      P = 32/G nonzeros are in flight per step and each warp load moves
//      whole 128-byte rows; subgroup g walks the sorted positions
//      [g*G, g*G+G) and keeps a running float32 sum while the target row
//      stays the same (Section 5.1, computing phase);
//   4. at the end of a run the sum goes either to the CTA's shared-memory
//      accumulator of that row (the mode's hot rows, found at build time from
//      a histogram, or every row when the whole mode fits), or straight to
//      global memory with one vector red.global.add.v4.f32 per lane
//      (Section 5.2's register-based path); at the end of the CTA the
//      shared accumulators are added to global memory once (Section 5.1's
//      local stash + final merge, with Section 5.3's choice replaced by the
//      per-row hot/cold split).
// The grid is persistent (a multiple of the SM count); warps stride over the
// tiles so that the warps running at any moment cover a narrow window of the
// ALTO order and share factor rows in L2.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "internal.h"

namespace blco {
namespace {

constexpr int kThreads = 512;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kHotBytes = 64 * 1024;

// The key/value stream is read once per launch: cache-streaming loads
// (evict-first) keep it from displacing factor rows in L1/L2.
__device__ __forceinline__ uint64_t ld_stream_u64(const uint64_t *p) {
    return (uint64_t)__ldcs(reinterpret_cast<const unsigned long long *>(p));
}
__device__ __forceinline__ float ld_stream_f32(const float *p) { return __ldcs(p); }

__device__ __forceinline__ void red_add_v4(float *addr, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c),
                 "f"(d)
                 : "memory");
}

// 16 bytes of a factor row -> VEC floats.
template <typename T>
struct Row;

template <>
struct Row<float> {
    static constexpr int VEC = 4;
    __device__ __forceinline__ static void load(const void *base, size_t elem, float (&f)[VEC]) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(static_cast<const float *>(base) + elem));
        f[0] = v.x;
        f[1] = v.y;
        f[2] = v.z;
        f[3] = v.w;
    }
};

// bfloat16 -> float32 is exact: the 16 bits become the top half of the word.
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

template <>
struct Row<__nv_bfloat16> {
    static constexpr int VEC = 8;
    __device__ __forceinline__ static void load(const void *base, size_t elem, float (&f)[VEC]) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(static_cast<const __nv_bfloat16 *>(base) + elem));
        f[0] = bf16_lo(v.x);
        f[1] = bf16_hi(v.x);
        f[2] = bf16_lo(v.y);
        f[3] = bf16_hi(v.y);
        f[4] = bf16_lo(v.z);
        f[5] = bf16_hi(v.z);
        f[6] = bf16_lo(v.w);
        f[7] = bf16_hi(v.w);
    }
};

template <>
struct Row<__half> {
    static constexpr int VEC = 8;
    __device__ __forceinline__ static void load(const void *base, size_t elem, float (&f)[VEC]) {
        const uint4 v = __ldg(reinterpret_cast<const uint4 *>(static_cast<const __half *>(base) + elem));
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            __half2 h = *reinterpret_cast<const __half2 *>(&w[i]);
            float2 t = __half22float2(h);
            f[2 * i] = t.x;
            f[2 * i + 1] = t.y;
        }
    }
};

// Section 4.1/4.2: i_n = ((key >> shift_n) & mask_n) + (block high bits << w_n).
__device__ __forceinline__ void delinearize(const StoreView &sv, uint64_t key, int64_t pos, bool valid,
                                            uint32_t (&idx)[MAXN]) {
    uint32_t base[MAXN];
#pragma unroll
    for (int k = 0; k < MAXN; ++k) base[k] = 0;
    if (!sv.single_block && valid) {
        uint32_t b = __ldg(sv.tile_block + (pos >> 5));
        while (pos >= __ldg(sv.bstart + b + 1)) ++b;
        const uint32_t *bb = sv.bbase + (size_t)b * MAXN;
#pragma unroll
        for (int k = 0; k < MAXN; ++k)
            if (k < sv.N) base[k] = __ldg(bb + k);
    }
#pragma unroll
    for (int k = 0; k < MAXN; ++k)
        idx[k] = (k < sv.N) ? (uint32_t)((key >> sv.shift[k]) & sv.mask[k]) + base[k] : 0u;
}

struct WarpStage {
    uint32_t idx[MAXN][32];
    float val[32];
};

__device__ __forceinline__ uint32_t hot_hash(uint32_t row, int log2ts) {
    return (row * 0x9E3779B1u) >> (32 - log2ts);
}

// -------------------------------------------------------------------------
// MTTKRP
// -------------------------------------------------------------------------
template <typename T, int R>
__global__ void __launch_bounds__(kThreads, 2)
    k_mttkrp(const StoreView sv, const FactorSet fs, const HotRows hot, const int hot_n, const int log2ts,
             float *__restrict__ out, const int mode) {
    constexpr int VEC = Row<T>::VEC;
    constexpr int G = R / VEC;   // lanes per nonzero
    static_assert(G >= 1 && G <= 32 && (32 % G) == 0, "rank must give 1..32 lanes per row");
    constexpr int STEPS = G;     // sorted positions per subgroup (P = 32 / G subgroups)
    constexpr int RS = R + 4;    // shared accumulator row stride (bank spread, 16B aligned)

    extern __shared__ __align__(16) unsigned char smem[];
    WarpStage *stage = reinterpret_cast<WarpStage *>(smem);
    float *acc = reinterpret_cast<float *>(smem + sizeof(WarpStage) * kWarps);
    const int ts = (hot_n > 0 && !hot.dense) ? (1 << log2ts) : 0;
    uint32_t *tkey = reinterpret_cast<uint32_t *>(acc + (size_t)hot_n * RS);
    uint32_t *tslot = tkey + ts;

    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int g = lane / G;
    const int c = lane % G;
    WarpStage &st = stage[wid];

    // --- shared accumulators of the hot rows: zero them, build the hash table
    for (int i = threadIdx.x; i < hot_n * RS; i += kThreads) acc[i] = 0.f;
    for (int i = threadIdx.x; i < ts; i += kThreads) tkey[i] = kNoRow;
    __syncthreads();
    if (ts > 0) {
        // open addressing, linear probing; the table has 2x more slots than
        // rows, so every insertion finds a free slot within ts probes
        for (int i = threadIdx.x; i < hot_n; i += kThreads) {
            const uint32_t row = __ldg(hot.rows + i);
            uint32_t h = hot_hash(row, log2ts);
            for (int probe = 0; probe < ts; ++probe) {
                if (atomicCAS(&tkey[h], kNoRow, row) == kNoRow) {
                    tslot[h] = (uint32_t)i;
                    break;
                }
                h = (h + 1) & (ts - 1);
            }
        }
    }
    __syncthreads();

    const int64_t span = sv.end - sv.begin;
    const int64_t ntiles = (span + 31) >> 5;
    const int64_t wstride = (int64_t)gridDim.x * kWarps;
    int64_t tile = (int64_t)blockIdx.x * kWarps + wid;

    uint64_t key = 0;
    float val = 0.f;
    {
        const int64_t pos = sv.begin + tile * 32 + lane;
        if (tile < ntiles && pos < sv.end) {
            key = ld_stream_u64(sv.keys + (pos - sv.key_origin));
            val = ld_stream_f32(sv.vals + (pos - sv.val_origin));
        }
    }
    while (tile < ntiles) {
        const int64_t pos = sv.begin + tile * 32 + lane;
        const bool valid = pos < sv.end;
        // prefetch the next tile's stream entries
        const int64_t ntile = tile + wstride;
        uint64_t nkey = 0;
        float nval = 0.f;
        {
            const int64_t npos = sv.begin + ntile * 32 + lane;
            if (ntile < ntiles && npos < sv.end) {
                nkey = ld_stream_u64(sv.keys + (npos - sv.key_origin));
                nval = ld_stream_f32(sv.vals + (npos - sv.val_origin));
            }
        }

        uint32_t idx[MAXN];
        delinearize(sv, key, pos, valid, idx);
        uint32_t t = kNoRow;
#pragma unroll
        for (int k = 0; k < MAXN; ++k)
            if (k == mode) t = idx[k];
        if (!valid) t = kNoRow;

        // --- group equal target rows; counting sort of the groups by leader
        const unsigned peers = __match_any_sync(kFull, t);
        const int leader = __ffs(peers) - 1;
        const unsigned mine = (lane == leader) ? (unsigned)__popc(peers) : 0u;
        unsigned incl = mine;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned y = __shfl_up_sync(kFull, incl, d);
            if (lane >= d) incl += y;
        }
        const unsigned seg_base = __shfl_sync(kFull, incl - mine, leader);
        const unsigned spos = seg_base + __popc(peers & ((1u << lane) - 1u));
        const unsigned heads = __reduce_or_sync(kFull, lane == leader ? (1u << seg_base) : 0u);
        const int nvalid = __popc(__ballot_sync(kFull, valid));

#pragma unroll
        for (int k = 0; k < MAXN; ++k)
            if (k < sv.N) st.idx[k][spos] = idx[k];
        st.val[spos] = val;
        __syncwarp();

        // --- rank-parallel products and run-length accumulation
        float sum[VEC];
#pragma unroll
        for (int e = 0; e < VEC; ++e) sum[e] = 0.f;
#pragma unroll
        for (int step = 0; step < STEPS; ++step) {
            const int s = g * STEPS + step;
            const float v = st.val[s];
            float p[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) p[e] = v;
#pragma unroll
            for (int k = 0; k < MAXN; ++k) {
                if (k < sv.N && k != mode) {
                    float f[VEC];
                    Row<T>::load(fs.ptr[k], (size_t)st.idx[k][s] * R + c * VEC, f);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) p[e] *= f[e];
                }
            }
#pragma unroll
            for (int e = 0; e < VEC; ++e) sum[e] += p[e];
            const bool run_end = (s == 31) || ((heads >> (s + 1)) & 1u) || (step == STEPS - 1);
            if (run_end) {
                if (s < nvalid) {
                    const uint32_t row = st.idx[mode][s];
                    int slot = -1;
                    if (hot_n > 0) {
                        if (hot.dense) {
                            slot = (int)row;
                        } else {
                            uint32_t h = hot_hash(row, log2ts);
                            for (int probe = 0; probe < ts; ++probe) {
                                const uint32_t kk = tkey[h];
                                if (kk == row) {
                                    slot = (int)tslot[h];
                                    break;
                                }
                                if (kk == kNoRow) break;
                                h = (h + 1) & (ts - 1);
                            }
                        }
                    }
                    if (slot >= 0) {
                        float *a = acc + (size_t)slot * RS + c * VEC;
#pragma unroll
                        for (int e = 0; e < VEC; ++e) atomicAdd(a + e, sum[e]);
                    } else {
                        float *o = out + (size_t)row * R + c * VEC;
#pragma unroll
                        for (int e = 0; e < VEC; e += 4) red_add_v4(o + e, sum[e], sum[e + 1], sum[e + 2], sum[e + 3]);
                    }
                }
#pragma unroll
                for (int e = 0; e < VEC; ++e) sum[e] = 0.f;
            }
        }
        __syncwarp();
        tile = ntile;
        key = nkey;
        val = nval;
    }

    // --- add the CTA's shared accumulators to the output once
    if (hot_n > 0) {
        __syncthreads();
        constexpr int Q = R / 4;
        for (int i = threadIdx.x; i < hot_n * Q; i += kThreads) {
            const int slot = i / Q, q = i % Q;
            const uint32_t row = hot.dense ? (uint32_t)slot : __ldg(hot.rows + slot);
            const float4 v = *reinterpret_cast<const float4 *>(acc + (size_t)slot * RS + q * 4);
            if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f)
                red_add_v4(out + (size_t)row * R + q * 4, v.x, v.y, v.z, v.w);
        }
    }
}

// -------------------------------------------------------------------------
// CP model at the nonzeros: xhat = sum_r prod_n A_n[i_n, r]
// -------------------------------------------------------------------------
template <typename T, int R>
__global__ void __launch_bounds__(kThreads, 2)
    k_cp_fwd(const StoreView sv, const FactorSet fs, float *__restrict__ xhat, const int64_t xorigin) {
    constexpr int VEC = Row<T>::VEC;
    constexpr int G = R / VEC;
    constexpr int STEPS = G;
    __shared__ WarpStage stage[kWarps];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int g = lane / G;
    const int c = lane % G;
    WarpStage &st = stage[wid];
    const int64_t span = sv.end - sv.begin;
    const int64_t ntiles = (span + 31) >> 5;
    const int64_t wstride = (int64_t)gridDim.x * kWarps;
    for (int64_t tile = (int64_t)blockIdx.x * kWarps + wid; tile < ntiles; tile += wstride) {
        const int64_t pos = sv.begin + tile * 32 + lane;
        const bool valid = pos < sv.end;
        uint64_t key = valid ? ld_stream_u64(sv.keys + (pos - sv.key_origin)) : 0ull;
        uint32_t idx[MAXN];
        delinearize(sv, key, pos, valid, idx);
#pragma unroll
        for (int k = 0; k < MAXN; ++k)
            if (k < sv.N) st.idx[k][lane] = idx[k];
        __syncwarp();
#pragma unroll
        for (int step = 0; step < STEPS; ++step) {
            const int s = g * STEPS + step;
            float p[VEC];
#pragma unroll
            for (int e = 0; e < VEC; ++e) p[e] = 1.f;
#pragma unroll
            for (int k = 0; k < MAXN; ++k) {
                if (k < sv.N) {
                    float f[VEC];
                    Row<T>::load(fs.ptr[k], (size_t)st.idx[k][s] * R + c * VEC, f);
#pragma unroll
                    for (int e = 0; e < VEC; ++e) p[e] *= f[e];
                }
            }
            float part = 0.f;
#pragma unroll
            for (int e = 0; e < VEC; ++e) part += p[e];
#pragma unroll
            for (int o = G / 2; o >= 1; o >>= 1) part += __shfl_xor_sync(kFull, part, o);
            if (c == 0) st.val[s] = part;
        }
        __syncwarp();
        if (valid) xhat[pos - xorigin] = st.val[lane];
        __syncwarp();
    }
}

// -------------------------------------------------------------------------
// launch helpers
// -------------------------------------------------------------------------
template <typename T, int R>
int hot_capacity_t() {
    constexpr int RS = R + 4;
    int h = 1;
    while ((h * 2) * RS * 4 <= kHotBytes) h *= 2;
    return h;
}

template <typename T, int R>
cudaError_t run_mttkrp(const StoreView &sv, const FactorSet &fs, int mode, const HotRows &hot,
                       float *out, cudaStream_t s) {
    int hot_n = 0, log2ts = 0;
    const int cap = hot_capacity_t<T, R>();
    if (hot.count > 0) {
        hot_n = hot.count < cap ? hot.count : cap;
        if (!hot.dense) {
            while ((1 << log2ts) < 2 * hot_n) ++log2ts;
        }
    }
    const int ts = (hot_n > 0 && !hot.dense) ? (1 << log2ts) : 0;
    const size_t shm = sizeof(WarpStage) * kWarps + (size_t)hot_n * (R + 4) * sizeof(float) +
                       (size_t)ts * 2 * sizeof(uint32_t);
    auto kern = k_mttkrp<T, R>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, shm);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int64_t tiles = (sv.end - sv.begin + 31) / 32;
    int64_t grid = (int64_t)sm_count() * per_sm;
    const int64_t need = (tiles + kWarps - 1) / kWarps;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kThreads, shm, s>>>(sv, fs, hot, hot_n, log2ts, out, mode);
    return cudaGetLastError();
}

template <typename T, int R>
cudaError_t run_cp_fwd(const StoreView &sv, const FactorSet &fs, float *xhat, int64_t xorigin, cudaStream_t s) {
    auto kern = k_cp_fwd<T, R>;
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int64_t tiles = (sv.end - sv.begin + 31) / 32;
    int64_t grid = (int64_t)sm_count() * per_sm;
    const int64_t need = (tiles + kWarps - 1) / kWarps;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    kern<<<(unsigned)grid, kThreads, 0, s>>>(sv, fs, xhat, xorigin);
    return cudaGetLastError();
}

template <typename T>
cudaError_t dispatch_mttkrp(const StoreView &sv, const FactorSet &fs, int R, int mode, const HotRows &hot,
                            float *out, cudaStream_t s) {
    switch (R) {
        case 8: return run_mttkrp<T, 8>(sv, fs, mode, hot, out, s);
        case 16: return run_mttkrp<T, 16>(sv, fs, mode, hot, out, s);
        case 32: return run_mttkrp<T, 32>(sv, fs, mode, hot, out, s);
        case 64: return run_mttkrp<T, 64>(sv, fs, mode, hot, out, s);
        case 128: return run_mttkrp<T, 128>(sv, fs, mode, hot, out, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t dispatch_cp_fwd(const StoreView &sv, const FactorSet &fs, int R, float *xhat, int64_t xo,
                            cudaStream_t s) {
    switch (R) {
        case 8: return run_cp_fwd<T, 8>(sv, fs, xhat, xo, s);
        case 16: return run_cp_fwd<T, 16>(sv, fs, xhat, xo, s);
        case 32: return run_cp_fwd<T, 32>(sv, fs, xhat, xo, s);
        case 64: return run_cp_fwd<T, 64>(sv, fs, xhat, xo, s);
        case 128: return run_cp_fwd<T, 128>(sv, fs, xhat, xo, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

bool rank_supported(int R) { return R == 8 || R == 16 || R == 32 || R == 64 || R == 128; }

int mttkrp_hot_capacity(int R) {
    switch (R) {
        case 8: return hot_capacity_t<float, 8>();
        case 16: return hot_capacity_t<float, 16>();
        case 32: return hot_capacity_t<float, 32>();
        case 64: return hot_capacity_t<float, 64>();
        case 128: return hot_capacity_t<float, 128>();
    }
    return 0;
}

cudaError_t launch_mttkrp(const StoreView &sv, const FactorSet &fs, blco_dtype fdt, int R, int mode,
                          const HotRows &hot, float *out, cudaStream_t s) {
    if (sv.end <= sv.begin) return cudaSuccess;
    switch (fdt) {
        case BLCO_F32: return dispatch_mttkrp<float>(sv, fs, R, mode, hot, out, s);
        case BLCO_BF16: return dispatch_mttkrp<__nv_bfloat16>(sv, fs, R, mode, hot, out, s);
        case BLCO_F16: return dispatch_mttkrp<__half>(sv, fs, R, mode, hot, out, s);
    }
    return cudaErrorInvalidValue;
}

cudaError_t launch_cp_fwd(const StoreView &sv, const FactorSet &fs, blco_dtype fdt, int R, float *xhat,
                          int64_t xorigin, cudaStream_t s) {
    if (sv.end <= sv.begin) return cudaSuccess;
    switch (fdt) {
        case BLCO_F32: return dispatch_cp_fwd<float>(sv, fs, R, xhat, xorigin, s);
        case BLCO_BF16: return dispatch_cp_fwd<__nv_bfloat16>(sv, fs, R, xhat, xorigin, s);
        case BLCO_F16: return dispatch_cp_fwd<__half>(sv, fs, R, xhat, xorigin, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace blco
