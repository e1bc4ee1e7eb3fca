// Sparse MTTKRP (Eq. 1) with float64 values, factors and accumulation -- the
// precision of the paper's evaluation (Section 6) -- over a BLCO store built
// with float64 values. Same tile scheme as the float32 kernel
// (mttkrp_kernels.cuh): one warp per 32 consecutive stored nonzeros, a
// __match_any_sync counting sort of the tile by target row, G = R / 2 lanes
// per nonzero each holding two elements of every gathered row (one 16-byte
// load), running sums per run of equal target rows, the mode's hottest rows
// in per-warp shared-memory copies (float64) and every other row reduced
// into global memory with red.global.add.f64.
#include "mttkrp_kernels.cuh"

namespace blco {
namespace {

__device__ __forceinline__ void red_add_f64(double *addr, double v) {
    asm volatile("red.global.add.f64 [%0], %1;" ::"l"(addr), "d"(v));
}

template <int NG>
struct Stage64 {
    uint32_t idx[gather_slots<NG>()][32];
    double val[32];
    uint2 rs[32];  // (row, slot)
};

// Per-warp float64 copies of the hot rows: 4 KB per warp, as the float32 kernel.
constexpr int kWarpTierBytes64 = 4 * 1024;
int warp_tier_rows64(int R) { return kWarpTierBytes64 / (R * (int)sizeof(double)); }

struct SmemLayout64 {
    size_t wacc, table, total;
};
__host__ __device__ __forceinline__ SmemLayout64 smem_layout64(size_t stage_bytes, int kw, int R, int nb) {
    SmemLayout64 L;
    L.wacc = align16(stage_bytes * kWarps);
    L.table = align16(L.wacc + (size_t)kWarps * (kw + 1) * R * sizeof(double));
    L.total = align16(L.table + (size_t)nb * sizeof(uint4));
    return L;
}

template <int R, int NG>
__global__ void __launch_bounds__(kThreads, 2) k_mttkrp64(const KParams p, const double *__restrict__ vals64,
                                                           double *__restrict__ out) {
    constexpr int G = R / 2;  // lanes per nonzero, two elements each
    static_assert(G >= 1 && G <= 32 && (32 % G) == 0, "rank must give 1..32 lanes per row");
    constexpr int STEPS = G;
    constexpr int CH = STEPS < 4 ? STEPS : 4;  // positions per register batch
    constexpr int NS = gather_slots<NG>();

    extern __shared__ __align__(16) unsigned char smem[];
    const int kw = p.kw;
    const int nb = p.log2nb >= 0 ? (1 << p.log2nb) : 0;
    const SmemLayout64 L = smem_layout64(sizeof(Stage64<NG>), kw, R, nb);
    Stage64<NG> *stage = reinterpret_cast<Stage64<NG> *>(smem);
    double *wacc_all = reinterpret_cast<double *>(smem + L.wacc);
    uint4 *table = reinterpret_cast<uint4 *>(smem + L.table);

    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int g = lane / G;
    const int c = lane % G;
    Stage64<NG> &st = stage[wid];
    double *wacc = wacc_all + (size_t)wid * (kw + 1) * R;
    const int ng = n_gather<NG>(p);

    for (int i = threadIdx.x; i < kWarps * (kw + 1) * R; i += kThreads) wacc_all[i] = 0.0;
    for (int i = threadIdx.x; i < nb; i += kThreads) table[i] = make_uint4(kNoRow, 0u, kNoRow, 0u);
    __syncthreads();
    if (nb > 0 && threadIdx.x == 0) {
        for (int i = 0; i < kw; ++i) {
            const uint32_t row = __ldg(p.hot_rows + i);
            uint4 &bk = table[hot_hash(row, p.log2nb)];
            if (bk.x == kNoRow) {
                bk.x = row;
                bk.y = (uint32_t)i;
            } else if (bk.z == kNoRow) {
                bk.z = row;
                bk.w = (uint32_t)i;
            }
        }
    }
    __syncthreads();

    const int64_t ntiles = (p.end - p.begin + 31) >> 5;
    const int64_t wstride = (int64_t)gridDim.x * kWarps;
    for (int64_t tile = (int64_t)blockIdx.x * kWarps + wid; tile < ntiles; tile += wstride) {
        const int64_t pos = p.begin + tile * 32 + lane;
        const bool valid = pos < p.end;
        uint64_t key = valid ? ld_stream_u64(p.keys + (pos - p.key_origin)) : 0ull;
        double val = valid ? __ldcs(vals64 + (pos - p.val_origin)) : 0.0;
        // padded lanes of a ragged tile: lane 0's key (every row they read
        // exists), value 0, and a group of their own summed into the spare slot
        const uint64_t key0 = __shfl_sync(kFull, key, 0);
        if (!valid) key = key0;
        uint32_t t = (uint32_t)((key >> p.t_shift) & p.t_mask);
        uint32_t o[NS];
#pragma unroll
        for (int q = 0; q < NS; ++q)
            o[q] = (q < ng) ? (uint32_t)((key >> p.gat[q].shift) & p.gat[q].mask) : 0u;
        if (!p.single_block) {
            const uint32_t *bb = p.bbase + (size_t)block_of(p, valid ? pos : p.begin + tile * 32) * MAXN;
            t += __ldg(bb + p.t_mode);
#pragma unroll
            for (int q = 0; q < NS; ++q)
                if (q < ng) o[q] += __ldg(bb + p.gat[q].mode);
        }
        int slot = -1;
        if (p.hot_dense) {
            slot = (int)t;
        } else if (nb > 0) {
            const uint4 bk = table[hot_hash(t, p.log2nb)];
            slot = (bk.x == t) ? (int)bk.y : ((bk.z == t) ? (int)bk.w : -1);
        }
        if (!valid) {
            t = kNoRow;
            slot = kw;
        }
        // group equal target rows; counting sort of the groups by leader
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
#pragma unroll
        for (int q = 0; q < NS; ++q)
            if (q < ng) st.idx[q][spos] = o[q];
        st.val[spos] = val;
        st.rs[spos] = make_uint2(t, (uint32_t)slot);
        __syncwarp();

        // subgroup g walks sorted positions [g*G, g*G+G); a run's sum is
        // stored where it ends or where the range ends (the part of a run
        // that continues into the next range, at the last step, by atomics)
        const unsigned ends = (heads >> 1) | 0x80000000u;
        double acc0 = 0.0, acc1 = 0.0;
#pragma unroll
        for (int c0 = 0; c0 < STEPS; c0 += CH) {
            double pr0[CH], pr1[CH];
#pragma unroll
            for (int j = 0; j < CH; ++j) pr0[j] = pr1[j] = st.val[g * STEPS + c0 + j];
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                if (q < ng) {
                    double2 f[CH];
#pragma unroll
                    for (int j = 0; j < CH; ++j)
                        f[j] = __ldg(reinterpret_cast<const double2 *>(static_cast<const double *>(p.gat[q].ptr) +
                                                                       (size_t)st.idx[q][g * STEPS + c0 + j] * R) +
                                     c);
#pragma unroll
                    for (int j = 0; j < CH; ++j) {
                        pr0[j] *= f[j].x;
                        pr1[j] *= f[j].y;
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < CH; ++j) {
                const int step = c0 + j;
                const int s = g * STEPS + step;
                acc0 += pr0[j];
                acc1 += pr1[j];
                const bool run_end = (ends >> s) & 1u;
                const bool last = step == STEPS - 1;
                if (last) __syncwarp();
                if (run_end || last) {
                    const uint2 rsw = st.rs[s];
                    const int sl = (int)rsw.y;
                    const bool warp_tier = sl >= 0;
                    const bool cont = last && !run_end && warp_tier;
                    if (!warp_tier) {
                        double *o2 = out + (size_t)rsw.x * R + c * 2;
                        red_add_f64(o2, acc0);
                        red_add_f64(o2 + 1, acc1);
                    } else if (cont) {
                        double *a = wacc + (size_t)sl * R + c * 2;
                        atomicAdd(a, acc0);
                        atomicAdd(a + 1, acc1);
                    }
                    if (last) __syncwarp();
                    if (warp_tier && !cont) {
                        double2 *a = reinterpret_cast<double2 *>(wacc + (size_t)sl * R + c * 2);
                        double2 cur = *a;
                        cur.x += acc0;
                        cur.y += acc1;
                        *a = cur;
                    }
                    acc0 = acc1 = 0.0;
                }
            }
        }
        __syncwarp();
    }

    // add the CTA's per-warp copies to the output once
    __syncthreads();
    for (int i = threadIdx.x; i < kw * R; i += kThreads) {
        const int sl = i / R, e = i % R;
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) v += wacc_all[((size_t)w * (kw + 1) + sl) * R + e];
        const uint32_t row = p.hot_dense ? (uint32_t)sl : __ldg(p.hot_rows + sl);
        if (v != 0.0) red_add_f64(out + (size_t)row * R + e, v);
    }
}

template <int R, int NG>
cudaError_t run_mttkrp64(const KParams &p, const double *vals64, double *out, cudaStream_t s) {
    const int nb = p.log2nb >= 0 ? (1 << p.log2nb) : 0;
    const size_t shm = smem_layout64(sizeof(Stage64<NG>), p.kw, R, nb).total;
    auto kern = k_mttkrp64<R, NG>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess) return e;
    const int grid = grid_for((const void *)kern, shm, p.end - p.begin);
    kern<<<grid, kThreads, shm, s>>>(p, vals64, out);
    return cudaGetLastError();
}

template <int R>
cudaError_t by_ng64(const KParams &p, const double *vals64, double *out, cudaStream_t s) {
    switch (p.n_gather) {
        case 2: return run_mttkrp64<R, 2>(p, vals64, out, s);
        case 3: return run_mttkrp64<R, 3>(p, vals64, out, s);
        default: return run_mttkrp64<R, 0>(p, vals64, out, s);
    }
}

}  // namespace

bool rank_supported_f64(int R) { return R == 8 || R == 16 || R == 32 || R == 64; }

cudaError_t launch_mttkrp_f64(const StoreView &sv, const double *const *factors, int R, int mode, const HotRows &hot,
                              double *out, cudaStream_t s) {
    if (sv.end <= sv.begin) return cudaSuccess;
    KParams p = make_params(sv);
    p.t_shift = sv.shift[mode];
    p.t_mask = sv.mask[mode];
    p.t_mode = mode;
    int q = 0;
    for (int k = 0; k < sv.N; ++k) {
        if (k == mode) continue;
        p.gat[q].ptr = factors[k];
        p.gat[q].shift = sv.shift[k];
        p.gat[q].mask = sv.mask[k];
        p.gat[q].mode = k;
        ++q;
    }
    p.n_gather = q;
    const int cap = warp_tier_rows64(R);
    if (hot.dense && hot.count <= cap) {
        p.hot_dense = 1;
        p.kw = hot.count;
    } else if (hot.rows && hot.count > 0) {
        p.hot_rows = hot.rows;
        p.kw = hot.count < cap ? hot.count : cap;
        int l = 0;
        while ((1 << l) < 2 * p.kw) ++l;
        p.log2nb = l;
    }
    switch (R) {
        case 8: return by_ng64<8>(p, sv.vals64, out, s);
        case 16: return by_ng64<16>(p, sv.vals64, out, s);
        case 32: return by_ng64<32>(p, sv.vals64, out, s);
        case 64: return by_ng64<64>(p, sv.vals64, out, s);
    }
    return cudaErrorInvalidValue;
}

int warp_tier_capacity_f64(int R) { return rank_supported_f64(R) ? warp_tier_rows64(R) : 0; }

}  // namespace blco
