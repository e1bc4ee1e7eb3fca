// All-mode sparse MTTKRP in one pass over the store: every mode's Eq. 1 for
// one set of factors, as blco_mttkrp_all computes it for 5-mode tensors.
//
// A per-mode MTTKRP gathers N - 1 factor rows per nonzero, so computing all N
// modes one after another gathers N (N - 1) rows per nonzero and reads the
// store N times. Here each nonzero's N rows are gathered once and the N
// products x * prod_{k != n} A_k[i_k, :] come from prefix and suffix
// products (3N - 5 multiplications per element for N >= 3), each added to
// its mode's output.
//
// Store order is kept (no per-tile sort: one order cannot suit every mode):
// subgroup g of G = R / VEC lanes walks the tile's positions [g*G, g*G+G),
// and for every mode keeps a running sum while that mode's row stays the
// same. Where a mode's row changes, the run's sum goes to the warp's
// shared-memory copy of the row if the row is one of that mode's hottest
// (picked at build time), else to global memory with red.global.add.v4.f32.
// Two subgroups may store the same hot row in the same step, so stores to
// the shared copies are serialized over the subgroups that have one pending
// (a warp ballot). Row ids and the row's slot in the shared copies are staged
// as one word: id | slot << 24 (modes of at most 2^24 rows; slot 0xFF: no
// copy).
//
// Without the per-mode sort a run ends at almost every nonzero, so each
// nonzero costs N global or shared stores: the store side, not the gathers,
// bounds this kernel. It pays where gathers dominate the per-mode kernels:
// at 5 modes it runs 1.4-1.7x faster than five per-mode launches; at 3 and 4
// modes the per-mode kernels (sorted tiles, 2 or 3 gathers per nonzero) are
// as fast or faster, and blco_mttkrp_all uses them there.
#include "mttkrp_kernels.cuh"

namespace blco {
namespace {

constexpr int kFusedModes = 5;  // the order this kernel serves
constexpr uint32_t kSlotNone = 0xFFu;
constexpr uint32_t kIdMask = 0xFFFFFFu;
// no open run; never a staged word, whose slot byte is a row below kw <= 128
// or kSlotNone
constexpr uint32_t kRunNone = 0xFEFFFFFFu;

struct FusedParams {
    const uint64_t *keys;
    int64_t key_origin;
    const float *vals;
    int64_t val_origin;
    int64_t begin, end;
    const uint32_t *tile_block;
    const int64_t *bstart;
    const uint32_t *bbase;
    int single_block;
    const void *fac[MAXN];        // factor n, I_n x R row-major
    int shift[MAXN];
    uint64_t mask[MAXN];
    float *out[MAXN];             // NULL: mode not requested
    const uint32_t *hot_rows[MAXN];
    int kw[MAXN];                 // rows of mode n with a per-warp copy
    int hot_dense[MAXN];          // 1: every row of mode n has a copy, slot == row
    int log2nb[MAXN];             // table of mode n: 2^log2nb buckets of two (row, slot) pairs; -1 none
    int wacc_off[MAXN];           // float offset of mode n's copies in a warp's area
    int table_off[MAXN];          // bucket offset of mode n's table
    int warp_floats;              // floats of one warp's copies (all modes)
    int table_buckets;            // buckets of all tables
};

template <int N>
struct FStage {
    uint32_t id[N][32];  // row | slot << 24, per mode
    float val[32];
};

__host__ __device__ __forceinline__ size_t fused_smem(int N, int warp_floats, int buckets) {
    const size_t stage = align16((size_t)(N + 1) * 32 * sizeof(uint32_t)) * kWarps;
    return align16(stage + (size_t)kWarps * warp_floats * sizeof(float)) + (size_t)buckets * sizeof(uint4);
}

template <int R, int VEC, int H>
__device__ __forceinline__ void fused_red_global(float *out, uint32_t row, int c, const f2 (&s)[H]) {
    float sv[VEC];
#pragma unroll
    for (int h = 0; h < H; ++h) unpack2(s[h], sv[2 * h], sv[2 * h + 1]);
    float *o2 = out + (size_t)row * R + c * VEC;
#pragma unroll
    for (int e = 0; e < VEC; e += 4) red_add_v4(o2 + e, sv[e], sv[e + 1], sv[e + 2], sv[e + 3]);
}

template <int VEC, int H>
__device__ __forceinline__ void fused_rmw(float *a, const f2 (&s)[H]) {
    f2 *p2 = reinterpret_cast<f2 *>(a);
#pragma unroll
    for (int h = 0; h < H; h += 2) {
        ulonglong2 cur = *reinterpret_cast<ulonglong2 *>(p2 + h);
        cur.x = add2(cur.x, s[h]);
        cur.y = add2(cur.y, s[h + 1]);
        *reinterpret_cast<ulonglong2 *>(p2 + h) = cur;
    }
}

__device__ __forceinline__ uint32_t fused_block_of(const uint32_t *tile_block, const int64_t *bstart, int64_t pos) {
    uint32_t b = __ldg(tile_block + (pos >> 5));
    while (pos >= __ldg(bstart + b + 1)) ++b;
    return b;
}

template <typename T, int R, int N>
__host__ __device__ constexpr int fused_min_ctas() {
    return 2;
}

template <typename T, int R, int N>
__global__ void __launch_bounds__(kThreads, fused_min_ctas<T, R, N>()) k_mttkrp_fused(const FusedParams p) {
    constexpr int VEC = lane_vec<T, R>();
    constexpr int H = VEC / 2;
    constexpr int G = R / VEC;
    static_assert(G >= 1 && G <= 32 && (32 % G) == 0, "rank must give 1..32 lanes per row");
    static_assert(H % 2 == 0, "the shared-copy update moves 16 bytes at a time");
    constexpr int STEPS = G;
    constexpr int CH = 1;  // positions whose rows load back to back

    extern __shared__ __align__(16) unsigned char smem[];
    const size_t stage_bytes = align16((size_t)(N + 1) * 32 * sizeof(uint32_t));
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int g = lane / G;
    const int c = lane % G;
    FStage<N> &st = *reinterpret_cast<FStage<N> *>(smem + stage_bytes * wid);
    float *wacc_all = reinterpret_cast<float *>(smem + stage_bytes * kWarps);
    float *wacc = wacc_all + (size_t)wid * p.warp_floats;
    uint4 *tables =
        reinterpret_cast<uint4 *>(smem + align16(stage_bytes * kWarps + (size_t)kWarps * p.warp_floats * sizeof(float)));

    // --- zero the copies; thread n fills mode n's table in order of decreasing count
    for (int i = threadIdx.x; i < kWarps * p.warp_floats; i += kThreads) wacc_all[i] = 0.f;
    for (int i = threadIdx.x; i < p.table_buckets; i += kThreads) tables[i] = make_uint4(kNoRow, 0u, kNoRow, 0u);
    __syncthreads();
    if (threadIdx.x < N && p.log2nb[threadIdx.x] >= 0) {
        const int n = threadIdx.x;
        uint4 *tb = tables + p.table_off[n];
        for (int i = 0; i < p.kw[n]; ++i) {
            const uint32_t row = __ldg(p.hot_rows[n] + i);
            uint4 &bk = tb[hot_hash(row, p.log2nb[n])];
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

    const char *rowp[N];
#pragma unroll
    for (int n = 0; n < N; ++n) rowp[n] = static_cast<const char *>(p.fac[n]) + (size_t)c * VEC * sizeof(T);

    const int64_t ntiles = (p.end - p.begin + 31) >> 5;
    const int64_t wstride = (int64_t)gridDim.x * kWarps;
    int64_t tile = (int64_t)blockIdx.x * kWarps + wid;
    uint64_t key = 0;
    float val = 0.f;
    if (tile < ntiles) {
        const int64_t pos = p.begin + tile * 32 + lane;
        if (pos < p.end) {
            key = ld_stream_u64(p.keys + (pos - p.key_origin));
            val = ld_stream_f32(p.vals + (pos - p.val_origin));
        }
    }
    while (tile < ntiles) {
        const int64_t base = p.begin + tile * 32;
        const int64_t pos = base + lane;
        const bool valid = pos < p.end;
        const int nvalid = p.end - base < 32 ? (int)(p.end - base) : 32;
        const int64_t ntile = tile + wstride;
        uint64_t nkey = 0;
        float nval = 0.f;
        {
            const int64_t npos = p.begin + ntile * 32 + lane;
            if (ntile < ntiles && npos < p.end) {
                nkey = ld_stream_u64(p.keys + (npos - p.key_origin));
                nval = ld_stream_f32(p.vals + (npos - p.val_origin));
            }
        }
        // --- de-linearize every mode's row; look up its on-chip slot; stage
        uint32_t blockbase[N];
#pragma unroll
        for (int n = 0; n < N; ++n) blockbase[n] = 0u;
        if (!p.single_block && valid) {
            const uint32_t *bb = p.bbase + (size_t)fused_block_of(p.tile_block, p.bstart, pos) * MAXN;
#pragma unroll
            for (int n = 0; n < N; ++n) blockbase[n] = __ldg(bb + n);
        }
#pragma unroll
        for (int n = 0; n < N; ++n) {
            const uint32_t r = valid ? (uint32_t)((key >> p.shift[n]) & p.mask[n]) + blockbase[n] : 0u;
            uint32_t slot = kSlotNone;
            if (p.hot_dense[n]) {
                slot = r;
            } else if (p.log2nb[n] >= 0) {
                const uint4 bk = tables[p.table_off[n] + hot_hash(r, p.log2nb[n])];
                slot = (bk.x == r) ? bk.y : ((bk.z == r) ? bk.w : kSlotNone);
            }
            st.id[n][lane] = r | (slot << 24);
        }
        st.val[lane] = valid ? val : 0.f;
        __syncwarp();

        // --- subgroup g walks positions [g*G, g*G+G) in store order
        uint32_t cur[N];
        f2 acc[N][H];
#pragma unroll
        for (int n = 0; n < N; ++n) {
            cur[n] = kRunNone;
#pragma unroll
            for (int h = 0; h < H; ++h) acc[n][h] = 0ull;
        }
        // stores the open run of every mode with flush[n] set: cold rows by
        // vector reductions, hot rows by read-modify-write of the warp's copy,
        // one subgroup at a time (warp-uniform call)
        auto store_runs = [&](const bool (&flush)[N]) {
            bool hot_pending = false;
#pragma unroll
            for (int n = 0; n < N; ++n) {
                if (!flush[n] || !p.out[n]) continue;
                const uint32_t sl = cur[n] >> 24;
                if (sl == kSlotNone) {
                    fused_red_global<R, VEC, H>(p.out[n], cur[n] & kIdMask, c, acc[n]);
                } else {
                    hot_pending = true;
                }
            }
            unsigned pend = __ballot_sync(kFull, hot_pending);
            while (pend) {
                const int sg = (__ffs(pend) - 1) / G;
                if (g == sg && hot_pending) {
#pragma unroll
                    for (int n = 0; n < N; ++n) {
                        if (!flush[n] || !p.out[n]) continue;
                        const uint32_t sl = cur[n] >> 24;
                        if (sl != kSlotNone) fused_rmw<VEC, H>(wacc + p.wacc_off[n] + (size_t)sl * R + c * VEC, acc[n]);
                    }
                }
                __syncwarp();
                pend &= ~((G == 32 ? kFull : ((1u << G) - 1u)) << (sg * G));
            }
        };
#pragma unroll
        for (int j0 = 0; j0 < STEPS; j0 += CH) {
            uint32_t w[CH][N];
            f2 pre[CH][H];  // value times the rows of modes before n
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                const int s = g * STEPS + j0 + i;
                const float v = st.val[s];
#pragma unroll
                for (int n = 0; n < N; ++n) w[i][n] = st.id[n][s];
                const f2 vv = pack2(v, v);
#pragma unroll
                for (int h = 0; h < H; ++h) pre[i][h] = vv;
            }
            f2 rowv[CH][N][H];
#pragma unroll
            for (int n = 0; n < N; ++n)
#pragma unroll
                for (int i = 0; i < CH; ++i)
                    Chunk<T>::load(rowp[n] + (size_t)(w[i][n] & kIdMask) * (R * sizeof(T)), rowv[i][n]);
#pragma unroll
            for (int i = 0; i < CH; ++i) {
                const int s = g * STEPS + j0 + i;
                const bool in = s < nvalid;
                // products for every mode: prefix (value and modes < n) times suffix (modes > n)
                f2 prod[N][H];
                {
                    f2 run[H];
#pragma unroll
                    for (int h = 0; h < H; ++h) run[h] = pre[i][h];
#pragma unroll
                    for (int n = 0; n < N; ++n) {
#pragma unroll
                        for (int h = 0; h < H; ++h) {
                            prod[n][h] = run[h];
                            run[h] = mul2(run[h], rowv[i][n][h]);
                        }
                    }
#pragma unroll
                    for (int h = 0; h < H; ++h) run[h] = rowv[i][N - 1][h];
#pragma unroll
                    for (int n = N - 2; n >= 0; --n) {
#pragma unroll
                        for (int h = 0; h < H; ++h) {
                            prod[n][h] = mul2(prod[n][h], run[h]);
                            if (n > 0) run[h] = mul2(run[h], rowv[i][n][h]);
                        }
                    }
                }
                bool flush[N];
#pragma unroll
                for (int n = 0; n < N; ++n) flush[n] = in && cur[n] != kRunNone && w[i][n] != cur[n];
                store_runs(flush);
                if (in) {
#pragma unroll
                    for (int n = 0; n < N; ++n) {
                        if (cur[n] == kRunNone || w[i][n] != cur[n]) {
                            cur[n] = w[i][n];
#pragma unroll
                            for (int h = 0; h < H; ++h) acc[n][h] = prod[n][h];
                        } else {
#pragma unroll
                            for (int h = 0; h < H; ++h) acc[n][h] = add2(acc[n][h], prod[n][h]);
                        }
                    }
                }
            }
        }
        // the range's open runs
        {
            bool flush[N];
#pragma unroll
            for (int n = 0; n < N; ++n) flush[n] = cur[n] != kRunNone;
            store_runs(flush);
        }
        __syncwarp();
        tile = ntile;
        key = nkey;
        val = nval;
    }

    // --- add the CTA's per-warp copies to the outputs once
    __syncthreads();
    constexpr int Q = R / 4;
#pragma unroll
    for (int n = 0; n < N; ++n) {
        if (!p.out[n]) continue;
        for (int i = threadIdx.x; i < p.kw[n] * Q; i += kThreads) {
            const int sl = i / Q, q = i % Q;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int ww = 0; ww < kWarps; ++ww) {
                const float4 x = *reinterpret_cast<const float4 *>(wacc_all + (size_t)ww * p.warp_floats + p.wacc_off[n] +
                                                                   (size_t)sl * R + q * 4);
                v.x += x.x;
                v.y += x.y;
                v.z += x.z;
                v.w += x.w;
            }
            const uint32_t row = p.hot_dense[n] ? (uint32_t)sl : __ldg(p.hot_rows[n] + sl);
            if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f)
                red_add_v4(p.out[n] + (size_t)row * R + q * 4, v.x, v.y, v.z, v.w);
        }
    }
}

// Rows per warp on chip: 4 KB of float32 copies per warp, split over the modes.
constexpr int kFusedWarpBytes = 4 * 1024;

template <typename T, int R, int N>
cudaError_t run_fused(const FusedParams &p, cudaStream_t s) {
    const size_t shm = fused_smem(N, p.warp_floats, p.table_buckets);
    auto kern = k_mttkrp_fused<T, R, N>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess) return e;
    const int grid = grid_for((const void *)kern, shm, p.end - p.begin);
    kern<<<grid, kThreads, shm, s>>>(p);
    return cudaGetLastError();
}

template <typename T, int R>
cudaError_t fused_by_n(const FusedParams &p, int N, cudaStream_t s) {
    return N == kFusedModes ? run_fused<T, R, kFusedModes>(p, s) : cudaErrorInvalidValue;
}

template <typename T>
cudaError_t fused_as(const StoreView &sv, const FactorSet &fs, int R, const HotRows *hot, float *const *outs,
                     cudaStream_t s) {
    if (sv.end <= sv.begin) return cudaSuccess;
    FusedParams p;
    memset(&p, 0, sizeof(p));
    p.keys = sv.keys;
    p.key_origin = sv.key_origin;
    p.vals = sv.vals;
    p.val_origin = sv.val_origin;
    p.begin = sv.begin;
    p.end = sv.end;
    p.tile_block = sv.tile_block;
    p.bstart = sv.bstart;
    p.bbase = sv.bbase;
    p.single_block = sv.single_block;
    const int N = sv.N;
    const int budget = (kFusedWarpBytes / (R * (int)sizeof(float))) / N > 0 ? (kFusedWarpBytes / (R * 4)) / N : 1;
    int wf = 0, tb = 0;
    for (int n = 0; n < N; ++n) {
        p.fac[n] = fs.ptr[n];
        p.shift[n] = sv.shift[n];
        p.mask[n] = sv.mask[n];
        p.out[n] = outs[n];
        p.log2nb[n] = -1;
        p.wacc_off[n] = wf;
        p.table_off[n] = tb;
        if (sv.dims[n] <= budget) {
            p.hot_dense[n] = 1;
            p.kw[n] = (int)sv.dims[n];
        } else if (hot[n].rows && hot[n].count > 0) {
            p.hot_rows[n] = hot[n].rows;
            p.kw[n] = hot[n].count < budget ? hot[n].count : budget;
            int l = 0;
            while ((1 << l) < 2 * p.kw[n]) ++l;
            p.log2nb[n] = l;
            tb += 1 << l;
        }
        wf += p.kw[n] * R;
    }
    p.warp_floats = wf;
    p.table_buckets = tb;
    switch (R) {
        case 16: return fused_by_n<T, 16>(p, N, s);
        case 32: return fused_by_n<T, 32>(p, N, s);
        case 64: return fused_by_n<T, 64>(p, N, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace

bool fused_supported(const StoreView &sv, int R) {
    if (sv.N != kFusedModes) return false;
    if (R != 16 && R != 32 && R != 64) return false;
    for (int n = 0; n < sv.N; ++n)
        if (sv.dims[n] > ((int64_t)1 << 24)) return false;
    return true;
}

cudaError_t launch_mttkrp_fused(const StoreView &sv, const FactorSet &fs, blco_dtype fdt, int R, const HotRows *hot,
                                float *const *outs, cudaStream_t s) {
    switch (fdt) {
        case BLCO_F32: return fused_as<float>(sv, fs, R, hot, outs, s);
        case BLCO_BF16: return fused_as<__nv_bfloat16>(sv, fs, R, hot, outs, s);
        case BLCO_F16: return fused_as<__half>(sv, fs, R, hot, outs, s);
        default: break;
    }
    return cudaErrorInvalidValue;
}

}  // namespace blco
