// Sparse MTTKRP (Eq. 1, Fig. 3) and the CP model at the nonzeros over a
// BLCO store, for sm_103a.
//
// One warp owns a tile of 32 consecutive nonzeros of the store:
//   1. each lane streams one nonzero's key and value (cache-streaming loads,
//      issued one tile ahead) and de-linearizes only the fields it needs --
//      the target row and the gathered modes -- by shift and mask (Section
//      4.1, Fig. 6b), adding the block's high bits from the block table
//      (Section 4.2) when the store has any;
//   2. the warp groups lanes with equal target row with __match_any_sync and
//      orders the 32 nonzeros so that each group is contiguous (a counting
//      sort by group leader: one warp scan) -- in place of the paper's
//      per-tile histogram + prefix-sum reordering (Section 5.1, processing
//      phase); each lane also looks up, once, the shared-memory slot of its
//      row if the row is hot;
//   3. lanes are re-assigned across the rank: G = R/4 lanes per nonzero,
//      each loading 4 elements of every gathered factor row (16 bytes of
//      float32, 8 of bf16/fp16), so one warp load moves P = 32/G whole
//      rows; subgroup g walks the sorted positions [g*G, g*G+G), issuing the
//      row loads of up to 4 positions back to back, multiplying with packed
//      f32x2 arithmetic and keeping a running float32 sum (Kahan-compensated
//      for 16-bit factors unless disabled) while the target row stays the
//      same (Section 5.1, computing phase);
//   4. where a run ends the sum goes either to the warp's own shared-memory
//      copy of the row (the mode's hottest rows, plain read-modify-write) or
//      to global memory with one red.global.add.v4.f32 per 16 bytes (every
//      other row: Section 5.2's register-based path). Hot rows are picked at
//      build time from a per-mode histogram; when the whole mode fits, every
//      row is hot. Each CTA adds its warps' copies to global memory once at
//      exit (Section 5.1's local stash and final merge; the per-mode choice
//      of Section 5.3 becomes a per-row split). Short modes at R >= 64 reduce
//      into one of a few private output copies instead (the paper's per-GPC
//      copies of M), summed by a separate kernel after the launch.
// The grid is persistent (SM count x resident CTAs); warps stride over the
// tiles, so the warps running at any moment cover a narrow window of the ALTO
// order and share factor rows in L2.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstring>

#include "internal.h"

// Kernels and launchers are templates over the factor type; each of
// mttkrp_f32.cu / mttkrp_bf16.cu / mttkrp_f16.cu instantiates one type, so
// the three compile in parallel. Everything here has internal linkage.
namespace blco {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kMaxGather = MAXN;      // the CP model gathers all N modes

struct Gather {
    const void *ptr;  // factor matrix, I x R row-major
    uint64_t mask;    // in-block field mask
    int shift;        // in-block field offset
    int mode;         // mode index (block table column)
};

struct KParams {
    const uint64_t *keys;
    int64_t key_origin;
    const float *vals;
    int64_t val_origin;
    int64_t begin, end;
    const uint32_t *tile_block;
    const int64_t *bstart;
    const uint32_t *bbase;
    int single_block;
    int n_gather;
    Gather gat[kMaxGather];
    // target field (MTTKRP) / output origin (CP model)
    uint64_t t_mask;
    int t_shift;
    int t_mode;
    float *out;
    int64_t out_origin;
    // MTTKRP into private output copies (short modes): CTA b adds into copy
    // b % ncopies, copy_stride floats apart; ncopies == 1 means `out` itself
    int ncopies;
    int64_t copy_stride;
    // on-chip accumulation of the hottest rows: the first kw rows of
    // hot_rows get one private copy per warp; with hot_dense every row of
    // the mode does and slot == row
    const uint32_t *hot_rows;
    int kw;
    int hot_dense;
    int log2nb;  // 2^log2nb buckets of two hot row ids (-1: no table)
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ uint64_t ld_stream_u64(const uint64_t *p) {
    return (uint64_t)__ldcs(reinterpret_cast<const unsigned long long *>(p));
}
__device__ __forceinline__ float ld_stream_f32(const float *p) { return __ldcs(p); }

// Vector reduction into global memory. No "memory" clobber: the kernel never
// reads `out` and the adds commute, so the compiler may move loads across it.
__device__ __forceinline__ void red_add_v4(float *addr, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d));
}

// Packed pairs of float32 (f32x2 arithmetic, round to nearest even).
typedef unsigned long long f2;
__device__ __forceinline__ f2 pack2(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void unpack2(f2 r, float &a, float &b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// Running sum of a run. With COMP, Kahan's compensated summation: `c` holds
// the low-order part lost by the last addition (negated), fed back into the
// next one, so a run of many terms is summed to about one rounding of the
// result instead of one rounding per term. The arithmetic is explicit
// round-to-nearest (PTX or __fadd_rn/__fsub_rn), so nothing is contracted
// into an FMA.
template <bool COMP>
struct RunSum;

template <>
struct RunSum<false> {
    f2 s;
    __device__ __forceinline__ void clear() { s = 0ull; }
    __device__ __forceinline__ void add(f2 x) { s = add2(s, x); }
    __device__ __forceinline__ f2 value() const { return s; }
};

// The compensated sum runs on scalar float32 (two independent chains per
// pair): each Kahan step is a chain of four dependent additions, and packed
// f32x2 chains measured 6% slower here than two scalar chains.
template <>
struct RunSum<true> {
    float s0, s1, c0, c1;
    __device__ __forceinline__ void clear() { s0 = s1 = c0 = c1 = 0.f; }
    __device__ __forceinline__ static void step(float x, float &s, float &c) {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
    __device__ __forceinline__ void add(f2 x) {
        float x0, x1;
        unpack2(x, x0, x1);
        step(x0, s0, c0);
        step(x1, s1, c1);
    }
    __device__ __forceinline__ f2 value() const { return pack2(__fsub_rn(s0, c0), __fsub_rn(s1, c1)); }
};

// A lane's slice of a factor row: VEC elements loaded BYTES at a time as
// VEC/2 packed float pairs.
template <typename T>
struct Chunk;  // one BYTES-wide load -> PAIRS packed float pairs

template <>
struct Chunk<float> {
    static constexpr int PAIRS = 2;
    static constexpr int BYTES = 16;
    __device__ __forceinline__ static void load(const void *addr, f2 *f) {
        const ulonglong2 v = __ldg(reinterpret_cast<const ulonglong2 *>(addr));
        f[0] = v.x;
        f[1] = v.y;
    }
};

// bfloat16 -> float32 is exact: the 16 bits become the top half of the word.
__device__ __forceinline__ f2 bf16x2_to_f2(uint32_t w) {
    return pack2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
}

// 16-bit factors are read 8 bytes (4 elements) per load, so that a lane
// holds 4 elements and a warp has as many nonzeros in flight as with float32.
template <>
struct Chunk<__nv_bfloat16> {
    static constexpr int PAIRS = 2;
    static constexpr int BYTES = 8;
    __device__ __forceinline__ static void load(const void *addr, f2 *f) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(addr));
        f[0] = bf16x2_to_f2(v.x);
        f[1] = bf16x2_to_f2(v.y);
    }
};

template <>
struct Chunk<__half> {
    static constexpr int PAIRS = 2;
    static constexpr int BYTES = 8;
    __device__ __forceinline__ static void load(const void *addr, f2 *f) {
        const uint2 v = __ldg(reinterpret_cast<const uint2 *>(addr));
        const uint32_t w[2] = {v.x, v.y};
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float2 t = __half22float2(*reinterpret_cast<const __half2 *>(&w[i]));
            f[i] = pack2(t.x, t.y);
        }
    }
};

// Elements per lane for rank R: one vector load (4 elements). Wider slices
// (more loads per lane) cut per-nonzero overhead but multiply the subgroups
// that flush divergently, and measured slower on GB300.
template <typename T, int R>
__host__ __device__ constexpr int lane_vec() {
    return Chunk<T>::BYTES / (int)sizeof(T);
}

template <typename T, int VEC>
__device__ __forceinline__ void load_slice(const void *base, size_t elem, f2 (&f)[VEC / 2]) {
    constexpr int EPC = Chunk<T>::BYTES / (int)sizeof(T);  // elements per load
    const T *b = static_cast<const T *>(base) + elem;
#pragma unroll
    for (int i = 0; i < VEC / EPC; ++i) Chunk<T>::load(b + i * EPC, f + i * Chunk<T>::PAIRS);
}

// r[e] <- r[(e + k) mod V] for a runtime k, with static register indices
// (one conditional stage per bit of k).
template <int V>
__device__ __forceinline__ void rotate_left(float (&r)[V], int k) {
#pragma unroll
    for (int b = 1; b < V; b <<= 1) {
        if (k & b) {
            float t[V];
#pragma unroll
            for (int e = 0; e < V; ++e) t[e] = r[(e + b) % V];
#pragma unroll
            for (int e = 0; e < V; ++e) r[e] = t[e];
        }
    }
}

// Block index of store position pos (only for stores with nonzero high bits).
__device__ __forceinline__ uint32_t block_of(const KParams &p, int64_t pos) {
    uint32_t b = __ldg(p.tile_block + (pos >> 5));
    while (pos >= __ldg(p.bstart + b + 1)) ++b;
    return b;
}

__device__ __forceinline__ uint32_t hot_hash(uint32_t row, int log2n) {
    return log2n > 0 ? (row * 0x9E3779B1u) >> (32 - log2n) : 0u;
}

// Number of gathered modes: NG > 0 fixed at compile time, NG == 0 runtime.
template <int NG>
__device__ __forceinline__ int n_gather(const KParams &p) {
    return NG > 0 ? NG : p.n_gather;
}
template <int NG>
__host__ __device__ constexpr int gather_slots() {
    return NG > 0 ? NG : kMaxGather;
}

// Byte offsets of the MTTKRP kernel's shared-memory sections, each rounded
// up to 16 bytes: each warp's staging of its tile, the per-warp copies of
// the hot rows (kw rows plus one spare row that takes the padded lanes of a
// ragged tile and is never merged), and the table of hot row ids (nb buckets
// of two (row, slot) pairs, 16 bytes each, read with one vector load).
struct SmemLayout {
    size_t wacc, table, total;
};
__host__ __device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }
__host__ __device__ __forceinline__ SmemLayout smem_layout(size_t stage_bytes, int kw, int R, int nb) {
    SmemLayout L;
    L.wacc = align16(stage_bytes * kWarps);
    L.table = align16(L.wacc + (size_t)kWarps * (kw + 1) * R * sizeof(float));
    L.total = align16(L.table + (size_t)nb * sizeof(uint4));
    return L;
}

// The MTTKRP kernel's staging of one tile's sorted positions: gathered row
// ids and values by field, the target row and its on-chip slot as one 8-byte
// word (read with one shared load where a run ends).
template <int NG>
struct MStage {
    uint32_t idx[gather_slots<NG>()][32];
    float val[32];
    uint2 rs[32];  // (row, slot)
};

// The CP-model kernel's staging: gathered row ids in, model values out.
template <int NG>
struct Stage {
    uint32_t idx[gather_slots<NG>()][32];
    float val[32];
};

// -------------------------------------------------------------------------
// MTTKRP
// -------------------------------------------------------------------------
// Resident CTAs per SM the register budget is sized for (64 registers for
// 4, 80 for 3, 128 for 2). Measured on GB300: the MTTKRP kernel is fastest
// with 4 up to R = 32, loading the rows of 2 positions at a time (3 CTAs
// with 4 positions: 3% slower on the 3-mode Zipf workload, 4% on the 4-mode
// one); with 3 at R = 64 and two gathered modes (82 registers, hence 2
// CTAs, made the planted 3-mode R = 64 adjoint 15% slower); more gathered
// rows at R = 64 keep 2. The CP-model kernel runs 3 (80 registers) with
// batches of 16 elements per gathered row and one reduce-scatter per G
// positions: 8% faster at R = 64 (the planted 3-mode workload) and 14% at
// R = 32 (the 3-mode Zipf shape) than 2 CTAs with 32-element batches and a
// shuffle reduction per position.
template <int R, int NG>
__host__ __device__ constexpr int mttkrp_min_ctas() {
    return (NG == 0 || R > 64 || (R == 64 && NG > 2)) ? 2 : (R <= 32 ? 4 : 3);
}
template <int R, int NG>
__host__ __device__ constexpr int cp_min_ctas() {
    return NG == 0 ? 2 : 3;
}

template <typename T, int R, int NG, bool COMP>
__global__ void __launch_bounds__(kThreads, mttkrp_min_ctas<R, NG>()) k_mttkrp(const KParams p) {
    constexpr int VEC = lane_vec<T, R>();  // elements per lane
    constexpr int H = VEC / 2;   // packed pairs per lane
    constexpr int G = R / VEC;   // lanes per nonzero
    static_assert(G >= 1 && G <= 32 && (32 % G) == 0, "rank must give 1..32 lanes per row");
    constexpr int STEPS = G;     // sorted positions per subgroup (P = 32 / G subgroups)
    // positions whose row loads are issued back to back: 8 elements of each
    // gathered row per lane at 4 CTAs per SM, 16 otherwise
    constexpr int CHE = mttkrp_min_ctas<R, NG>() == 4 ? 8 : 16;
    constexpr int CH = STEPS < CHE / VEC ? STEPS : CHE / VEC;
    constexpr int NS = gather_slots<NG>();

    extern __shared__ __align__(16) unsigned char smem[];
    const int kw = p.kw;  // warp tier: the hottest rows, one private copy per warp
    const int nb = p.log2nb >= 0 ? (1 << p.log2nb) : 0;  // buckets of two row ids
    const SmemLayout L = smem_layout(sizeof(MStage<NG>), kw, R, nb);
    MStage<NG> *stage = reinterpret_cast<MStage<NG> *>(smem);
    float *wacc_all = reinterpret_cast<float *>(smem + L.wacc);
    uint4 *table = reinterpret_cast<uint4 *>(smem + L.table);

    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int g = lane / G;
    const int c = lane % G;
    MStage<NG> &st = stage[wid];
    float *wacc = wacc_all + (size_t)wid * (kw + 1) * R;
    const int ng = n_gather<NG>(p);
    float *const outp = p.out + (p.ncopies > 1 ? (size_t)(blockIdx.x % p.ncopies) * p.copy_stride : 0);

    // --- zero the accumulators; thread 0 fills the hot-row table in order of
    // decreasing count (one hash, buckets of two (row, slot) pairs; a row that
    // finds its bucket full stays off chip and is simply a cold row)
    for (int i = threadIdx.x; i < kWarps * (kw + 1) * R; i += kThreads) wacc_all[i] = 0.f;
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
    int64_t tile = (int64_t)blockIdx.x * kWarps + wid;
    uint64_t key = 0;
    float val = 0.f;
    {
        const int64_t pos = p.begin + tile * 32 + lane;
        if (tile < ntiles && pos < p.end) {
            key = ld_stream_u64(p.keys + (pos - p.key_origin));
            val = ld_stream_f32(p.vals + (pos - p.val_origin));
        }
    }
    while (tile < ntiles) {
        const int64_t pos = p.begin + tile * 32 + lane;
        const bool valid = pos < p.end;
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

        // Lanes past the end of the store (the ragged last tile) take lane 0's
        // key with value 0, so that every row they read exists; below they
        // form a group of their own, whose sum is never stored.
        {
            const uint64_t key0 = __shfl_sync(kFull, key, 0);
            if (!valid) {
                key = key0;
                val = 0.f;
            }
        }
        // --- de-linearize the target row and the gathered rows
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
        // --- on-chip slot of this lane's row (one lookup per nonzero: one
        // 16-byte shared load of the row's bucket, no probing loop)
        int slot = -1;
        {
            if (p.hot_dense) {
                slot = (int)t;
            } else if (nb > 0) {
                const uint4 bk = table[hot_hash(t, p.log2nb)];
                slot = (bk.x == t) ? (int)bk.y : ((bk.z == t) ? (int)bk.w : -1);
            }
        }
        // padded lanes: a group of their own (kNoRow is no row), which the
        // sort places after every real nonzero, summed into the warp's spare
        // slot kw, which is never merged into the output -- so a factor row
        // holding Inf never meets a padded lane's 0
        if (!valid) {
            t = kNoRow;
            slot = kw;
        }

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
#pragma unroll
        for (int q = 0; q < NS; ++q)
            if (q < ng) st.idx[q][spos] = o[q];
        st.val[spos] = val;
        st.rs[spos] = make_uint2(t, (uint32_t)slot);
        __syncwarp();

        // --- rank-parallel products; subgroup g walks the sorted positions
        // [g*G, g*G+G) and adds each run (or the part of a run inside its
        // range) to the row's accumulator where the run ends or the range
        // ends. Before the last step two lanes of the warp never flush the
        // same row in the same step (a run has one end), so warp-tier rows
        // take a plain read-modify-write. At the last step the part of a run
        // that continues into the next range meets another update of its row
        // in that step only if the run also covers the next range up to its
        // last position (that range then flushes the same row too); such
        // parts use atomics, ordered before the plain updates by __syncwarp,
        // and every other part is the only update of its row in the step.
        const unsigned ends = (heads >> 1) | 0x80000000u;  // bit s: a run ends at s
        // the next range [(g+1)*G, (g+2)*G) has no run end before its last
        // position (only used where a run continues past this range, so g+1
        // is a range of the tile)
        const bool next_unbroken =
            g + 1 < 32 / G && ((ends >> (((g + 1) * STEPS) & 31)) & ((1u << (STEPS - 1)) - 1u)) == 0u;
        RunSum<COMP> acc[H];
#pragma unroll
        for (int h = 0; h < H; ++h) acc[h].clear();
#pragma unroll
        for (int c0 = 0; c0 < STEPS; c0 += CH) {
            f2 pr[CH][H];
            uint32_t ridx[CH][NS];
#pragma unroll
            for (int j = 0; j < CH; ++j) {
                const float v = st.val[g * STEPS + c0 + j];
#pragma unroll
                for (int q = 0; q < NS; ++q) ridx[j][q] = (q < ng) ? st.idx[q][g * STEPS + c0 + j] : 0u;
                const f2 vv = pack2(v, v);
#pragma unroll
                for (int h = 0; h < H; ++h) pr[j][h] = vv;
            }
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                if (q < ng) {
                    f2 f[CH][H];
#pragma unroll
                    for (int j = 0; j < CH; ++j)
                        load_slice<T, VEC>(p.gat[q].ptr, (size_t)ridx[j][q] * R + c * VEC, f[j]);
#pragma unroll
                    for (int j = 0; j < CH; ++j)
#pragma unroll
                        for (int h = 0; h < H; ++h) pr[j][h] = mul2(pr[j][h], f[j][h]);
                }
            }
#pragma unroll
            for (int j = 0; j < CH; ++j) {
                const int step = c0 + j;
                const int s = g * STEPS + step;
#pragma unroll
                for (int h = 0; h < H; ++h) acc[h].add(pr[j][h]);
                const bool run_end = (ends >> s) & 1u;
                const bool last = step == STEPS - 1;
                // order the earlier steps' plain updates before the atomics below
                if (last) __syncwarp();
                if (run_end || last) {
                    f2 sum[H];
#pragma unroll
                    for (int h = 0; h < H; ++h) sum[h] = acc[h].value();
                    const uint2 rsw = st.rs[s];
                    const uint32_t row = rsw.x;
                    const int sl = (int)rsw.y;
                    const bool warp_tier = sl >= 0;
                    // continuation parts that meet another update at the
                    // last step: atomics first
                    const bool cont = last && !run_end && warp_tier && next_unbroken;
                    if (!warp_tier) {
                        float sv[VEC];
#pragma unroll
                        for (int h = 0; h < H; ++h) unpack2(sum[h], sv[2 * h], sv[2 * h + 1]);
                        float *o2 = outp + (size_t)row * R + c * VEC;
#pragma unroll
                        for (int e = 0; e < VEC; e += 4)
                            red_add_v4(o2 + e, sv[e], sv[e + 1], sv[e + 2], sv[e + 3]);
                    } else if (cont) {
                        float sv[VEC];
#pragma unroll
                        for (int h = 0; h < H; ++h) unpack2(sum[h], sv[2 * h], sv[2 * h + 1]);
                        float *a = wacc + (size_t)sl * R + c * VEC;
#pragma unroll
                        for (int e = 0; e < VEC; ++e) atomicAdd(a + e, sv[e]);
                    }
                    if (last) __syncwarp();
                    if (warp_tier && !cont) {
                        f2 *a = reinterpret_cast<f2 *>(wacc + (size_t)sl * R + c * VEC);
#pragma unroll
                        for (int h = 0; h < H; h += 2) {
                            ulonglong2 cur = *reinterpret_cast<ulonglong2 *>(a + h);
                            cur.x = add2(cur.x, sum[h]);
                            cur.y = add2(cur.y, sum[h + 1]);
                            *reinterpret_cast<ulonglong2 *>(a + h) = cur;
                        }
                    }
#pragma unroll
                    for (int h = 0; h < H; ++h) acc[h].clear();
                }
            }
        }
        __syncwarp();
        tile = ntile;
        key = nkey;
        val = nval;
    }

    // --- add the CTA's accumulators to the output once
    __syncthreads();
    constexpr int Q = R / 4;
    for (int i = threadIdx.x; i < kw * Q; i += kThreads) {
        const int sl = i / Q, q = i % Q;
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
            const float4 x = *reinterpret_cast<const float4 *>(wacc_all + ((size_t)w * (kw + 1) + sl) * R + q * 4);
            v.x += x.x;
            v.y += x.y;
            v.z += x.z;
            v.w += x.w;
        }
        const uint32_t row = p.hot_dense ? (uint32_t)sl : __ldg(p.hot_rows + sl);
        if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f)
            red_add_v4(outp + (size_t)row * R + q * 4, v.x, v.y, v.z, v.w);
    }
}

// -------------------------------------------------------------------------
// CP model at the nonzeros: xhat = sum_r prod_n A_n[i_n, r] (all N modes gathered)
// -------------------------------------------------------------------------
template <typename T, int R, int NG>
__global__ void __launch_bounds__(kThreads, cp_min_ctas<R, NG>()) k_cp_fwd(const KParams p) {
    constexpr int VEC = lane_vec<T, R>();
    constexpr int H = VEC / 2;
    constexpr int G = R / VEC;
    constexpr int STEPS = G;
    constexpr int CH = STEPS < 16 / VEC ? STEPS : 16 / VEC;  // positions per register batch (16 floats)
    constexpr int NS = gather_slots<NG>();
    __shared__ Stage<NG> stage[kWarps];
    const int lane = threadIdx.x & 31;
    const int wid = threadIdx.x >> 5;
    const int g = lane / G;
    const int c = lane % G;
    Stage<NG> &st = stage[wid];
    const int ng = n_gather<NG>(p);
    const int64_t ntiles = (p.end - p.begin + 31) >> 5;
    const int64_t wstride = (int64_t)gridDim.x * kWarps;
    for (int64_t tile = (int64_t)blockIdx.x * kWarps + wid; tile < ntiles; tile += wstride) {
        const int64_t pos = p.begin + tile * 32 + lane;
        const bool valid = pos < p.end;
        const uint64_t key = valid ? ld_stream_u64(p.keys + (pos - p.key_origin)) : 0ull;
        uint32_t o[NS];
#pragma unroll
        for (int q = 0; q < NS; ++q)
            o[q] = (q < ng) ? (uint32_t)((key >> p.gat[q].shift) & p.gat[q].mask) : 0u;
        if (!p.single_block && valid) {
            const uint32_t *bb = p.bbase + (size_t)block_of(p, pos) * MAXN;
#pragma unroll
            for (int q = 0; q < NS; ++q)
                if (q < ng) o[q] += __ldg(bb + p.gat[q].mode);
        }
#pragma unroll
        for (int q = 0; q < NS; ++q)
            if (q < ng) st.idx[q][lane] = valid ? o[q] : 0u;
        __syncwarp();
        float parts[STEPS];  // partial sum over this lane's elements, per position
#pragma unroll
        for (int c0 = 0; c0 < STEPS; c0 += CH) {
            f2 pr[CH][H];
#pragma unroll
            for (int j = 0; j < CH; ++j)
#pragma unroll
                for (int h = 0; h < H; ++h) pr[j][h] = pack2(1.f, 1.f);
#pragma unroll
            for (int q = 0; q < NS; ++q) {
                if (q < ng) {
                    f2 f[CH][H];
#pragma unroll
                    for (int j = 0; j < CH; ++j)
                        load_slice<T, VEC>(p.gat[q].ptr, (size_t)st.idx[q][g * STEPS + c0 + j] * R + c * VEC, f[j]);
#pragma unroll
                    for (int j = 0; j < CH; ++j)
#pragma unroll
                        for (int h = 0; h < H; ++h) pr[j][h] = mul2(pr[j][h], f[j][h]);
                }
            }
#pragma unroll
            for (int j = 0; j < CH; ++j) {
                float part = 0.f;
#pragma unroll
                for (int h = 0; h < H; ++h) {
                    float a, b;
                    unpack2(pr[j][h], a, b);
                    part += a + b;
                }
                parts[c0 + j] = part;
            }
        }
        // reduce-scatter of the G positions' partial sums over the subgroup's
        // G lanes (G - 1 shuffles instead of log2(G) per position): in the
        // round with distance hh a lane keeps the half of its sums whose
        // position has bit hh equal to its own lane bit and sends the other
        // half to lane ^ hh, so lane c ends with the sum of position g*G + c
#pragma unroll
        for (int hh = G / 2; hh >= 1; hh >>= 1) {
            const bool up = (c & hh) != 0;
#pragma unroll
            for (int i = 0; i < hh; ++i) {
                const float send = up ? parts[i] : parts[i + hh];
                const float keep = up ? parts[i + hh] : parts[i];
                parts[i] = keep + __shfl_xor_sync(kFull, send, hh);
            }
        }
        st.val[g * STEPS + c] = parts[0];
        __syncwarp();
        if (valid) p.out[pos - p.out_origin] = st.val[lane];
        __syncwarp();
    }
}

// -------------------------------------------------------------------------
// launch helpers
// -------------------------------------------------------------------------
// Shared memory for on-chip accumulation: kWarps private copies of kw rows
// per CTA. Measured on GB300, a second tier of rows shared by the CTA's warps
// (shared-memory atomics) was slower than sending those rows to global
// memory, and more rows per warp take L1 capacity from the factor-row
// gathers: 4 KB per warp is the measured optimum at R = 16..64.
constexpr int kWarpTierBytes = 4 * 1024;  // per warp

int warp_tier_rows(int R) { return kWarpTierBytes / (R * (int)sizeof(float)); }

KParams make_params(const StoreView &sv) {
    KParams p;
    memset(&p, 0, sizeof(p));
    p.log2nb = -1;
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
    return p;
}

int grid_for(const void *kern, size_t shm, int64_t span) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, shm) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int64_t tiles = (span + 31) / 32;
    int64_t grid = (int64_t)sm_count() * per_sm;
    const int64_t need = (tiles + kWarps - 1) / kWarps;
    if (grid > need) grid = need;
    if (grid < 1) grid = 1;
    return (int)grid;
}

template <typename T, int R, int NG, bool COMP>
cudaError_t run_mttkrp_impl(const KParams &p, cudaStream_t s) {
    const int nb = p.log2nb >= 0 ? (1 << p.log2nb) : 0;
    const size_t shm = smem_layout(sizeof(MStage<NG>), p.kw, R, nb).total;
    auto kern = k_mttkrp<T, R, NG, COMP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e != cudaSuccess) return e;
    const int grid = grid_for((const void *)kern, shm, p.end - p.begin);
    kern<<<grid, kThreads, shm, s>>>(p);
    return cudaGetLastError();
}

template <typename T, int R, int NG>
cudaError_t run_cp_fwd_impl(const KParams &p, cudaStream_t s) {
    auto kern = k_cp_fwd<T, R, NG>;
    const int grid = grid_for((const void *)kern, 0, p.end - p.begin);
    kern<<<grid, kThreads, 0, s>>>(p);
    return cudaGetLastError();
}

// Compile-time gather counts for 3-, 4- and 5-mode tensors at ranks 16..64;
// every other case runs the generic instantiation (runtime count).
template <typename T, int R, bool COMP>
cudaError_t by_ng_mttkrp(const KParams &p, cudaStream_t s) {
    switch (p.n_gather) {
        case 2: return run_mttkrp_impl<T, R, 2, COMP>(p, s);
        case 3: return run_mttkrp_impl<T, R, 3, COMP>(p, s);
        case 4: return run_mttkrp_impl<T, R, 4, COMP>(p, s);
        default: return run_mttkrp_impl<T, R, 0, COMP>(p, s);
    }
}
template <typename T, int R>
cudaError_t by_ng_cp(const KParams &p, cudaStream_t s) {
    switch (p.n_gather) {
        case 3: return run_cp_fwd_impl<T, R, 3>(p, s);
        case 4: return run_cp_fwd_impl<T, R, 4>(p, s);
        case 5: return run_cp_fwd_impl<T, R, 5>(p, s);
        default: return run_cp_fwd_impl<T, R, 0>(p, s);
    }
}

template <typename T, bool COMP>
cudaError_t by_rank_mttkrp(const KParams &p, int R, cudaStream_t s) {
    switch (R) {
        case 8: return run_mttkrp_impl<T, 8, 0, COMP>(p, s);
        case 16: return by_ng_mttkrp<T, 16, COMP>(p, s);
        case 32: return by_ng_mttkrp<T, 32, COMP>(p, s);
        case 64: return by_ng_mttkrp<T, 64, COMP>(p, s);
        case 128: return run_mttkrp_impl<T, 128, 0, COMP>(p, s);
    }
    return cudaErrorInvalidValue;
}
template <typename T>
cudaError_t by_rank_cp(const KParams &p, int R, cudaStream_t s) {
    switch (R) {
        case 8: return run_cp_fwd_impl<T, 8, 0>(p, s);
        case 16: return by_ng_cp<T, 16>(p, s);
        case 32: return by_ng_cp<T, 32>(p, s);
        case 64: return by_ng_cp<T, 64>(p, s);
        case 128: return run_cp_fwd_impl<T, 128, 0>(p, s);
    }
    return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t mttkrp_as(const StoreView &sv, const FactorSet &fs, int R, int mode, const HotRows &hot, float *out,
                      const OutCopies &oc, bool compensated, cudaStream_t s) {
    if (sv.end <= sv.begin) return cudaSuccess;
    KParams p = make_params(sv);
    p.t_shift = sv.shift[mode];
    p.t_mask = sv.mask[mode];
    p.t_mode = mode;
    int q = 0;
    for (int k = 0; k < sv.N; ++k) {
        if (k == mode) continue;
        p.gat[q].ptr = fs.ptr[k];
        p.gat[q].shift = sv.shift[k];
        p.gat[q].mask = sv.mask[k];
        p.gat[q].mode = k;
        ++q;
    }
    p.n_gather = q;
    p.out = out;
    p.ncopies = oc.n > 1 ? oc.n : 1;
    p.copy_stride = oc.stride;
    if (hot.dense) {
        // every row of the mode fits the warp tier: slot == row, no table
        p.hot_dense = 1;
        p.kw = hot.count;
    } else if (hot.count > 0) {
        p.hot_rows = hot.rows;
        p.kw = hot.count < warp_tier_rows(R) ? hot.count : warp_tier_rows(R);
        int l = 0;
        while ((1 << l) < 2 * p.kw) ++l;
        p.log2nb = l;
    }
    // float32 factors: plain run sums only; 16-bit factors: compensated
    // unless the caller asked for plain sums
    if constexpr (sizeof(T) == 2) {
        if (compensated) return by_rank_mttkrp<T, true>(p, R, s);
    }
    return by_rank_mttkrp<T, false>(p, R, s);
}

template <typename T>
cudaError_t cp_fwd_as(const StoreView &sv, const FactorSet &fs, int R, float *xhat, int64_t xorigin,
                      cudaStream_t s) {
    if (sv.end <= sv.begin) return cudaSuccess;
    KParams p = make_params(sv);
    for (int k = 0; k < sv.N; ++k) {
        p.gat[k].ptr = fs.ptr[k];
        p.gat[k].shift = sv.shift[k];
        p.gat[k].mask = sv.mask[k];
        p.gat[k].mode = k;
    }
    p.n_gather = sv.N;
    p.out = xhat;
    p.out_origin = xorigin;
    return by_rank_cp<T>(p, R, s);
}

}  // namespace
}  // namespace blco
