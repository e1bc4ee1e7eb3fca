// BLCO construction on the GPU (Section 4, and the construction pipeline of
// Section 6 -- linearize, sort, block, re-encode -- moved from the host CPU
// to the device):
//   k_linearize   ALTO linear index of every nonzero (Section 4.1, Fig. 6a),
//                 range check of every coordinate;
//   radix sort    stable LSD sort of (linear index, input position), 8-bit
//                 digits; per-tile digit counts, one exclusive scan, and a
//                 stable per-tile scatter ranked with __match_any_sync;
//   k_reencode    per stored nonzero: in-block key = concatenated per-mode
//                 low fields, mode 0 lowest (Fig. 6b), value and input
//                 position gathered, packed block key = bits above the line;
//   runs/blocks   block boundaries where the block key changes (Section 4.2),
//                 compacted on the device, split at the cap on the host.
#include <algorithm>
#include <cstring>

#include "internal.h"

namespace blco {

// ---------------------------------------------------------------------------
// host: layout
// ---------------------------------------------------------------------------
bool plan_layout(Layout &L, std::string &why) {
    if (L.N < 1 || L.N > MAXN) {
        why = "order N must be in 1..8";
        return false;
    }
    int maxb = 0;
    L.B = 0;
    for (int n = 0; n < L.N; ++n) {
        if (L.dims[n] < 1 || L.dims[n] > 0xFFFFFFFFll) {
            why = "mode lengths must be in 1..2^32-1";
            return false;
        }
        int b = 0;
        while (b < 32 && ((int64_t)1 << b) < L.dims[n]) ++b;
        L.bits[n] = b;
        L.B += b;
        maxb = std::max(maxb, b);
    }
    if (L.B > 128) {
        why = "more than 128 index bits";
        return false;
    }
    if (L.line < 1 || L.line > 64) {
        why = "line_bits must be in 1..64";
        return false;
    }
    if (L.B - L.line > 64) {
        why = "more than 64 bits above the encoding line";
        return false;
    }
    int pos = 0;
    for (int n = 0; n < L.N; ++n) L.kbits[n] = 0;
    for (int l = 0; l < maxb; ++l)
        for (int n = 0; n < L.N; ++n)
            if (L.bits[n] > l) {
                L.keypos[n][l] = (uint8_t)pos;
                if (pos >= L.line) L.kbits[n]++;
                ++pos;
            }
    int off = 0, boff = 0;
    for (int n = 0; n < L.N; ++n) {
        L.width[n] = L.bits[n] - L.kbits[n];
        L.shift[n] = off;
        off += L.width[n];
        L.boff[n] = boff;
        boff += L.kbits[n];
    }
    return true;
}

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

struct LinArgs {
    int N;
    int B;
    uint32_t dims_m1[MAXN];  // I_n - 1
    int bits[MAXN];
    uint8_t keypos[MAXN][32];
};

// ---------------------------------------------------------------------------
// ALTO key of every nonzero; lo = key bits 0..63, hi = bits 64..127
// ---------------------------------------------------------------------------
__global__ void k_linearize(const uint32_t *__restrict__ coords, int64_t nnz, const LinArgs a,
                            uint64_t *__restrict__ lo, uint64_t *__restrict__ hi, uint32_t *__restrict__ idx,
                            unsigned long long *__restrict__ first_bad) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz;
         j += (int64_t)gridDim.x * blockDim.x) {
        uint64_t l = 0, h = 0;
        bool bad = false;
#pragma unroll
        for (int n = 0; n < MAXN; ++n) {
            if (n < a.N) {
                const uint32_t c = coords[j * a.N + n];
                bad |= c > a.dims_m1[n];
                for (int lev = 0; lev < a.bits[n]; ++lev) {
                    const uint64_t bit = (c >> lev) & 1u;
                    const int p = a.keypos[n][lev];
                    if (p < 64)
                        l |= bit << p;
                    else
                        h |= bit << (p - 64);
                }
            }
        }
        if (bad) atomicMin(first_bad, (unsigned long long)j);
        lo[j] = l;
        if (hi) hi[j] = h;
        idx[j] = (uint32_t)j;
    }
}

// ---------------------------------------------------------------------------
// exclusive scan of uint32 (in place), any length, recursive over tile sums
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *sh, uint32_t &total) {
    // warp inclusive scan
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = lane < (int)(blockDim.x / 32) ? sh[lane] : 0u;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, s, d);
            if (lane >= d) s += y;
        }
        if (lane < (int)(blockDim.x / 32)) sh[lane] = s;
    }
    __syncthreads();
    const uint32_t before = w > 0 ? sh[w - 1] : 0u;
    total = sh[blockDim.x / 32 - 1];
    __syncthreads();
    return before + x - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ d, int64_t n,
                                                              uint32_t *__restrict__ sums) {
    __shared__ uint32_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    uint32_t s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t p = base + (int64_t)i * kScanThreads + threadIdx.x;
        if (p < n) s += d[p];
    }
    uint32_t total;
    block_exclusive_scan(s, sh, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_down(uint32_t *__restrict__ d, int64_t n,
                                                            const uint32_t *__restrict__ offs) {
    __shared__ uint32_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    // blocked arrangement: thread t owns items [t*16, t*16+16)
    uint32_t v[kScanItems];
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t p = base + (int64_t)threadIdx.x * kScanItems + i;
        v[i] = p < n ? d[p] : 0u;
        s += v[i];
    }
    uint32_t total;
    uint32_t run = block_exclusive_scan(s, sh, total) + (offs ? offs[blockIdx.x] : 0u);
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t p = base + (int64_t)threadIdx.x * kScanItems + i;
        if (p < n) d[p] = run;
        run += v[i];
    }
}

cudaError_t scan_exclusive(uint32_t *d, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 1) {
        k_scan_down<<<1, kScanThreads, 0, s>>>(d, n, nullptr);
        return cudaGetLastError();
    }
    uint32_t *sums = nullptr;
    cudaError_t e = cudaMallocAsync(&sums, sizeof(uint32_t) * tiles, s);
    if (e != cudaSuccess) return e;
    k_scan_reduce<<<(unsigned)tiles, kScanThreads, 0, s>>>(d, n, sums);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = scan_exclusive(sums, tiles, s);
    if (e == cudaSuccess) {
        k_scan_down<<<(unsigned)tiles, kScanThreads, 0, s>>>(d, n, sums);
        e = cudaGetLastError();
    }
    cudaFreeAsync(sums, s);
    return e;
}

// ---------------------------------------------------------------------------
// stable LSD radix sort of (key, uint32 value) pairs, 8-bit digits
// ---------------------------------------------------------------------------
constexpr int kRsThreads = 256;
constexpr int kRsWarps = kRsThreads / 32;
constexpr int kRsRounds = 16;
constexpr int kRsTile = kRsThreads * kRsRounds;  // 4096 items

template <typename K>
__global__ void __launch_bounds__(kRsThreads) k_rs_count(const K *__restrict__ keys, int64_t n, int shift,
                                                         uint32_t *__restrict__ counts, int64_t ntiles) {
    __shared__ uint32_t hist[256];
    hist[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    const int lane = threadIdx.x & 31;
    for (int r = 0; r < kRsRounds; ++r) {
        const int64_t p = base + (int64_t)r * kRsThreads + threadIdx.x;
        const bool valid = p < n;
        const uint32_t dg = valid ? (uint32_t)((keys[p] >> shift) & 0xFFu) : 256u;
        const unsigned peers = __match_any_sync(kFull, dg);
        if (valid && lane == __ffs(peers) - 1) atomicAdd(&hist[dg], (uint32_t)__popc(peers));
    }
    __syncthreads();
    counts[(int64_t)threadIdx.x * ntiles + blockIdx.x] = hist[threadIdx.x];
}

template <typename K>
__global__ void __launch_bounds__(kRsThreads) k_rs_scatter(const K *__restrict__ kin, const uint32_t *__restrict__ vin,
                                                           K *__restrict__ kout, uint32_t *__restrict__ vout,
                                                           int64_t n, int shift, const uint32_t *__restrict__ offs,
                                                           int64_t ntiles) {
    extern __shared__ __align__(16) unsigned char smem[];
    K *sk = reinterpret_cast<K *>(smem);
    uint32_t *sv = reinterpret_cast<uint32_t *>(sk + kRsTile);
    uint32_t *whist = sv + kRsTile;            // [kRsWarps][256]
    uint32_t *tbase = whist + kRsWarps * 256;  // [256]
    uint32_t *tmp = tbase + 256;               // [32]

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kRsWarps * 256; i += kRsThreads) whist[i] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * kRsTile;
    const int64_t tile_n64 = n - base < kRsTile ? n - base : kRsTile;
    const int tile_n = (int)tile_n64;

    K kr[kRsRounds];
    uint32_t vr[kRsRounds];
    uint32_t rr[kRsRounds];
    // warp w ranks items [w*512, w*512+512) of the tile, 32 at a time, in order
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
        const int it = w * (kRsTile / kRsWarps) + r * 32 + lane;
        const bool valid = it < tile_n;
        kr[r] = valid ? kin[base + it] : (K)0;
        vr[r] = valid ? vin[base + it] : 0u;
        const uint32_t dg = valid ? (uint32_t)((kr[r] >> shift) & 0xFFu) : 256u;
        const unsigned peers = __match_any_sync(kFull, dg);
        const int leader = __ffs(peers) - 1;
        const uint32_t prev = valid ? whist[w * 256 + (dg & 0xFFu)] : 0u;
        __syncwarp();
        if (valid && lane == leader) whist[w * 256 + dg] = prev + (uint32_t)__popc(peers);
        __syncwarp();
        rr[r] = prev + (uint32_t)__popc(peers & ((1u << lane) - 1u));
    }
    __syncthreads();
    // per digit: exclusive over warps, and the tile total
    uint32_t total_d;
    {
        const int d = threadIdx.x;  // 256 threads, one per digit
        uint32_t run = 0;
        for (int ww = 0; ww < kRsWarps; ++ww) {
            const uint32_t t = whist[ww * 256 + d];
            whist[ww * 256 + d] = run;
            run += t;
        }
        total_d = run;
    }
    __syncthreads();
    uint32_t all;
    const uint32_t excl = block_exclusive_scan(total_d, tmp, all);
    tbase[threadIdx.x] = excl;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kRsRounds; ++r) {
        const int it = w * (kRsTile / kRsWarps) + r * 32 + lane;
        if (it < tile_n) {
            const uint32_t dg = (uint32_t)((kr[r] >> shift) & 0xFFu);
            const uint32_t lp = tbase[dg] + whist[w * 256 + dg] + rr[r];
            sk[lp] = kr[r];
            sv[lp] = vr[r];
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < tile_n; i += kRsThreads) {
        const K k = sk[i];
        const uint32_t dg = (uint32_t)((k >> shift) & 0xFFu);
        const int64_t gp = (int64_t)offs[(int64_t)dg * ntiles + blockIdx.x] + (i - (int64_t)tbase[dg]);
        kout[gp] = k;
        vout[gp] = sv[i];
    }
}

template <typename K>
size_t rs_scatter_smem() {
    return sizeof(K) * kRsTile + sizeof(uint32_t) * kRsTile + sizeof(uint32_t) * (kRsWarps * 256 + 256 + 32);
}

// Sorts (keys, vals) by key bits [0, nbits); result ends in (keys, vals).
template <typename K>
cudaError_t radix_sort_pairs(K *keys, uint32_t *vals, K *kalt, uint32_t *valt, int64_t n, int nbits,
                             cudaStream_t s) {
    if (n <= 1 || nbits <= 0) return cudaSuccess;
    const int64_t ntiles = (n + kRsTile - 1) / kRsTile;
    uint32_t *counts = nullptr;
    cudaError_t e = cudaMallocAsync(&counts, sizeof(uint32_t) * 256 * ntiles, s);
    if (e != cudaSuccess) return e;
    const size_t shm = rs_scatter_smem<K>();
    e = cudaFuncSetAttribute(k_rs_scatter<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    K *ki = keys, *ko = kalt;
    uint32_t *vi = vals, *vo = valt;
    for (int shift = 0; shift < nbits && e == cudaSuccess; shift += 8) {
        k_rs_count<K><<<(unsigned)ntiles, kRsThreads, 0, s>>>(ki, n, shift, counts, ntiles);
        e = cudaGetLastError();
        if (e == cudaSuccess) e = scan_exclusive(counts, 256 * ntiles, s);
        if (e == cudaSuccess) {
            k_rs_scatter<K><<<(unsigned)ntiles, kRsThreads, shm, s>>>(ki, vi, ko, vo, n, shift, counts, ntiles);
            e = cudaGetLastError();
        }
        std::swap(ki, ko);
        std::swap(vi, vo);
    }
    if (e == cudaSuccess && ki != keys) {
        e = cudaMemcpyAsync(keys, ki, sizeof(K) * n, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vals, vi, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
    }
    cudaFreeAsync(counts, s);
    return e;
}

// ---------------------------------------------------------------------------
// gathers and re-encoding
// ---------------------------------------------------------------------------
__global__ void k_gather_u64(const uint64_t *__restrict__ src, const uint32_t *__restrict__ idx, int64_t n,
                             uint64_t *__restrict__ dst) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        dst[j] = src[idx[j]];
}

struct EncArgs {
    int N;
    int has_blocks;
    uint32_t lowmask[MAXN];
    int shift[MAXN];
    int width[MAXN];
    int boff[MAXN];
};

__global__ void k_reencode(const uint32_t *__restrict__ coords, const float *__restrict__ vals,
                           const uint32_t *__restrict__ perm, int64_t nnz, const EncArgs a,
                           uint64_t *__restrict__ skeys, float *__restrict__ svals,
                           uint64_t *__restrict__ bkey) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = perm[j];
        uint64_t key = 0, bk = 0;
#pragma unroll
        for (int n = 0; n < MAXN; ++n) {
            if (n < a.N) {
                const uint32_t c = coords[p * a.N + n];
                key |= (uint64_t)(c & a.lowmask[n]) << a.shift[n];
                if (a.has_blocks) bk |= (a.width[n] >= 32 ? 0ull : (uint64_t)(c >> a.width[n])) << a.boff[n];
            }
        }
        skeys[j] = key;
        svals[j] = vals ? vals[p] : 0.f;  // no float32 values: a float64 store gathers its own
        if (a.has_blocks) bkey[j] = bk;
    }
}

__global__ void k_gather_f64(const double *__restrict__ src, const uint32_t *__restrict__ perm, int64_t nnz,
                             double *__restrict__ dst) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < nnz; j += (int64_t)gridDim.x * blockDim.x)
        dst[j] = src[perm[j]];
}

__global__ void k_run_flags(const uint64_t *__restrict__ bkey, int64_t n, uint32_t *__restrict__ flags) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        flags[j] = (j == 0 || bkey[j] != bkey[j - 1]) ? 1u : 0u;
}

__global__ void k_run_compact(const uint64_t *__restrict__ bkey, const uint32_t *__restrict__ scanned,
                              int64_t n, int64_t *__restrict__ starts, uint64_t *__restrict__ keys_out) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        if (j == 0 || bkey[j] != bkey[j - 1]) {
            const uint32_t r = scanned[j];
            starts[r] = j;
            keys_out[r] = bkey[j];
        }
    }
}

__global__ void k_tile_block(const int64_t *__restrict__ bstart, int64_t nblocks, int64_t ntiles,
                             uint32_t *__restrict__ tb) {
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t pos = t * 32;
        // last block b with bstart[b] <= pos
        int64_t lo = 0, hi = nblocks - 1;
        while (lo < hi) {
            const int64_t mid = (lo + hi + 1) >> 1;
            if (bstart[mid] <= pos)
                lo = mid;
            else
                hi = mid - 1;
        }
        tb[t] = (uint32_t)lo;
    }
}

// Row counts of one mode over a systematic sample of the store: every
// `stride`-th 32-nonzero tile (all tiles when stride is 1), one warp per
// sampled tile. The counts only rank rows for on-chip accumulation, so a
// sample of tens of millions of nonzeros is enough to find the heavy rows.
__global__ void k_histogram(const StoreView sv, int mode, int64_t stride, uint32_t *__restrict__ counts) {
    const int64_t ntiles = (sv.end - sv.begin + 31) >> 5;
    const int64_t nsamp = (ntiles + stride - 1) / stride;
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    // the loop bound is uniform over the warp, so whole warps iterate together
    for (int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; j < nsamp; j += nwarps) {
        const int64_t pos = sv.begin + j * stride * 32 + lane;
        const bool live = pos < sv.end;
        uint32_t row = 0;
        if (live) {
            const uint64_t key = sv.keys[pos - sv.key_origin];
            uint32_t base = 0;
            if (!sv.single_block) {
                uint32_t b = sv.tile_block[pos >> 5];
                while (pos >= sv.bstart[b + 1]) ++b;
                base = sv.bbase[(size_t)b * MAXN + mode];
            }
            row = (uint32_t)((key >> sv.shift[mode]) & sv.mask[mode]) + base;
        }
        const unsigned lanes = __ballot_sync(0xFFFFFFFFu, live);
        if (live) {
            const unsigned peers = __match_any_sync(lanes, row);
            if (lane == __ffs(peers) - 1) atomicAdd(&counts[row], (uint32_t)__popc(peers));
        }
    }
}

__global__ void k_pack_count_row(const uint32_t *__restrict__ counts, int64_t I, uint32_t *__restrict__ key,
                                 uint32_t *__restrict__ row) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < I; i += (int64_t)gridDim.x * blockDim.x) {
        key[i] = ~counts[i];  // ascending sort of ~count = descending count
        row[i] = (uint32_t)i;
    }
}

unsigned grid_for(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count() * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

}  // namespace

// ---------------------------------------------------------------------------
cudaError_t build_store(const Layout &L, const uint32_t *coords, const float *vals, int64_t nnz, int64_t cap,
                        BuildOut &out, cudaStream_t s, std::string &why) {
    cudaError_t e = cudaSuccess;
    const int64_t npad = ((nnz + 31) / 32) * 32 + 32;
    uint64_t *lo = nullptr, *lo2 = nullptr, *hi = nullptr, *hi2 = nullptr, *bkey = nullptr;
    uint32_t *idx = nullptr, *idx2 = nullptr;
    unsigned long long *d_bad = nullptr;
    const bool wide = L.B > 64;
    const bool has_blocks = L.B > L.line;
#define TRY(x)                      \
    do {                            \
        e = (x);                    \
        if (e != cudaSuccess) goto done; \
    } while (0)
    TRY(cudaMalloc(&out.keys, sizeof(uint64_t) * npad));
    TRY(cudaMalloc(&out.vals, sizeof(float) * npad));
    TRY(cudaMalloc(&out.perm, sizeof(uint32_t) * (nnz > 0 ? nnz : 1)));
    TRY(cudaMemsetAsync(out.keys, 0, sizeof(uint64_t) * npad, s));
    TRY(cudaMemsetAsync(out.vals, 0, sizeof(float) * npad, s));
    if (nnz > 0) {
        TRY(cudaMallocAsync(&lo, sizeof(uint64_t) * nnz, s));
        TRY(cudaMallocAsync(&lo2, sizeof(uint64_t) * nnz, s));
        TRY(cudaMallocAsync(&idx2, sizeof(uint32_t) * nnz, s));
        TRY(cudaMallocAsync(&d_bad, sizeof(unsigned long long), s));
        TRY(cudaMemsetAsync(d_bad, 0xFF, sizeof(unsigned long long), s));
        idx = out.perm;
        if (wide) {
            TRY(cudaMallocAsync(&hi, sizeof(uint64_t) * nnz, s));
            TRY(cudaMallocAsync(&hi2, sizeof(uint64_t) * nnz, s));
        }
        {
            LinArgs a;
            memset(&a, 0, sizeof(a));
            a.N = L.N;
            a.B = L.B;
            for (int n = 0; n < L.N; ++n) {
                a.dims_m1[n] = (uint32_t)(L.dims[n] - 1);
                a.bits[n] = L.bits[n];
                memcpy(a.keypos[n], L.keypos[n], 32);
            }
            k_linearize<<<grid_for(nnz, 256), 256, 0, s>>>(coords, nnz, a, lo, hi, idx, d_bad);
            TRY(cudaGetLastError());
        }
        {
            unsigned long long bad = 0;
            TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(bad), cudaMemcpyDeviceToHost, s));
            TRY(cudaStreamSynchronize(s));
            if (bad != ~0ull) {
                out.first_bad = (int64_t)bad;
                why = "coordinate row " + std::to_string((long long)bad) + " is out of range";
                goto done;
            }
        }
        // sort by the low word, then (stably) by the high word
        TRY(radix_sort_pairs<uint64_t>(lo, idx, lo2, idx2, nnz, std::min(L.B, 64), s));
        if (wide) {
            k_gather_u64<<<grid_for(nnz, 256), 256, 0, s>>>(hi, idx, nnz, hi2);
            TRY(cudaGetLastError());
            TRY(radix_sort_pairs<uint64_t>(hi2, idx, hi, idx2, nnz, L.B - 64, s));
        }
        {
            EncArgs a;
            memset(&a, 0, sizeof(a));
            a.N = L.N;
            a.has_blocks = has_blocks ? 1 : 0;
            for (int n = 0; n < L.N; ++n) {
                a.lowmask[n] = L.width[n] >= 32 ? 0xFFFFFFFFu : ((1u << L.width[n]) - 1u);
                a.shift[n] = L.shift[n];
                a.width[n] = L.width[n];
                a.boff[n] = L.boff[n];
            }
            if (has_blocks) TRY(cudaMallocAsync(&bkey, sizeof(uint64_t) * nnz, s));
            k_reencode<<<grid_for(nnz, 256), 256, 0, s>>>(coords, vals, idx, nnz, a, out.keys, out.vals, bkey);
            TRY(cudaGetLastError());
        }
    }
    // block runs
    {
        std::vector<int64_t> run_start;
        std::vector<uint64_t> run_key;
        if (nnz > 0 && has_blocks) {
            uint32_t *flags = idx2;  // reuse
            k_run_flags<<<grid_for(nnz, 256), 256, 0, s>>>(bkey, nnz, flags);
            TRY(cudaGetLastError());
            uint32_t last_flag = 0;
            TRY(cudaMemcpyAsync(&last_flag, flags + nnz - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            TRY(scan_exclusive(flags, nnz, s));
            uint32_t last_scan = 0;
            TRY(cudaMemcpyAsync(&last_scan, flags + nnz - 1, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
            TRY(cudaStreamSynchronize(s));
            const int64_t nruns = (int64_t)last_scan + last_flag;
            int64_t *d_starts = reinterpret_cast<int64_t *>(lo2);  // reuse: nruns <= nnz
            uint64_t *d_rkeys = lo;
            k_run_compact<<<grid_for(nnz, 256), 256, 0, s>>>(bkey, flags, nnz, d_starts, d_rkeys);
            TRY(cudaGetLastError());
            run_start.resize(nruns);
            run_key.resize(nruns);
            TRY(cudaMemcpyAsync(run_start.data(), d_starts, sizeof(int64_t) * nruns, cudaMemcpyDeviceToHost, s));
            TRY(cudaMemcpyAsync(run_key.data(), d_rkeys, sizeof(uint64_t) * nruns, cudaMemcpyDeviceToHost, s));
            TRY(cudaStreamSynchronize(s));
        } else if (nnz > 0) {
            run_start.push_back(0);
            run_key.push_back(0);
        }
        // split runs at the cap: pieces of ceil(c / ceil(c / cap)) entries
        out.bstart.clear();
        out.bhigh.clear();
        for (size_t r = 0; r < run_start.size(); ++r) {
            const int64_t a = run_start[r];
            const int64_t b = (r + 1 < run_start.size()) ? run_start[r + 1] : nnz;
            const int64_t cnt = b - a;
            const int64_t pieces = (cnt + cap - 1) / cap;
            const int64_t piece = (cnt + pieces - 1) / pieces;
            for (int64_t p = a; p < b; p += piece) {
                out.bstart.push_back(p);
                for (int n = 0; n < L.N; ++n) {
                    const uint64_t m = L.kbits[n] >= 64 ? ~0ull : ((1ull << L.kbits[n]) - 1ull);
                    out.bhigh.push_back((uint32_t)((run_key[r] >> L.boff[n]) & m));
                }
            }
        }
        out.bstart.push_back(nnz);
    }
done:
#undef TRY
    if (lo) cudaFreeAsync(lo, s);
    if (lo2) cudaFreeAsync(lo2, s);
    if (hi) cudaFreeAsync(hi, s);
    if (hi2) cudaFreeAsync(hi2, s);
    if (idx2) cudaFreeAsync(idx2, s);
    if (bkey) cudaFreeAsync(bkey, s);
    if (d_bad) cudaFreeAsync(d_bad, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    return e;
}

cudaError_t gather_f64(const double *src, const uint32_t *perm, int64_t nnz, double *dst, cudaStream_t s) {
    if (nnz <= 0) return cudaSuccess;
    k_gather_f64<<<grid_for(nnz, 256), 256, 0, s>>>(src, perm, nnz, dst);
    return cudaGetLastError();
}

cudaError_t build_tile_block(const int64_t *d_bstart, int64_t nblocks, int64_t nnz, uint32_t *tile_block,
                             cudaStream_t s) {
    const int64_t ntiles = (nnz + 31) / 32;
    if (ntiles == 0) return cudaSuccess;
    k_tile_block<<<grid_for(ntiles, 256), 256, 0, s>>>(d_bstart, nblocks, ntiles, tile_block);
    return cudaGetLastError();
}

cudaError_t mode_histogram(const StoreView &sv, int mode, uint32_t *counts, cudaStream_t s) {
    if (sv.end <= sv.begin) return cudaSuccess;
    const int64_t ntiles = (sv.end - sv.begin + 31) / 32;
    const int64_t stride = std::max<int64_t>(1, ntiles >> 20);  // at most ~2^20 sampled tiles
    const int64_t nsamp = (ntiles + stride - 1) / stride;
    k_histogram<<<grid_for(nsamp * 32, 256), 256, 0, s>>>(sv, mode, stride, counts);
    return cudaGetLastError();
}

cudaError_t top_rows(const uint32_t *counts, int64_t I, int k, uint32_t *rows_out, cudaStream_t s) {
    uint32_t *key = nullptr, *row = nullptr, *key2 = nullptr, *row2 = nullptr;
    cudaError_t e = cudaMallocAsync(&key, sizeof(uint32_t) * I, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&row, sizeof(uint32_t) * I, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&key2, sizeof(uint32_t) * I, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&row2, sizeof(uint32_t) * I, s);
    if (e == cudaSuccess) {
        k_pack_count_row<<<grid_for(I, 256), 256, 0, s>>>(counts, I, key, row);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = radix_sort_pairs<uint32_t>(key, row, key2, row2, I, 32, s);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(rows_out, row, sizeof(uint32_t) * std::min<int64_t>(k, I), cudaMemcpyDeviceToDevice, s);
    if (key) cudaFreeAsync(key, s);
    if (row) cudaFreeAsync(row, s);
    if (key2) cudaFreeAsync(key2, s);
    if (row2) cudaFreeAsync(row2, s);
    return e;
}

}  // namespace blco
