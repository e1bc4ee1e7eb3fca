// The C ABI of libblco.so (include/blco.h): argument checks, the handle, host
// staging, and the out-of-memory streaming engine of Section 4.2 (device
// queues with reserved memory reused across batches of blocks; the copy of
// a pending batch overlaps the MTTKRP of an active one).
#include <algorithm>
#include <atomic>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace blco {

static thread_local std::string g_err;

int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (cache[dev] == 0) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cache[dev] = v > 0 ? v : 1;
    }
    return cache[dev];
}

namespace {

constexpr int64_t kDefaultCap = (int64_t)1 << 27;

blco_status fail(blco_status st, const std::string &msg) {
    g_err = msg;
    return st;
}

blco_status cuda_fail(cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")";
    return fail(e == cudaErrorMemoryAllocation ? BLCO_ERR_OOM : BLCO_ERR_CUDA, m);
}

// Host-side fault injection (blco_inject_fault): events of a kind left
// until the armed one fails; 0 = disarmed.
std::atomic<long> g_fault_left[3];
bool fault_now(int kind) {
    long v = g_fault_left[kind].load();
    while (v > 0)
        if (g_fault_left[kind].compare_exchange_weak(v, v - 1)) return v == 1;
    return false;
}

bool is_device_ptr(const void *p) {
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

}  // namespace
}  // namespace blco

using namespace blco;

struct blco_tensor {
    int device = 0;
    Layout L;
    int64_t nnz = 0;
    int64_t npad = 0;
    int64_t max_nnz = kDefaultCap;
    int nq = 8;
    int64_t budget = 0;
    bool streamed = false;
    bool host_reads = false;   // streamed store read in host memory by the kernels (no queues)
    bool compensated = false;  // 16-bit factors: Kahan-compensated run sums (build option)
    // store (device when resident, pinned host when streamed)
    uint64_t *d_keys = nullptr;
    float *d_vals = nullptr;
    double *d_vals64 = nullptr;  // float64 values (stores built by blco_build_f64)
    bool f64 = false;
    uint32_t *d_perm = nullptr;
    uint64_t *h_keys = nullptr;
    float *h_vals = nullptr;
    uint32_t *h_perm = nullptr;
    uint64_t *hd_keys = nullptr;  // device views of h_keys / h_vals (host_reads)
    float *hd_vals = nullptr;
    // block table
    std::vector<int64_t> bstart;
    std::vector<uint32_t> bhigh;
    int64_t *d_bstart = nullptr;
    uint32_t *d_bbase = nullptr;
    uint32_t *d_tile_block = nullptr;
    bool single_block = true;
    // hot rows per mode
    uint32_t *d_hot[MAXN] = {};
    int hot_count[MAXN] = {};
    // streaming queues
    int64_t queue_nnz = 0;
    uint64_t *q_keys[8] = {};
    float *q_vals[8] = {};
    cudaStream_t q_stream[8] = {};
    cudaEvent_t q_done[8] = {};    // after each kernel on the queue: its reservation is free
    cudaEvent_t q_copied[8] = {};  // after each batch upload into the queue's reservation
    cudaStream_t q_up = nullptr;   // all batch uploads, one after another
    cudaEvent_t ev_fork = nullptr;
    struct Batch {
        int64_t begin, end;
    };
    std::vector<Batch> batches;
    // staging workspace for host arguments
    void *ws = nullptr;
    size_t ws_bytes = 0;
    // private output copies of short modes (grown on demand)
    float *d_copies = nullptr;
    size_t copies_bytes = 0;
    // host-argument copies of blco_mttkrp_all (created on first use): uploads
    // and downloads on their own streams, so they overlap other modes' kernels
    cudaStream_t up = nullptr, down = nullptr;
    cudaEvent_t ev_call = nullptr, ev_down = nullptr;
    cudaEvent_t ev_up[MAXN] = {}, ev_out[MAXN] = {};
    int64_t dev_bytes = 0;
    int64_t host_bytes = 0;
    bool building = false;  // construction: the budget is checked once at the end
    // kernel timing
    bool profiling = false;
    struct Mark {
        const char *name;
        cudaEvent_t a, b;
    };
    std::vector<Mark> marks;

    cudaError_t dalloc(void **p, size_t bytes) {
        if (fault_now(BLCO_FAULT_ALLOC)) return cudaErrorMemoryAllocation;
        if (!building && budget > 0 && dev_bytes + (int64_t)bytes > budget) return cudaErrorMemoryAllocation;
        cudaError_t e = cudaMalloc(p, bytes ? bytes : 1);
        if (e == cudaSuccess) dev_bytes += (int64_t)bytes;
        return e;
    }
    void dfree(void *p, size_t bytes) {
        if (p) {
            cudaFree(p);
            dev_bytes -= (int64_t)bytes;
        }
    }
    cudaError_t workspace(size_t bytes, void **p) {
        if (bytes > ws_bytes) {
            if (ws) dfree(ws, ws_bytes);
            ws = nullptr;
            ws_bytes = 0;
            cudaError_t e = dalloc(&ws, bytes);
            if (e != cudaSuccess) return e;
            ws_bytes = bytes;
        }
        *p = ws;
        return cudaSuccess;
    }
    StoreView view() const {
        StoreView sv;
        memset(&sv, 0, sizeof(sv));
        sv.keys = d_keys;
        sv.key_origin = 0;
        sv.vals = d_vals;
        sv.val_origin = 0;
        sv.vals64 = d_vals64;
        sv.begin = 0;
        sv.end = nnz;
        sv.tile_block = d_tile_block;
        sv.bstart = d_bstart;
        sv.bbase = d_bbase;
        sv.single_block = single_block ? 1 : 0;
        sv.N = L.N;
        for (int n = 0; n < L.N; ++n) {
            sv.dims[n] = L.dims[n];
            sv.shift[n] = L.shift[n];
            sv.mask[n] = L.width[n] >= 64 ? ~0ull : ((1ull << L.width[n]) - 1ull);
        }
        return sv;
    }
};

namespace {

void release(blco_tensor *h) {
    if (!h) return;
    DeviceGuard g(h->device);
    cudaDeviceSynchronize();
    h->dfree(h->d_keys, 0);
    h->dfree(h->d_vals, 0);
    h->dfree(h->d_vals64, 0);
    h->dfree(h->d_perm, 0);
    h->dfree(h->d_bstart, 0);
    h->dfree(h->d_bbase, 0);
    h->dfree(h->d_tile_block, 0);
    for (int n = 0; n < MAXN; ++n) h->dfree(h->d_hot[n], 0);
    for (int q = 0; q < 8; ++q) {
        h->dfree(h->q_keys[q], 0);
        h->dfree(h->q_vals[q], 0);
        if (h->q_stream[q]) cudaStreamDestroy(h->q_stream[q]);
        if (h->q_done[q]) cudaEventDestroy(h->q_done[q]);
        if (h->q_copied[q]) cudaEventDestroy(h->q_copied[q]);
    }
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->q_up) cudaStreamDestroy(h->q_up);
    if (h->up) cudaStreamDestroy(h->up);
    if (h->down) cudaStreamDestroy(h->down);
    for (cudaEvent_t ev : {h->ev_call, h->ev_down})
        if (ev) cudaEventDestroy(ev);
    for (int n = 0; n < MAXN; ++n) {
        if (h->ev_up[n]) cudaEventDestroy(h->ev_up[n]);
        if (h->ev_out[n]) cudaEventDestroy(h->ev_out[n]);
    }
    for (auto &m : h->marks) {
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    h->dfree(h->ws, 0);
    h->dfree(h->d_copies, 0);
    if (h->h_keys) cudaFreeHost(h->h_keys);
    if (h->h_vals) cudaFreeHost(h->h_vals);
    if (h->h_perm) cudaFreeHost(h->h_perm);
    delete h;
}

bool check_factors(const blco_tensor *h, const void *const *factors, int skip_mode, std::string &why) {
    if (!factors) {
        why = "factors is NULL";
        return false;
    }
    for (int k = 0; k < h->L.N; ++k) {
        if (k == skip_mode) continue;
        if (!factors[k]) {
            why = "factors[" + std::to_string(k) + "] is NULL";
            return false;
        }
        if (reinterpret_cast<uintptr_t>(factors[k]) & 15) {
            why = "factors[" + std::to_string(k) + "] is not 16-byte aligned";
            return false;
        }
    }
    return true;
}

size_t dtype_size(blco_dtype d) { return d == BLCO_F32 ? 4 : 2; }

bool dtype_ok(int d) { return d == BLCO_F32 || d == BLCO_BF16 || d == BLCO_F16; }

// Device copies of the factor matrices (host ones staged into ws at offsets).
struct Staged {
    FactorSet fs;
    size_t used = 0;
};

blco_status stage_factors(blco_tensor *h, const void *const *factors, int skip_mode, blco_dtype fdt, int R,
                          size_t extra, Staged &st, void **extra_ptr, cudaStream_t s) {
    size_t need = 0;
    bool host[MAXN] = {};
    for (int k = 0; k < h->L.N; ++k) {
        st.fs.ptr[k] = nullptr;
        if (k == skip_mode) continue;
        host[k] = !is_device_ptr(factors[k]);
        if (host[k]) need += ((size_t)h->L.dims[k] * R * dtype_size(fdt) + 255) / 256 * 256;
    }
    for (int k = h->L.N; k < MAXN; ++k) st.fs.ptr[k] = nullptr;
    const size_t total = need + (extra + 255) / 256 * 256;
    char *base = nullptr;
    if (total > 0) {
        void *p = nullptr;
        cudaError_t e = h->workspace(total, &p);
        if (e != cudaSuccess) return cuda_fail(e, "staging workspace");
        base = static_cast<char *>(p);
    }
    size_t off = 0;
    for (int k = 0; k < h->L.N; ++k) {
        if (k == skip_mode) continue;
        if (host[k]) {
            const size_t b = (size_t)h->L.dims[k] * R * dtype_size(fdt);
            cudaError_t e = cudaMemcpyAsync(base + off, factors[k], b, cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return cuda_fail(e, "factor upload");
            st.fs.ptr[k] = base + off;
            off += (b + 255) / 256 * 256;
        } else {
            st.fs.ptr[k] = factors[k];
        }
    }
    if (extra_ptr) *extra_ptr = extra ? base + off : nullptr;
    st.used = total;
    return BLCO_OK;
}

// Launches `launch` on stream s, bracketed by an event pair when timing is on.
template <typename F>
cudaError_t timed(blco_tensor *h, const char *name, cudaStream_t s, F &&launch) {
    if (!h->profiling) return launch();
    blco_tensor::Mark m{name, nullptr, nullptr};
    cudaError_t e = cudaEventCreate(&m.a);
    if (e == cudaSuccess) e = cudaEventCreate(&m.b);
    if (e == cudaSuccess) e = cudaEventRecord(m.a, s);
    if (e == cudaSuccess) e = launch();
    if (e == cudaSuccess) e = cudaEventRecord(m.b, s);
    if (e != cudaSuccess) {
        if (m.a) cudaEventDestroy(m.a);
        if (m.b) cudaEventDestroy(m.b);
        return e;
    }
    h->marks.push_back(m);
    return cudaSuccess;
}

// Runs one kernel over the whole store: resident in one launch, streamed as
// batches of blocks through the device queues. `vals_ext` replaces the
// stored values when non-null (a device array in store order).
template <typename F>
blco_status over_store(blco_tensor *h, const char *name, const float *vals_ext, cudaStream_t s, F &&launch_fn,
                       int64_t range_begin = 0, int64_t range_end = -1) {
    // name == nullptr: launch_fn times its own launches
    auto launch = [&](const StoreView &sv, cudaStream_t q) {
        if (!name) return launch_fn(sv, q);
        return timed(h, name, q, [&]() { return launch_fn(sv, q); });
    };
    if (h->nnz == 0) return BLCO_OK;
    if (!h->streamed || h->host_reads) {
        // resident, or read in pinned host memory by the kernel itself: one
        // launch over the store (or the requested part of it)
        StoreView sv = h->view();
        if (h->host_reads) {
            sv.keys = h->hd_keys;
            sv.vals = h->hd_vals;
        }
        if (vals_ext) sv.vals = vals_ext;
        if (range_end >= 0) {  // a part of the store
            sv.begin = range_begin;
            sv.end = range_end;
            if (sv.end <= sv.begin) return BLCO_OK;
        }
        cudaError_t e = launch(sv, s);
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
        return BLCO_OK;
    }
    // Batches go through the queues round-robin. All uploads run on one
    // stream (q_up), back to back: concurrent host-to-device copies on
    // several streams share the link less efficiently than one stream. An
    // upload into a queue's reservation waits only for the previous kernel
    // on that queue (q_done), so uploads run ahead across modes; the kernel
    // waits for its upload (q_copied) and, the first time in this call, for
    // earlier work on `s` (ev_fork: the output zeroing, the previous mode).
    // Whatever happens, the queues and the upload stream that received work
    // are joined back into `s` before returning, so no work of a failed
    // call outlives it.
    cudaError_t e = cudaEventRecord(h->ev_fork, s);
    if (e != cudaSuccess) return cuda_fail(e, "event record");
    bool used[8] = {}, uploaded = false;
    blco_status st = BLCO_OK;
    for (size_t b = 0; b < h->batches.size() && st == BLCO_OK; ++b) {
        const int q = (int)(b % h->nq);
        const auto &bt = h->batches[b];
        const int64_t n = bt.end - bt.begin;
        if (fault_now(BLCO_FAULT_COPY)) {
            st = fail(BLCO_ERR_CUDA, "injected host-to-device copy fault");
            break;
        }
        e = cudaStreamWaitEvent(h->q_up, h->q_done[q], 0);
        if (e == cudaSuccess)
            e = timed(h, "upload", h->q_up, [&]() {
                cudaError_t ce = cudaMemcpyAsync(h->q_keys[q], h->h_keys + bt.begin, sizeof(uint64_t) * n,
                                                 cudaMemcpyHostToDevice, h->q_up);
                if (ce == cudaSuccess && !vals_ext)
                    ce = cudaMemcpyAsync(h->q_vals[q], h->h_vals + bt.begin, sizeof(float) * n,
                                         cudaMemcpyHostToDevice, h->q_up);
                return ce;
            });
        if (e == cudaSuccess) e = cudaEventRecord(h->q_copied[q], h->q_up);
        uploaded = true;
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->q_stream[q], h->q_copied[q], 0);
        if (e != cudaSuccess) {
            st = cuda_fail(e, "queue upload");
            break;
        }
        used[q] = true;
        StoreView sv = h->view();
        sv.keys = h->q_keys[q];
        sv.key_origin = bt.begin;
        if (vals_ext) {
            sv.vals = vals_ext;
            sv.val_origin = 0;
        } else {
            sv.vals = h->q_vals[q];
            sv.val_origin = bt.begin;
        }
        sv.begin = bt.begin;
        sv.end = bt.end;
        if (b < (size_t)h->nq) {  // the queue's first kernel of this call
            e = cudaStreamWaitEvent(h->q_stream[q], h->ev_fork, 0);
            if (e != cudaSuccess) {
                st = cuda_fail(e, "stream wait");
                break;
            }
        }
        e = launch(sv, h->q_stream[q]);
        if (e == cudaSuccess) e = cudaEventRecord(h->q_done[q], h->q_stream[q]);
        if (e != cudaSuccess) st = cuda_fail(e, "kernel launch");
    }
    for (int q = 0; q < h->nq; ++q) {
        if (!used[q]) continue;
        e = cudaEventRecord(h->q_done[q], h->q_stream[q]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->q_done[q], 0);
        if (e != cudaSuccess && st == BLCO_OK) st = cuda_fail(e, "queue join");
    }
    if (uploaded) {  // an upload whose kernel was never launched (an error) must not outlive the call
        e = cudaEventRecord(h->ev_fork, h->q_up);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_fork, 0);
        if (e != cudaSuccess && st == BLCO_OK) st = cuda_fail(e, "upload join");
    }
    return st;
}

// Rows of `mode` accumulated on chip: every row when the mode fits, else the
// mode's most frequent rows (by count).
HotRows hot_for(const blco_tensor *h, int mode, int R) {
    HotRows hr;
    hr.rows = h->d_hot[mode];
    hr.count = h->hot_count[mode];
    hr.dense = 0;
    if (h->L.dims[mode] <= warp_tier_capacity(R)) {
        hr.rows = nullptr;
        hr.count = (int)h->L.dims[mode];
        hr.dense = 1;
    }
    return hr;
}

// Device memory for n private output copies of `floats` each; false (and
// no error left pending) when it cannot be had, e.g. under a device budget.
bool copy_buffer(blco_tensor *h, size_t bytes, float **p) {
    if (bytes > h->copies_bytes) {
        h->dfree(h->d_copies, h->copies_bytes);
        h->d_copies = nullptr;
        h->copies_bytes = 0;
        if (h->dalloc((void **)&h->d_copies, bytes) != cudaSuccess) {
            cudaGetLastError();
            h->d_copies = nullptr;
            return false;
        }
        h->copies_bytes = bytes;
    }
    *p = h->d_copies;
    return true;
}

blco_status mttkrp_device(blco_tensor *h, int mode, const FactorSet &fs, blco_dtype fdt, int R, float *out,
                          const float *vals_ext, cudaStream_t s, int64_t range_begin = 0, int64_t range_end = -1) {
    const int64_t n = h->L.dims[mode] * (int64_t)R;
    const HotRows hot = hot_for(h, mode, R);
    // short modes: reduce into one private copy per SM, then sum the copies
    OutCopies oc;
    float *dst = out;
    const int nc = hot.dense ? 1 : output_copies(h->L.dims[mode], R);
    if (nc > 1 && copy_buffer(h, sizeof(float) * (size_t)nc * n, &dst)) {
        oc.n = nc;
        oc.stride = n;
    } else {
        dst = out;
    }
    cudaError_t e = timed(h, "zero", s, [&]() { return launch_zero(dst, n * oc.n, s); });
    if (e != cudaSuccess) return cuda_fail(e, "zero output");
    blco_status st = over_store(
        h, "mttkrp", vals_ext, s,
        [&](const StoreView &sv, cudaStream_t q) {
            return launch_mttkrp(sv, fs, fdt, R, mode, hot, dst, oc, h->compensated, q);
        },
        range_begin, range_end);
    if (st != BLCO_OK || oc.n == 1) return st;
    e = timed(h, "sum_copies", s, [&]() { return launch_sum_copies(dst, oc.n, n, out, s); });
    if (e != cudaSuccess) return cuda_fail(e, "sum of output copies");
    return BLCO_OK;
}

blco_status check_common(blco_tensor *h, blco_dtype fdt, int R) {
    if (!h) return fail(BLCO_ERR_ARG, "handle is NULL");
    if (h->f64) return fail(BLCO_ERR_STATE, "the store holds float64 values; use blco_mttkrp_f64");
    if (!dtype_ok(fdt)) return fail(BLCO_ERR_ARG, "unknown factor dtype");
    if (!rank_supported(R)) return fail(BLCO_ERR_UNSUPPORTED, "rank must be 8, 16, 32, 64 or 128");
    return BLCO_OK;
}

}  // namespace

extern "C" {

const char *blco_last_error(void) { return g_err.c_str(); }

blco_status blco_inject_fault(int kind, int64_t k) {
    if (kind != BLCO_FAULT_ALLOC && kind != BLCO_FAULT_COPY) return fail(BLCO_ERR_ARG, "unknown fault kind");
    if (k < 0) return fail(BLCO_ERR_ARG, "k must be >= 0");
    g_fault_left[kind].store((long)k);
    return BLCO_OK;
}

blco_status blco_default_opts(blco_build_opts *o) {
    if (!o) return fail(BLCO_ERR_ARG, "opts is NULL");
    memset(o, 0, sizeof(*o));
    o->max_nnz_per_block = kDefaultCap;
    o->line_bits = 64;
    o->n_queues = 8;
    return BLCO_OK;
}

// blco_build, and blco_build_f64's store without float32 values (vals NULL)
static blco_status build_impl(const uint32_t *coords, const float *vals, int64_t nnz, const int64_t *dims, int N,
                              const blco_build_opts *opts, blco_stream stream, blco_handle *out, bool no_vals) {
    g_err.clear();
    if (!out) return fail(BLCO_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (N < 1 || N > MAXN) return fail(BLCO_ERR_ARG, "order N must be in 1..8");
    if (!dims) return fail(BLCO_ERR_ARG, "dims is NULL");
    if (nnz < 0 || nnz >= ((int64_t)1 << 32) - 64) return fail(BLCO_ERR_ARG, "nnz must be in 0..2^32-65");
    if (nnz > 0 && (!coords || (!vals && !no_vals))) return fail(BLCO_ERR_ARG, "coords/vals is NULL");
    blco_build_opts o;
    blco_default_opts(&o);
    if (opts) {
        if (opts->max_nnz_per_block < 0 || opts->line_bits < 0 || opts->line_bits > 64 || opts->n_queues < 0 ||
            opts->n_queues > 8 || opts->device_budget_bytes < 0)
            return fail(BLCO_ERR_ARG, "bad build option");
        if (opts->max_nnz_per_block) o.max_nnz_per_block = opts->max_nnz_per_block;
        if (opts->line_bits) o.line_bits = opts->line_bits;
        if (opts->n_queues) o.n_queues = opts->n_queues;
        o.device_budget_bytes = opts->device_budget_bytes;
        o.force_stream = opts->force_stream;
        o.compensated_sums = opts->compensated_sums;
        o.host_reads = opts->host_reads;
    }
    blco_tensor *h = new blco_tensor();
    h->L.N = N;
    for (int n = 0; n < N; ++n) h->L.dims[n] = dims[n];
    h->L.line = o.line_bits;
    std::string why;
    if (!plan_layout(h->L, why)) {
        delete h;
        return fail(BLCO_ERR_ARG, why);
    }
    h->nnz = nnz;
    h->building = true;
    h->npad = ((nnz + 31) / 32) * 32 + 32;
    h->max_nnz = o.max_nnz_per_block;
    h->nq = o.n_queues;
    h->budget = o.device_budget_bytes;
    h->compensated = o.compensated_sums != 0;
    if (cudaGetDevice(&h->device) != cudaSuccess) {
        cudaGetLastError();
        delete h;
        return fail(BLCO_ERR_CUDA, "no CUDA device");
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    const uint32_t *dc = coords;
    const float *dv = vals;
    uint32_t *tc = nullptr;
    float *tv = nullptr;
    blco_status st = BLCO_OK;
    BuildOut bo;
#define BAIL(status_expr)       \
    do {                        \
        st = (status_expr);     \
        goto cleanup;           \
    } while (0)
    if (nnz > 0 && !is_device_ptr(coords)) {
        e = cudaMallocAsync(&tc, sizeof(uint32_t) * nnz * N, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tc, coords, sizeof(uint32_t) * nnz * N, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) BAIL(cuda_fail(e, "coordinate upload"));
        dc = tc;
    }
    if (nnz > 0 && vals && !is_device_ptr(vals)) {
        e = cudaMallocAsync(&tv, sizeof(float) * nnz, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tv, vals, sizeof(float) * nnz, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) BAIL(cuda_fail(e, "value upload"));
        dv = tv;
    }
    if (fault_now(BLCO_FAULT_ALLOC)) BAIL(fail(BLCO_ERR_OOM, "injected allocation fault (construction scratch)"));
    e = build_store(h->L, dc, dv, nnz, h->max_nnz, bo, s, why);
    if (e != cudaSuccess) BAIL(cuda_fail(e, "store construction"));
    if (bo.first_bad >= 0) BAIL(fail(BLCO_ERR_INDEX, why));
    h->d_keys = bo.keys;
    h->d_vals = bo.vals;
    h->d_perm = bo.perm;
    bo.keys = nullptr;
    bo.vals = nullptr;
    bo.perm = nullptr;
    h->dev_bytes += h->npad * 12 + nnz * 4;
    h->bstart = bo.bstart;
    h->bhigh = bo.bhigh;
    {
        const int64_t nb = (int64_t)h->bstart.size() - 1;
        bool zero_high = true;
        for (uint32_t v : h->bhigh) zero_high &= (v == 0);
        // all-zero high bits (one block, or one block split at the cap): no
        // per-tile block lookups are needed to de-linearize
        h->single_block = zero_high;
        std::vector<uint32_t> bbase((size_t)std::max<int64_t>(nb, 1) * MAXN, 0u);
        for (int64_t b = 0; b < nb; ++b)
            for (int n = 0; n < N; ++n)
                bbase[b * MAXN + n] = h->L.width[n] >= 32 ? 0u : (h->bhigh[b * N + n] << h->L.width[n]);
        e = h->dalloc((void **)&h->d_bstart, sizeof(int64_t) * (nb + 1));
        if (e == cudaSuccess) e = h->dalloc((void **)&h->d_bbase, sizeof(uint32_t) * bbase.size());
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->d_bstart, h->bstart.data(), sizeof(int64_t) * (nb + 1), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(h->d_bbase, bbase.data(), sizeof(uint32_t) * bbase.size(), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess && !h->single_block && nnz > 0) {
            e = h->dalloc((void **)&h->d_tile_block, sizeof(uint32_t) * ((nnz + 31) / 32));
            if (e == cudaSuccess) e = build_tile_block(h->d_bstart, nb, nnz, h->d_tile_block, s);
        }
        if (e != cudaSuccess) BAIL(cuda_fail(e, "block table"));
    }
    // hot rows per mode (histogram of the stored indices, top counts)
    if (nnz > 0) {
        uint32_t *counts = nullptr;
        for (int n = 0; n < N && e == cudaSuccess; ++n) {
            const int64_t I = h->L.dims[n];
            // as many rows as the smallest supported rank can hold on chip
            const int k = (int)std::min<int64_t>(I, warp_tier_capacity(8));
            e = cudaMallocAsync(&counts, sizeof(uint32_t) * I, s);
            if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * I, s);
            if (e == cudaSuccess) e = mode_histogram(h->view(), n, counts, s);
            if (e == cudaSuccess) e = h->dalloc((void **)&h->d_hot[n], sizeof(uint32_t) * k);
            if (e == cudaSuccess) e = top_rows(counts, I, k, h->d_hot[n], s);
            h->hot_count[n] = k;
            if (counts) cudaFreeAsync(counts, s);
            counts = nullptr;
        }
        if (e != cudaSuccess) BAIL(cuda_fail(e, "hot rows"));
    }
    // residency: keep the store on the device, or move it to pinned host
    // memory and reserve device queues (Section 4.2)
    {
        int64_t maxblk = 1;
        for (size_t b = 0; b + 1 < h->bstart.size(); ++b) maxblk = std::max(maxblk, h->bstart[b + 1] - h->bstart[b]);
        const int64_t store_bytes = h->npad * 12 + nnz * 4;
        const bool over = h->budget > 0 && h->dev_bytes > h->budget;
        if (o.force_stream || over) {
            h->streamed = true;
            h->queue_nnz = ((std::max(maxblk, std::min(h->max_nnz, nnz)) + 31) / 32) * 32;
            // mapped: with host_reads the kernels load keys and values from here
            e = cudaHostAlloc((void **)&h->h_keys, sizeof(uint64_t) * h->npad, cudaHostAllocMapped);
            if (e == cudaSuccess) e = cudaHostAlloc((void **)&h->h_vals, sizeof(float) * h->npad, cudaHostAllocMapped);
            if (e == cudaSuccess) e = cudaHostAlloc((void **)&h->h_perm, sizeof(uint32_t) * std::max<int64_t>(nnz, 1), cudaHostAllocDefault);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_keys, h->d_keys, sizeof(uint64_t) * h->npad, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_vals, h->d_vals, sizeof(float) * h->npad, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(h->h_perm, h->d_perm, sizeof(uint32_t) * nnz, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) BAIL(cuda_fail(e, "move store to host"));
            h->host_bytes = store_bytes;
            cudaFree(h->d_keys);
            cudaFree(h->d_vals);
            cudaFree(h->d_perm);
            h->d_keys = nullptr;
            h->d_vals = nullptr;
            h->d_perm = nullptr;
            h->dev_bytes -= store_bytes;
            if (o.host_reads) {
                // the kernels read the store where it is: device views of the
                // mapped host arrays, no queues or batches
                h->host_reads = true;
                h->nq = 0;
                h->queue_nnz = 0;
                void *dk = nullptr, *dv = nullptr;
                e = cudaHostGetDevicePointer(&dk, h->h_keys, 0);
                if (e == cudaSuccess) e = cudaHostGetDevicePointer(&dv, h->h_vals, 0);
                if (e != cudaSuccess) BAIL(cuda_fail(e, "device view of the host store"));
                h->hd_keys = static_cast<uint64_t *>(dk);
                h->hd_vals = static_cast<float *>(dv);
                h->building = false;
            } else {
                // queues: as many as the budget allows (at least one)
                const int64_t qbytes = h->queue_nnz * 12;
                while (h->nq > 1 && h->budget > 0 && h->dev_bytes + h->nq * qbytes > h->budget) h->nq--;
                if (h->budget > 0 && h->dev_bytes + h->nq * qbytes > h->budget)
                    BAIL(fail(BLCO_ERR_OOM, "device budget cannot hold one queue reservation; lower max_nnz_per_block"));
                h->building = false;
                for (int q = 0; q < h->nq && e == cudaSuccess; ++q) {
                    e = h->dalloc((void **)&h->q_keys[q], sizeof(uint64_t) * h->queue_nnz);
                    if (e == cudaSuccess) e = h->dalloc((void **)&h->q_vals[q], sizeof(float) * h->queue_nnz);
                    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->q_stream[q], cudaStreamNonBlocking);
                    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->q_done[q], cudaEventDisableTiming);
                    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->q_copied[q], cudaEventDisableTiming);
                }
                if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
                if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->q_up, cudaStreamNonBlocking);
                if (e != cudaSuccess) BAIL(cuda_fail(e, "queue reservation"));
                // batches: consecutive whole blocks up to the reservation (Section 4.2)
                int64_t b0 = 0;
                const int64_t nb = (int64_t)h->bstart.size() - 1;
                while (b0 < nb) {
                    int64_t b1 = b0 + 1;
                    while (b1 < nb && h->bstart[b1 + 1] - h->bstart[b0] <= h->queue_nnz) ++b1;
                    h->batches.push_back({h->bstart[b0], h->bstart[b1]});
                    b0 = b1;
                }
            }
        } else if (h->budget > 0 && h->dev_bytes > h->budget) {
            BAIL(fail(BLCO_ERR_OOM, "device budget exceeded"));
        }
    }
    h->building = false;
    if (h->budget > 0 && h->dev_bytes > h->budget) BAIL(fail(BLCO_ERR_OOM, "device budget exceeded"));
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) BAIL(cuda_fail(e, "construction"));
cleanup:
#undef BAIL
    if (tc) cudaFreeAsync(tc, s);
    if (tv) cudaFreeAsync(tv, s);
    if (bo.keys) cudaFree(bo.keys);
    if (bo.vals) cudaFree(bo.vals);
    if (bo.perm) cudaFree(bo.perm);
    if (st != BLCO_OK) {
        cudaStreamSynchronize(s);
        cudaGetLastError();
        release(h);
        return st;
    }
    cudaStreamSynchronize(s);
    *out = h;
    return BLCO_OK;
}

blco_status blco_build(const uint32_t *coords, const float *vals, int64_t nnz, const int64_t *dims, int N,
                       const blco_build_opts *opts, blco_stream stream, blco_handle *out) {
    return build_impl(coords, vals, nnz, dims, N, opts, stream, out, false);
}

blco_status blco_build_f64(const uint32_t *coords, const double *vals, int64_t nnz, const int64_t *dims, int N,
                           const blco_build_opts *opts, blco_stream stream, blco_handle *out) {
    g_err.clear();
    if (!out) return fail(BLCO_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nnz > 0 && !vals) return fail(BLCO_ERR_ARG, "vals is NULL");
    if (opts && opts->force_stream) return fail(BLCO_ERR_UNSUPPORTED, "float64 stores are kept on the device");
    blco_handle h = nullptr;
    blco_status st = build_impl(coords, nullptr, nnz, dims, N, opts, stream, &h, true);
    if (st != BLCO_OK) return st;
    if (h->streamed) {
        release(h);
        return fail(BLCO_ERR_UNSUPPORTED, "float64 stores are kept on the device (the budget would stream it)");
    }
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const double *dv = vals;
    double *tv = nullptr;
    cudaError_t e = cudaSuccess;
    if (nnz > 0 && !is_device_ptr(vals)) {
        e = cudaMallocAsync(&tv, sizeof(double) * nnz, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(tv, vals, sizeof(double) * nnz, cudaMemcpyHostToDevice, s);
        dv = tv;
    }
    if (e == cudaSuccess) e = h->dalloc((void **)&h->d_vals64, sizeof(double) * h->npad);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->d_vals64, 0, sizeof(double) * h->npad, s);
    if (e == cudaSuccess) e = gather_f64(dv, h->d_perm, nnz, h->d_vals64, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (tv) cudaFreeAsync(tv, s);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(s);
        release(h);
        return cuda_fail(e, "float64 values");
    }
    h->dfree(h->d_vals, 0);  // the float32 values (zeros) are not kept
    h->dev_bytes -= (int64_t)sizeof(float) * h->npad;
    h->d_vals = nullptr;
    h->f64 = true;
    if (h->budget > 0 && h->dev_bytes > h->budget) {
        release(h);
        return fail(BLCO_ERR_OOM, "device budget exceeded");
    }
    *out = h;
    return BLCO_OK;
}

blco_status blco_mttkrp_f64(blco_handle h, int mode, const double *const *factors, int R, double *out,
                            blco_stream stream) {
    g_err.clear();
    if (!h) return fail(BLCO_ERR_ARG, "handle is NULL");
    if (!h->f64) return fail(BLCO_ERR_STATE, "the store holds float32 values; use blco_mttkrp");
    if (!rank_supported_f64(R)) return fail(BLCO_ERR_UNSUPPORTED, "rank must be 8, 16, 32 or 64");
    if (mode < 0 || mode >= h->L.N) return fail(BLCO_ERR_ARG, "mode out of range");
    if (!out) return fail(BLCO_ERR_ARG, "out is NULL");
    if (reinterpret_cast<uintptr_t>(out) & 15) return fail(BLCO_ERR_ARG, "out is not 16-byte aligned");
    std::string why;
    if (!check_factors(h, reinterpret_cast<const void *const *>(factors), mode, why)) return fail(BLCO_ERR_ARG, why);
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // host arguments are staged in the workspace
    const int N = h->L.N;
    bool host_in[MAXN] = {};
    size_t off[MAXN] = {}, total = 0;
    for (int k = 0; k < N; ++k) {
        if (k == mode) continue;
        host_in[k] = !is_device_ptr(factors[k]);
        if (host_in[k]) {
            off[k] = total;
            total += ((size_t)h->L.dims[k] * R * sizeof(double) + 255) / 256 * 256;
        }
    }
    const bool host_out = !is_device_ptr(out);
    const size_t out_bytes = (size_t)h->L.dims[mode] * R * sizeof(double);
    const size_t out_off = total;
    if (host_out) total += (out_bytes + 255) / 256 * 256;
    char *base = nullptr;
    if (total > 0) {
        void *p = nullptr;
        cudaError_t e = h->workspace(total, &p);
        if (e != cudaSuccess) return cuda_fail(e, "staging workspace");
        base = static_cast<char *>(p);
    }
    const double *fs[MAXN] = {};
    for (int k = 0; k < N; ++k) {
        if (k == mode) continue;
        fs[k] = factors[k];
        if (host_in[k]) {
            cudaError_t e = cudaMemcpyAsync(base + off[k], factors[k], (size_t)h->L.dims[k] * R * sizeof(double),
                                            cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return cuda_fail(e, "factor upload");
            fs[k] = reinterpret_cast<const double *>(base + off[k]);
        }
    }
    double *o = host_out ? reinterpret_cast<double *>(base + out_off) : out;
    HotRows hot;
    hot.rows = h->d_hot[mode];
    hot.count = h->hot_count[mode];
    hot.dense = 0;
    if (h->L.dims[mode] <= warp_tier_capacity_f64(R)) {
        hot.rows = nullptr;
        hot.count = (int)h->L.dims[mode];
        hot.dense = 1;
    }
    const int64_t n = h->L.dims[mode] * (int64_t)R;
    cudaError_t e = timed(h, "zero", s, [&]() { return launch_zero(reinterpret_cast<float *>(o), 2 * n, s); });
    if (e != cudaSuccess) return cuda_fail(e, "zero output");
    if (h->nnz > 0) {
        StoreView sv = h->view();
        e = timed(h, "mttkrp_f64", s, [&]() { return launch_mttkrp_f64(sv, fs, R, mode, hot, o, s); });
        if (e != cudaSuccess) return cuda_fail(e, "kernel launch");
    }
    if (host_out) {
        e = cudaMemcpyAsync(out, o, out_bytes, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "result download");
    }
    if (total > 0) {
        e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "mttkrp_f64");
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mttkrp_f64");
    return BLCO_OK;
}

blco_status blco_mttkrp(blco_handle h, int mode, const void *const *factors, blco_dtype fdt, int R, float *out,
                        blco_stream stream) {
    g_err.clear();
    blco_status st = check_common(h, fdt, R);
    if (st != BLCO_OK) return st;
    if (mode < 0 || mode >= h->L.N) return fail(BLCO_ERR_ARG, "mode out of range");
    if (!out) return fail(BLCO_ERR_ARG, "out is NULL");
    if (reinterpret_cast<uintptr_t>(out) & 15) return fail(BLCO_ERR_ARG, "out is not 16-byte aligned");
    std::string why;
    if (!check_factors(h, factors, mode, why)) return fail(BLCO_ERR_ARG, why);
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool host_out = !is_device_ptr(out);
    const size_t out_bytes = (size_t)h->L.dims[mode] * R * sizeof(float);
    Staged sf;
    void *dout = nullptr;
    st = stage_factors(h, factors, mode, fdt, R, host_out ? out_bytes : 0, sf, &dout, s);
    if (st != BLCO_OK) return st;
    float *o = host_out ? static_cast<float *>(dout) : out;
    st = mttkrp_device(h, mode, sf.fs, fdt, R, o, nullptr, s);
    if (st != BLCO_OK) return st;
    if (host_out) {
        cudaError_t e = cudaMemcpyAsync(out, o, out_bytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "result download");
    } else if (sf.used > 0) {
        cudaError_t e = cudaStreamSynchronize(s);  // staged inputs live in the workspace
        if (e != cudaSuccess) return cuda_fail(e, "mttkrp");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mttkrp");
    return BLCO_OK;
}

blco_status blco_partition(int64_t nnz, int nparts, int64_t *bounds) {
    g_err.clear();
    if (!bounds) return fail(BLCO_ERR_ARG, "bounds is NULL");
    if (nparts < 1) return fail(BLCO_ERR_ARG, "nparts must be >= 1");
    if (nnz < 0 || nnz >= ((int64_t)1 << 32)) return fail(BLCO_ERR_ARG, "nnz must be in 0..2^32-1");
    // equal shares of the store order, cut at multiples of 32 positions
    bounds[0] = 0;
    for (int i = 1; i < nparts; ++i) {
        const int64_t b = nnz * i / nparts / 32 * 32;  // nnz < 2^32, i < 2^31: no overflow
        bounds[i] = std::max(bounds[i - 1], b);
    }
    bounds[nparts] = nnz;
    return BLCO_OK;
}

blco_status blco_mttkrp_range(blco_handle h, int mode, int64_t begin, int64_t end, const void *const *factors,
                              blco_dtype fdt, int R, float *out, blco_stream stream) {
    g_err.clear();
    blco_status st = check_common(h, fdt, R);
    if (st != BLCO_OK) return st;
    if (h->streamed && !h->host_reads)
        return fail(BLCO_ERR_STATE, "blco_mttkrp_range needs a store on the device or read in host memory (host_reads)");
    if (mode < 0 || mode >= h->L.N) return fail(BLCO_ERR_ARG, "mode out of range");
    if (begin < 0 || end < begin || end > h->nnz) return fail(BLCO_ERR_ARG, "range outside the store");
    if (begin % 32 != 0) return fail(BLCO_ERR_ARG, "begin must be a multiple of 32");
    if (!out) return fail(BLCO_ERR_ARG, "out is NULL");
    if (reinterpret_cast<uintptr_t>(out) & 15) return fail(BLCO_ERR_ARG, "out is not 16-byte aligned");
    std::string why;
    if (!check_factors(h, factors, mode, why)) return fail(BLCO_ERR_ARG, why);
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool host_out = !is_device_ptr(out);
    const size_t out_bytes = (size_t)h->L.dims[mode] * R * sizeof(float);
    Staged sf;
    void *dout = nullptr;
    st = stage_factors(h, factors, mode, fdt, R, host_out ? out_bytes : 0, sf, &dout, s);
    if (st != BLCO_OK) return st;
    float *o = host_out ? static_cast<float *>(dout) : out;
    st = mttkrp_device(h, mode, sf.fs, fdt, R, o, nullptr, s, begin, end);
    if (st != BLCO_OK) return st;
    if (host_out) {
        cudaError_t e = cudaMemcpyAsync(out, o, out_bytes, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "result download");
    } else if (sf.used > 0) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "mttkrp_range");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "mttkrp_range");
    return BLCO_OK;
}

// Streams and events of the pipelined host-argument path.
cudaError_t copy_streams(blco_tensor *h) {
    if (h->up) return cudaSuccess;
    cudaError_t e = cudaStreamCreateWithFlags(&h->up, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->down, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_call, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_down, cudaEventDisableTiming);
    for (int n = 0; n < MAXN && e == cudaSuccess; ++n) {
        e = cudaEventCreateWithFlags(&h->ev_up[n], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_out[n], cudaEventDisableTiming);
    }
    return e;
}

// All-mode MTTKRP in one pass over the store: on a streamed store every
// batch of blocks crosses the host link once per call (Section 4.2), and
// while it sits in its queue's reservation either the fused all-mode kernel
// (`fused`: each nonzero's N rows gathered once for every mode) or the
// kernels of all requested modes, one after another, run on it; on a
// resident store the same launches run once over the whole store. Host
// arguments are staged in the workspace: factors uploaded on `s` first,
// results downloaded at the end. Short modes accumulate straight into their
// outputs here (no private copies: their buffer holds one mode at a time).
static blco_status mttkrp_all_onepass(blco_tensor *h, FactorSet fs, const bool *host_in, const bool *host_out,
                                       const size_t *in_off, const size_t *out_off, size_t total, blco_dtype fdt, int R,
                                       float *const *outs, cudaStream_t s, bool fused) {
    const int N = h->L.N;
    char *base = nullptr;
    if (total > 0) {
        void *p = nullptr;
        cudaError_t e = h->workspace(total, &p);
        if (e != cudaSuccess) return cuda_fail(e, "staging workspace");
        base = static_cast<char *>(p);
    }
    float *dst[MAXN] = {};
    HotRows hot[MAXN];
    for (int k = 0; k < N; ++k) {
        if (!host_in[k]) continue;
        cudaError_t e = cudaMemcpyAsync(base + in_off[k], fs.ptr[k], (size_t)h->L.dims[k] * R * dtype_size(fdt),
                                        cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "factor upload");
        fs.ptr[k] = base + in_off[k];
    }
    for (int n = 0; n < N; ++n) {
        if (!outs[n]) continue;
        dst[n] = host_out[n] ? reinterpret_cast<float *>(base + out_off[n]) : outs[n];
        hot[n] = hot_for(h, n, R);
        const int64_t cnt = h->L.dims[n] * (int64_t)R;
        cudaError_t e = timed(h, "zero", s, [&]() { return launch_zero(dst[n], cnt, s); });
        if (e != cudaSuccess) return cuda_fail(e, "zero output");
    }
    const OutCopies one;
    HotRows hot_all[MAXN];
    for (int n = 0; n < N; ++n) {
        hot_all[n].rows = h->d_hot[n];
        hot_all[n].count = h->hot_count[n];
        hot_all[n].dense = 0;
    }
    float *dst_all[MAXN] = {};
    for (int n = 0; n < N; ++n) dst_all[n] = outs[n] ? dst[n] : nullptr;
    blco_status st = over_store(h, nullptr, nullptr, s, [&](const StoreView &sv, cudaStream_t q) {
        if (fused)
            return timed(h, "mttkrp_all_fused", q,
                         [&]() { return launch_mttkrp_fused(sv, fs, fdt, R, hot_all, dst_all, q); });
        for (int n = 0; n < N; ++n) {
            if (!outs[n]) continue;
            cudaError_t e = timed(h, "mttkrp", q, [&]() {
                return launch_mttkrp(sv, fs, fdt, R, n, hot[n], dst[n], one, h->compensated, q);
            });
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    });
    if (st != BLCO_OK) return st;
    for (int n = 0; n < N; ++n) {
        if (!outs[n] || !host_out[n]) continue;
        cudaError_t e = cudaMemcpyAsync(outs[n], dst[n], (size_t)h->L.dims[n] * R * sizeof(float),
                                        cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "result download");
    }
    if (total > 0) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "mttkrp_all");
    }
    return BLCO_OK;
}

blco_status blco_mttkrp_all(blco_handle h, const void *const *factors, blco_dtype fdt, int R, float *const *outs,
                            blco_stream stream) {
    g_err.clear();
    blco_status st = check_common(h, fdt, R);
    if (st != BLCO_OK) return st;
    if (!outs) return fail(BLCO_ERR_ARG, "outs is NULL");
    std::string why;
    if (!check_factors(h, factors, -1, why)) return fail(BLCO_ERR_ARG, why);
    for (int n = 0; n < h->L.N; ++n)
        if (outs[n] && (reinterpret_cast<uintptr_t>(outs[n]) & 15)) return fail(BLCO_ERR_ARG, "outs[n] is not 16-byte aligned");
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int N = h->L.N;
    bool host_in[MAXN] = {}, host_out[MAXN] = {};
    size_t in_off[MAXN] = {}, out_off[MAXN] = {}, total = 0;
    auto round256 = [](size_t b) { return (b + 255) / 256 * 256; };
    for (int k = 0; k < N; ++k) {
        host_in[k] = !is_device_ptr(factors[k]);
        if (host_in[k]) {
            in_off[k] = total;
            total += round256((size_t)h->L.dims[k] * R * dtype_size(fdt));
        }
    }
    for (int n = 0; n < N; ++n) {
        host_out[n] = outs[n] && !is_device_ptr(outs[n]);
        if (host_out[n]) {
            out_off[n] = total;
            total += round256((size_t)h->L.dims[n] * R * sizeof(float));
        }
    }
    FactorSet fs;
    for (int k = 0; k < MAXN; ++k) fs.ptr[k] = k < N ? factors[k] : nullptr;
    const bool fused = fused_supported(h->view(), R);
    // a store streamed through the queues crosses the host link once per call
    // (one pass, every mode on each batch); a store read in host memory runs
    // the per-mode kernels over it one mode after another, like a resident one
    if (fused || (h->streamed && !h->host_reads))
        return mttkrp_all_onepass(h, fs, host_in, host_out, in_off, out_off, total, fdt, R, outs, s, fused);
    if (total == 0) {  // device arguments: the modes one after another on s
        for (int n = 0; n < N; ++n) {
            if (!outs[n]) continue;
            st = mttkrp_device(h, n, fs, fdt, R, outs[n], nullptr, s);
            if (st != BLCO_OK) return st;
        }
        return BLCO_OK;
    }
    // Host arguments. Uploads run on h->up in the order the modes need them
    // (modes 1..N-1 first: mode 0's kernel overlaps the upload of factor 0);
    // each mode waits only for the factors it gathers; each host result is
    // downloaded on h->down as soon as its mode is done, overlapping the next
    // mode. The call joins both copy streams into s and returns when the host
    // results are complete.
    void *p = nullptr;
    cudaError_t e = h->workspace(total, &p);
    if (e != cudaSuccess) return cuda_fail(e, "staging workspace");
    char *base = static_cast<char *>(p);
    e = copy_streams(h);
    if (e != cudaSuccess) return cuda_fail(e, "copy streams");
    e = cudaEventRecord(h->ev_call, s);  // earlier work on s may still use the workspace
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->up, h->ev_call, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(h->down, h->ev_call, 0);
    if (e != cudaSuccess) return cuda_fail(e, "copy streams");
    bool uploaded = false, downloaded = false;
    for (int i = 0; i < N && st == BLCO_OK; ++i) {
        const int k = (i + 1) % N;
        if (!host_in[k]) continue;
        e = cudaMemcpyAsync(base + in_off[k], factors[k], (size_t)h->L.dims[k] * R * dtype_size(fdt),
                            cudaMemcpyHostToDevice, h->up);
        if (e == cudaSuccess) e = cudaEventRecord(h->ev_up[k], h->up);
        if (e != cudaSuccess) st = cuda_fail(e, "factor upload");
        fs.ptr[k] = base + in_off[k];
        uploaded = true;
    }
    bool waited[MAXN] = {};
    for (int n = 0; n < N && st == BLCO_OK; ++n) {
        if (!outs[n]) continue;
        for (int k = 0; k < N && st == BLCO_OK; ++k) {
            if (k == n || !host_in[k] || waited[k]) continue;
            e = cudaStreamWaitEvent(s, h->ev_up[k], 0);
            if (e != cudaSuccess) st = cuda_fail(e, "stream wait");
            waited[k] = true;
        }
        if (st != BLCO_OK) break;
        float *o = host_out[n] ? reinterpret_cast<float *>(base + out_off[n]) : outs[n];
        st = mttkrp_device(h, n, fs, fdt, R, o, nullptr, s);
        if (st != BLCO_OK || !host_out[n]) continue;
        e = cudaEventRecord(h->ev_out[n], s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(h->down, h->ev_out[n], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(outs[n], o, (size_t)h->L.dims[n] * R * sizeof(float), cudaMemcpyDeviceToHost, h->down);
        if (e != cudaSuccess) st = cuda_fail(e, "result download");
        downloaded = true;
    }
    // join the copy streams into s (also after an error: nothing of this call
    // may outlive it on the copy streams)
    for (cudaStream_t cs : {h->up, h->down}) {
        if ((cs == h->up && !uploaded) || (cs == h->down && !downloaded)) continue;
        e = cudaEventRecord(h->ev_down, cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, h->ev_down, 0);
        if (e != cudaSuccess && st == BLCO_OK) st = cuda_fail(e, "copy join");
    }
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess && st == BLCO_OK) st = cuda_fail(e, "mttkrp_all");
    return st;
}

blco_status blco_cp_fwd(blco_handle h, const void *const *factors, blco_dtype fdt, int R, float *xhat,
                        blco_stream stream) {
    g_err.clear();
    blco_status st = check_common(h, fdt, R);
    if (st != BLCO_OK) return st;
    if (!xhat && h->nnz > 0) return fail(BLCO_ERR_ARG, "xhat is NULL");
    std::string why;
    if (!check_factors(h, factors, -1, why)) return fail(BLCO_ERR_ARG, why);
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool host_out = h->nnz > 0 && !is_device_ptr(xhat);
    Staged sf;
    void *dx = nullptr;
    st = stage_factors(h, factors, -1, fdt, R, host_out ? sizeof(float) * h->nnz : 0, sf, &dx, s);
    if (st != BLCO_OK) return st;
    float *o = host_out ? static_cast<float *>(dx) : xhat;
    st = over_store(h, "cp_fwd", nullptr, s, [&](const StoreView &sv, cudaStream_t q) {
        return launch_cp_fwd(sv, sf.fs, fdt, R, o, 0, q);
    });
    if (st != BLCO_OK) return st;
    if (host_out) {
        cudaError_t e = cudaMemcpyAsync(xhat, o, sizeof(float) * h->nnz, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "result download");
    }
    if (sf.used > 0) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "cp_fwd");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "cp_fwd");
    return BLCO_OK;
}

blco_status blco_cp_bwd(blco_handle h, int mode, const float *grad, const void *const *factors, blco_dtype fdt,
                        int R, float *out, blco_stream stream) {
    g_err.clear();
    blco_status st = check_common(h, fdt, R);
    if (st != BLCO_OK) return st;
    if (mode < 0 || mode >= h->L.N) return fail(BLCO_ERR_ARG, "mode out of range");
    if (!out) return fail(BLCO_ERR_ARG, "out is NULL");
    if (!grad && h->nnz > 0) return fail(BLCO_ERR_ARG, "grad is NULL");
    if (reinterpret_cast<uintptr_t>(out) & 15) return fail(BLCO_ERR_ARG, "out is not 16-byte aligned");
    std::string why;
    if (!check_factors(h, factors, mode, why)) return fail(BLCO_ERR_ARG, why);
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const bool host_out = !is_device_ptr(out);
    const bool host_grad = h->nnz > 0 && !is_device_ptr(grad);
    const size_t out_bytes = (size_t)h->L.dims[mode] * R * sizeof(float);
    const size_t gbytes = host_grad ? ((sizeof(float) * h->nnz + 255) / 256 * 256) : 0;
    Staged sf;
    void *dx = nullptr;
    st = stage_factors(h, factors, mode, fdt, R, gbytes + (host_out ? out_bytes : 0), sf, &dx, s);
    if (st != BLCO_OK) return st;
    const float *gd = grad;
    if (host_grad) {
        cudaError_t e = cudaMemcpyAsync(dx, grad, sizeof(float) * h->nnz, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return cuda_fail(e, "gradient upload");
        gd = static_cast<const float *>(dx);
    }
    float *o = host_out ? reinterpret_cast<float *>(static_cast<char *>(dx) + gbytes) : out;
    st = mttkrp_device(h, mode, sf.fs, fdt, R, o, gd, s);
    if (st != BLCO_OK) return st;
    if (host_out) {
        cudaError_t e = cudaMemcpyAsync(out, o, out_bytes, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) return cuda_fail(e, "result download");
    }
    if (sf.used > 0) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "cp_bwd");
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "cp_bwd");
    return BLCO_OK;
}

static blco_status copy_out(blco_tensor *h, void *dst, const void *dsrc, const void *hsrc, size_t bytes,
                            cudaStream_t s) {
    if (bytes == 0) return BLCO_OK;
    const bool ddst = is_device_ptr(dst);
    const void *src = h->streamed ? hsrc : dsrc;
    cudaMemcpyKind k = h->streamed ? (ddst ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost)
                                   : (ddst ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost);
    cudaError_t e = cudaMemcpyAsync(dst, src, bytes, k, s);
    if (e == cudaSuccess && (!ddst || h->streamed)) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "copy out");
    return BLCO_OK;
}

blco_status blco_values(blco_handle h, float *vals, blco_stream stream) {
    g_err.clear();
    if (!h || (!vals && h->nnz > 0)) return fail(BLCO_ERR_ARG, "NULL argument");
    if (h->f64) return fail(BLCO_ERR_STATE, "the store holds float64 values");
    DeviceGuard g(h->device);
    return copy_out(h, vals, h->d_vals, h->h_vals, sizeof(float) * h->nnz, reinterpret_cast<cudaStream_t>(stream));
}

blco_status blco_keys(blco_handle h, uint64_t *keys, blco_stream stream) {
    g_err.clear();
    if (!h || (!keys && h->nnz > 0)) return fail(BLCO_ERR_ARG, "NULL argument");
    DeviceGuard g(h->device);
    return copy_out(h, keys, h->d_keys, h->h_keys, sizeof(uint64_t) * h->nnz, reinterpret_cast<cudaStream_t>(stream));
}

blco_status blco_perm(blco_handle h, int64_t *perm, blco_stream stream) {
    g_err.clear();
    if (!h || (!perm && h->nnz > 0)) return fail(BLCO_ERR_ARG, "NULL argument");
    if (h->nnz == 0) return BLCO_OK;
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::vector<uint32_t> tmp((size_t)h->nnz);
    cudaError_t e = cudaMemcpyAsync(tmp.data(), h->streamed ? (const void *)h->h_perm : (const void *)h->d_perm,
                                    sizeof(uint32_t) * h->nnz,
                                    h->streamed ? cudaMemcpyHostToHost : cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "perm download");
    std::vector<int64_t> wide(tmp.begin(), tmp.end());
    if (is_device_ptr(perm)) {
        e = cudaMemcpyAsync(perm, wide.data(), sizeof(int64_t) * h->nnz, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(e, "perm upload");
    } else {
        memcpy(perm, wide.data(), sizeof(int64_t) * h->nnz);
    }
    return BLCO_OK;
}

blco_status blco_blocks(blco_handle h, int64_t *bstart, uint32_t *bhigh) {
    g_err.clear();
    if (!h || !bstart || !bhigh) return fail(BLCO_ERR_ARG, "NULL argument");
    memcpy(bstart, h->bstart.data(), sizeof(int64_t) * h->bstart.size());
    if (!h->bhigh.empty()) memcpy(bhigh, h->bhigh.data(), sizeof(uint32_t) * h->bhigh.size());
    return BLCO_OK;
}

blco_status blco_info(blco_handle h, blco_info_t *info) {
    g_err.clear();
    if (!h || !info) return fail(BLCO_ERR_ARG, "NULL argument");
    memset(info, 0, sizeof(*info));
    info->nnz = h->nnz;
    info->order = h->L.N;
    info->total_bits = h->L.B;
    for (int n = 0; n < h->L.N; ++n) {
        info->dims[n] = h->L.dims[n];
        info->mode_bits[n] = h->L.bits[n];
        info->block_bits[n] = h->L.kbits[n];
        info->hot_rows[n] = h->hot_count[n];
    }
    info->line_bits = h->L.line;
    info->streamed = h->streamed ? 1 : 0;
    info->nblocks = (int64_t)h->bstart.size() - 1;
    info->max_nnz_per_block = h->max_nnz;
    info->queue_nnz = h->queue_nnz;
    info->n_queues = h->streamed ? h->nq : 0;
    info->device_bytes = h->dev_bytes;
    info->host_bytes = h->host_bytes;
    info->host_reads = h->host_reads ? 1 : 0;
    return BLCO_OK;
}

blco_status blco_sync(blco_handle h) {
    g_err.clear();
    if (!h) return fail(BLCO_ERR_ARG, "handle is NULL");
    DeviceGuard g(h->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "sync");
    return BLCO_OK;
}

void blco_destroy(blco_handle h) { release(h); }

blco_status blco_convert(const float *src, void *dst, blco_dtype dt, int64_t n, blco_stream stream) {
    g_err.clear();
    if (n < 0) return fail(BLCO_ERR_ARG, "n < 0");
    if (n > 0 && (!src || !dst)) return fail(BLCO_ERR_ARG, "NULL argument");
    if (dt != BLCO_BF16 && dt != BLCO_F16) return fail(BLCO_ERR_ARG, "dt must be BLCO_BF16 or BLCO_F16");
    cudaError_t e = launch_convert(src, dst, dt, n, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "convert");
    return BLCO_OK;
}

blco_status blco_gram(const void *A, blco_dtype fdt, int64_t I, int R, double *G, blco_stream stream) {
    g_err.clear();
    if (!G || (I > 0 && !A)) return fail(BLCO_ERR_ARG, "NULL argument");
    if (I < 0 || R < 1 || R > 128) return fail(BLCO_ERR_ARG, "bad shape");
    if (!dtype_ok(fdt)) return fail(BLCO_ERR_ARG, "unknown dtype");
    cudaError_t e = launch_gram(A, fdt, I, R, G, reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "gram");
    return BLCO_OK;
}

blco_status blco_cpals_update(const double *const *grams, int N, int mode, int R, const float *M, int64_t I,
                              float *A, double *lambda, double *G_out, int32_t *info, blco_stream stream) {
    g_err.clear();
    if (!grams || !M || !A || !lambda || !info) return fail(BLCO_ERR_ARG, "NULL argument");
    if (N < 1 || N > MAXN || mode < 0 || mode >= N) return fail(BLCO_ERR_ARG, "bad order or mode");
    if (R < 1 || R > 64) return fail(BLCO_ERR_UNSUPPORTED, "rank must be in 1..64");
    for (int k = 0; k < N; ++k)
        if (k != mode && !grams[k]) return fail(BLCO_ERR_ARG, "grams[k] is NULL");
    cudaError_t e = launch_cpals_update(grams, N, mode, R, M, I, A, lambda, G_out, info,
                                        reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "cpals_update");
    return BLCO_OK;
}

blco_status blco_cpals_fit(double normX2, const double *const *grams, int N, int R, const double *lambda,
                           const float *M_last, const float *A_last, int64_t I_last, double *fit,
                           blco_stream stream) {
    g_err.clear();
    if (!grams || !lambda || !M_last || !A_last || !fit) return fail(BLCO_ERR_ARG, "NULL argument");
    if (N < 1 || N > MAXN || R < 1 || R > 128) return fail(BLCO_ERR_ARG, "bad shape");
    if (!(normX2 > 0.0)) return fail(BLCO_ERR_ARG, "normX2 must be > 0");
    for (int k = 0; k < N; ++k)
        if (!grams[k]) return fail(BLCO_ERR_ARG, "grams[k] is NULL");
    cudaError_t e = launch_cpals_fit(normX2, grams, N, R, lambda, M_last, A_last, I_last, fit,
                                     reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "cpals_fit");
    return BLCO_OK;
}

blco_status blco_norm2(blco_handle h, double *out, blco_stream stream) {
    g_err.clear();
    if (!h || !out) return fail(BLCO_ERR_ARG, "NULL argument");
    if (h->f64) return fail(BLCO_ERR_STATE, "the store holds float64 values");
    DeviceGuard g(h->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = launch_norm2(nullptr, 0, out, s);  // zeroes *out
    if (e != cudaSuccess) return cuda_fail(e, "norm2");
    return over_store(h, "norm2", nullptr, s, [&](const StoreView &sv, cudaStream_t q) {
        return launch_norm2_acc(sv.vals + (sv.begin - sv.val_origin), sv.end - sv.begin, out, q);
    });
}

blco_status blco_profile_enable(blco_handle h, int enable) {
    g_err.clear();
    if (!h) return fail(BLCO_ERR_ARG, "handle is NULL");
    h->profiling = enable != 0;
    return BLCO_OK;
}

blco_status blco_profile_read(blco_handle h, blco_profile_entry *entries, int capacity, int *count) {
    g_err.clear();
    if (!h || !count || (capacity > 0 && !entries)) return fail(BLCO_ERR_ARG, "NULL argument");
    DeviceGuard g(h->device);
    std::vector<blco_profile_entry> agg;
    cudaError_t first = cudaSuccess;
    for (auto &m : h->marks) {
        float ms = 0.f;
        cudaError_t e = cudaEventSynchronize(m.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, m.a, m.b);
        if (e != cudaSuccess && first == cudaSuccess) first = e;
        size_t i = 0;
        while (i < agg.size() && strncmp(agg[i].name, m.name, sizeof(agg[i].name)) != 0) ++i;
        if (i == agg.size()) {
            blco_profile_entry pe;
            memset(&pe, 0, sizeof(pe));
            strncpy(pe.name, m.name, sizeof(pe.name) - 1);
            agg.push_back(pe);
        }
        agg[i].launches += 1;
        agg[i].total_ms += ms;
        cudaEventDestroy(m.a);
        cudaEventDestroy(m.b);
    }
    h->marks.clear();
    const int n = (int)std::min<size_t>(agg.size(), (size_t)std::max(capacity, 0));
    for (int i = 0; i < n; ++i) entries[i] = agg[i];
    *count = n;
    if (first != cudaSuccess) return cuda_fail(first, "profile read");
    return BLCO_OK;
}

blco_status blco_cpals_update_noalloc(const double *const *grams, int N, int mode, int R, const float *M,
                                      int64_t I, float *A, double *lambda, double *G_out, int32_t *info,
                                      blco_stream stream) {
    g_err.clear();
    if (!grams || !M || !A || !lambda || !info) return fail(BLCO_ERR_ARG, "NULL argument");
    if (N < 1 || N > MAXN || mode < 0 || mode >= N) return fail(BLCO_ERR_ARG, "bad order or mode");
    if (R < 1 || R > cpals_update_noalloc_max_rank())
        return fail(BLCO_ERR_ARG, "rank exceeds the fixed scratch of blco_cpals_update_noalloc (R <= 64)");
    if (I < 0) return fail(BLCO_ERR_ARG, "I < 0");
    for (int k = 0; k < N; ++k)
        if (k != mode && !grams[k]) return fail(BLCO_ERR_ARG, "grams[k] is NULL");
    cudaError_t e = launch_cpals_update_noalloc(grams, N, mode, R, M, I, A, lambda, G_out, info,
                                                reinterpret_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e, "cpals_update_noalloc");
    return BLCO_OK;
}

}  // extern "C"
