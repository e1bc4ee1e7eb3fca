/*
 * blco.h -- C ABI of libblco.so: sparse MTTKRP over a blocked, linearized
 * coordinate (BLCO) store on one NVIDIA GB300 (sm_103a).
 *
 * The paper ("Efficient, Out-of-Memory Sparse MTTKRP on Massively Parallel
 * Architectures", ICS'22) states the problem this library solves:
 *   - Eq. 1 (Section 2.3): the mode-n MTTKRP of an N-mode sparse tensor X
 *     with factor matrices A_1..A_N is M = X_(n) (A_N (.) ... (.) A_{n+1}
 *     (.) A_{n-1} (.) ... (.) A_1), computed per nonzero as in Fig. 3:
 *     M[i_n, :] += x * (Hadamard product of rows A_k[i_k, :], k != n).
 *   - Section 4: the BLCO store -- each nonzero's N indices linearized in
 *     ALTO order (Section 4.1, Fig. 6a), re-encoded as concatenated per-mode
 *     bit fields so that de-linearization is shift and mask (Fig. 6b), the
 *     bits above a 64-bit encoding line kept once per block (Section 4.2),
 *     blocks split at a nonzero cap and streamed from host memory when the
 *     tensor exceeds the device (Section 4.2, device queues).
 *   - Algorithm 1 (Section 2.2): CP-ALS, whose per-mode update needs the
 *     MTTKRP and the Hadamard product of the other factors' Grams.
 *
 * Conventions for every call:
 *   - Indices are 0-based (the paper's figures are 1-based).
 *   - Matrices are row-major: a factor A_k is I_k x R with the rank index
 *     contiguous; an MTTKRP result is I_n x R float32.
 *   - "Store order" is the order of nonzeros inside the store: blocks by
 *     block key, ALTO order inside a block, input order among duplicates.
 *   - Pointers marked "host or device" are classified with
 *     cudaPointerGetAttributes: device and managed memory are used in place;
 *     host memory (pinned or pageable) is copied through library-owned device
 *     buffers inside the call.
 *   - Calls are stream-ordered on the given stream (NULL = the legacy
 *     default stream) and return before the GPU work completes, except where
 *     a host pointer is involved, in which case the call synchronizes the
 *     stream before returning so that host results are complete.
 *   - Argument errors return at once with no work enqueued. Errors of
 *     enqueued GPU work surface as BLCO_ERR_CUDA on a later call or on
 *     blco_sync. blco_last_error() gives a message for the calling thread.
 *   - The caller owns every pointer it passes; the handle owns the store,
 *     its block table, queue buffers, output copies and workspace, all freed
 *     by blco_destroy. A handle may be used by one thread at a time, and its
 *     calls must not overlap on the GPU: calls on different streams share
 *     those buffers, so order them (one stream, or events).
 */
#ifndef BLCO_H
#define BLCO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define BLCO_MAX_MODES 8

typedef struct blco_tensor *blco_handle;
/* A cudaStream_t (both are pointers to struct CUstream_st). */
typedef struct CUstream_st *blco_stream;

typedef enum {
    BLCO_OK = 0,
    BLCO_ERR_ARG = 1,         /* bad argument: null pointer, size, mode, rank, dtype */
    BLCO_ERR_INDEX = 2,       /* a coordinate is outside its mode's length */
    BLCO_ERR_OOM = 3,         /* device/host allocation failed or budget exceeded */
    BLCO_ERR_CUDA = 4,        /* a CUDA runtime call or kernel failed */
    BLCO_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    BLCO_ERR_STATE = 6,       /* handle in the wrong state for the call */
    BLCO_ERR_UNSUPPORTED = 7  /* a valid request the library does not implement (a rank other than 8, 16, 32, 64, 128) */
} blco_status;

typedef enum { BLCO_F32 = 0, BLCO_BF16 = 1, BLCO_F16 = 2 } blco_dtype;

/* Construction options (Section 4.2). Zero-initialized fields take defaults. */
typedef struct {
    int64_t max_nnz_per_block;   /* block cap; 0 = 2^27 (the paper's setting) */
    int32_t line_bits;           /* encoding line length, 1..64; 0 = 64 */
    int32_t n_queues;            /* streaming device queues, 1..8; 0 = 8 */
    int64_t device_budget_bytes; /* cap on this handle's device memory; 0 = none */
    int32_t force_stream;        /* 1 = keep the store in pinned host memory */
    int32_t compensated_sums;    /* 1 = with bf16/fp16 factors, sum each run of
                                    equal output rows with Kahan's compensated
                                    summation instead of plain float32 (about one
                                    rounding per run instead of one per term; the
                                    measured errors at the benchmark sizes are the
                                    same, and the plain sums are 8-10% faster) */
    int32_t host_reads;          /* streamed stores only: 1 = the kernels read the
                                    store's keys and values straight from its
                                    pinned host memory over the host link (one
                                    launch over the whole store; no device queues,
                                    no batch copies, no queue reservations in
                                    device memory). 0 (default) = the paper's
                                    scheme: batches of blocks copied into device
                                    queues on a side stream, overlapped with the
                                    kernels (Section 4.2). On a coherent host link
                                    (NVLink-C2C) the GPU's loads read pinned host
                                    memory at the link's copy rate. An all-mode
                                    call with the per-mode kernels (stores of
                                    other than 5 modes) reads the store once per
                                    mode this way, against once per call through
                                    the queues */
} blco_build_opts;

typedef struct {
    int64_t nnz;
    int32_t order;                         /* N */
    int32_t total_bits;                    /* B = sum_n ceil(log2 I_n) */
    int64_t dims[BLCO_MAX_MODES];
    int32_t mode_bits[BLCO_MAX_MODES];     /* b_n */
    int32_t block_bits[BLCO_MAX_MODES];    /* bits of mode n above the line */
    int32_t line_bits;
    int32_t streamed;                      /* 1 if the store lives in pinned host memory */
    int64_t nblocks;
    int64_t max_nnz_per_block;
    int64_t queue_nnz;                     /* per-queue reservation (streamed stores) */
    int32_t n_queues;
    int32_t hot_rows[BLCO_MAX_MODES];      /* hottest rows kept per mode (a launch at rank R
                                              accumulates the first min(this, 1024 / R)
                                              of them on chip) */
    int64_t device_bytes;                  /* device memory held by the handle */
    int64_t host_bytes;                    /* pinned host memory held by the handle */
    int32_t host_reads;                    /* 1 if kernels read the streamed store in host memory */
} blco_info_t;

/* Fills *opts with the defaults. Returns BLCO_ERR_ARG for a null pointer. */
blco_status blco_default_opts(blco_build_opts *opts);

/*
 * Builds the BLCO store of a COO tensor (Section 4: linearize in ALTO order,
 * stable sort, block by the bits above the line, split at the cap,
 * re-encode). All steps run on the current CUDA device.
 *   coords  nnz x N uint32, row-major, 0-based (host or device)
 *   vals    nnz float32 (host or device)
 *   dims    N mode lengths I_n >= 1 (host), N in 1..BLCO_MAX_MODES,
 *           sum of ceil(log2 I_n) <= 128, each I_n <= 2^32 - 1
 *   opts    NULL for the defaults
 *   stream  stream for the construction work; the call synchronizes it
 *   out     receives the handle (NULL on error)
 * Duplicate coordinates are kept as separate nonzeros (input order).
 * Errors: BLCO_ERR_ARG, BLCO_ERR_INDEX (a coordinate >= its I_n),
 * BLCO_ERR_OOM, BLCO_ERR_CUDA. nnz may be 0.
 */
blco_status blco_build(const uint32_t *coords, const float *vals, int64_t nnz, const int64_t *dims,
                       int N, const blco_build_opts *opts, blco_stream stream, blco_handle *out);

/*
 * Mode-`mode` MTTKRP (Eq. 1, Fig. 3) of the stored tensor:
 *   out[i, r] = sum over nonzeros with i_mode = i of x * prod_{k != mode} A_k[i_k, r].
 *   factors  N pointers (host or device); factors[k] is I_k x R of type fdt;
 *            factors[mode] is not read and may be NULL
 *   R        rank: 8, 16, 32, 64 or 128
 *   out      I_mode x R float32 (host or device); overwritten
 * Accumulation is float32 (segmented within a warp, then in per-warp
 * shared-memory copies of the mode's hottest rows, then vector reductions to
 * global memory), so the summation order, and the last bits, vary from run
 * to run. With bf16/fp16 factors each in-warp run is Kahan-compensated if
 * the handle was built with compensated_sums.
 * With any host pointer the call returns when `out` is complete; with device
 * pointers only it is asynchronous on `stream`.
 * Errors: BLCO_ERR_ARG, BLCO_ERR_UNSUPPORTED (rank), BLCO_ERR_OOM (staging),
 * BLCO_ERR_STATE (a store built with float64 values: blco_mttkrp_f64),
 * BLCO_ERR_CUDA.
 */
blco_status blco_mttkrp(blco_handle h, int mode, const void *const *factors, blco_dtype fdt, int R,
                        float *out, blco_stream stream);

/*
 * All-mode MTTKRP with one set of factors: outs[n] = mode-n MTTKRP for every
 * n with outs[n] != NULL (Eq. 1 for each mode, as the paper's all-mode
 * measurements do). Same arguments and errors as blco_mttkrp. Host factor
 * matrices are uploaded once for all modes, on a copy stream of the handle,
 * in the order the modes need them; each mode's kernel waits only for the
 * factors it gathers, and each host result is downloaded on a second copy
 * stream while the next mode runs. The call returns when the host results
 * are complete. On a store streamed through the device queues each batch
 * of blocks crosses the host link once per call: while it sits in its
 * queue's reservation the kernels of every requested mode run on it
 * (Section 4.2); the factors and all the requested outputs stay on the
 * device meanwhile. On a store read in host memory (host_reads) the kernels
 * load the store over the host link: once per call at 5 modes, once per
 * requested mode otherwise.
 * A 5-mode store (every I_n <= 2^24, R = 16, 32 or 64) is computed in one
 * pass: each nonzero's five factor rows are gathered once and its product
 * goes to every requested output (Eq. 1 for all modes at once), one kernel
 * launch per call (per batch when streamed). Other stores run the per-mode
 * kernels; the results agree within float32 rounding either way.
 */
blco_status blco_mttkrp_all(blco_handle h, const void *const *factors, blco_dtype fdt, int R,
                            float *const *outs, blco_stream stream);

/*
 * Partial MTTKRP over a contiguous part of the store, for splitting one
 * MTTKRP across devices or calls. MTTKRP is a sum over nonzeros (Eq. 1),
 * and the store's parts are independent of one another (Section 4.2: blocks
 * are processed independently), so the MTTKRP of the whole tensor is the sum
 * of the partial results of any set of parts that covers the store once; the
 * paper names distributed memory as future work (Section 8).
 *   blco_partition: for a store of nnz nonzeros (nnz < 2^32; no handle or
 *     device needed), bounds[0..nparts] (host) receives nparts contiguous
 *     ranges of store positions of (nearly) equal size, every bound but the
 *     last a multiple of 32; bounds[0] = 0, bounds[nparts] = nnz. A range may
 *     cut a block: a part needs no whole blocks, as every position's block
 *     is looked up.
 *   blco_mttkrp_range: out (I_mode x R float32, host or device, overwritten)
 *     = the mode-`mode` MTTKRP of the nonzeros at store positions
 *     [begin, end); begin a multiple of 32, 0 <= begin <= end <= nnz. Other
 *     arguments as blco_mttkrp. The store must be resident on the device
 *     or read in host memory (host_reads; BLCO_ERR_STATE for a store
 *     streamed through the device queues).
 * Errors: BLCO_ERR_ARG, BLCO_ERR_STATE, BLCO_ERR_UNSUPPORTED, BLCO_ERR_OOM,
 * BLCO_ERR_CUDA.
 */
blco_status blco_partition(int64_t nnz, int nparts, int64_t *bounds);
blco_status blco_mttkrp_range(blco_handle h, int mode, int64_t begin, int64_t end, const void *const *factors,
                              blco_dtype fdt, int R, float *out, blco_stream stream);

/*
 * float64 values, factors and accumulation -- the precision of the paper's
 * evaluation (Section 6: double-precision values). blco_build_f64 builds the
 * same store as blco_build (same keys, order, blocks) holding the values as
 * float64 (vals: nnz doubles, host or device); it keeps the store on the
 * device (BLCO_ERR_UNSUPPORTED when force_stream is set or the device budget
 * would stream it). blco_mttkrp_f64 is Eq. 1 on such a store:
 *   factors  N pointers (host or device) to I_k x R float64 matrices,
 *            factors[mode] not read
 *   R        8, 16, 32 or 64 (BLCO_ERR_UNSUPPORTED otherwise)
 *   out      I_mode x R float64 (host or device), overwritten
 * accumulated in float64 (run sums, per-warp shared-memory copies of the hot
 * rows, red.global.add.f64), so only the summation order differs from the
 * exact-rounding FP64 definition. A float64 store serves blco_mttkrp_f64,
 * blco_perm, blco_keys, blco_blocks, blco_info and blco_destroy; the float32
 * calls (blco_mttkrp*, blco_cp_*, blco_values, blco_norm2) return
 * BLCO_ERR_STATE on it, and blco_mttkrp_f64 on a float32 store too.
 */
blco_status blco_build_f64(const uint32_t *coords, const double *vals, int64_t nnz, const int64_t *dims, int N,
                           const blco_build_opts *opts, blco_stream stream, blco_handle *out);
blco_status blco_mttkrp_f64(blco_handle h, int mode, const double *const *factors, int R, double *out,
                            blco_stream stream);

/*
 * CP model at every stored nonzero (Algorithm 1's model, Section 2.2):
 *   xhat[j] = sum_r prod_n A_n[i_n^j, r], j in store order.
 *   factors  N matrices I_n x R (host or device); xhat: nnz float32 (host or device)
 */
blco_status blco_cp_fwd(blco_handle h, const void *const *factors, blco_dtype fdt, int R,
                        float *xhat, blco_stream stream);

/*
 * Adjoint of blco_cp_fwd for mode `mode`: given g = dL/dxhat (nnz float32,
 * store order, host or device), out = dL/dA_mode = mode-`mode` MTTKRP with g
 * in place of the tensor values (Eq. 1); row products are recomputed, not
 * stored. out: I_mode x R float32 (host or device), overwritten.
 */
blco_status blco_cp_bwd(blco_handle h, int mode, const float *grad, const void *const *factors,
                        blco_dtype fdt, int R, float *out, blco_stream stream);

/* Copies out the store: values (nnz float32), input positions (nnz int64:
 * store position -> input row), in-block keys (nnz uint64). Host or device
 * destinations. */
blco_status blco_values(blco_handle h, float *vals, blco_stream stream);
blco_status blco_perm(blco_handle h, int64_t *perm, blco_stream stream);
blco_status blco_keys(blco_handle h, uint64_t *keys, blco_stream stream);

/* Block table (host arrays): bstart[nblocks + 1] store offsets and
 * bhigh[nblocks * N] the per-mode index bits above each mode's in-block
 * field (i_n = (bhigh[b*N+n] << field_width_n) | field_n). */
blco_status blco_blocks(blco_handle h, int64_t *bstart, uint32_t *bhigh);

/* Shape, layout and memory of the handle. */
blco_status blco_info(blco_handle h, blco_info_t *info);

/* Waits for all of the handle's work; reports asynchronous GPU errors. */
blco_status blco_sync(blco_handle h);

/* Frees everything the handle owns (waits for its work first). NULL is a no-op. */
void blco_destroy(blco_handle h);

/* Message for the last failed call on the calling thread ("" if none). */
const char *blco_last_error(void);

/*
 * float32 -> bfloat16 / float16 conversion, round to nearest even (for
 * factor matrices stored at 16 bits). src: n float32 (device), dst: n 16-bit
 * values (device). dt must be BLCO_BF16 or BLCO_F16.
 */
blco_status blco_convert(const float *src, void *dst, blco_dtype dt, int64_t n, blco_stream stream);

/*
 * FP64 pieces of CP-ALS (Algorithm 1), on the device.
 *
 * blco_gram: G = A^T A (R x R float64, device), A is I x R of type fdt
 * (device), 1 <= R <= 128. Each thread sums its dot products with Dot2
 * (Ogita, Rump and Oishi, 2005): exact float32 products (TwoProduct by FMA)
 * and error-free additions (TwoSum), i.e. as if in twice the float32
 * precision; partials of threads and CTAs are added in float64. The error
 * is about 2^-48 of sum_i |A[i,r] A[i,c]| for typical data (the bound grows
 * with the square of the rows per thread times 2^-24).
 */
blco_status blco_gram(const void *A, blco_dtype fdt, int64_t I, int R, double *G, blco_stream stream);

/*
 * blco_cpals_update: the factor update of Algorithm 1 for one mode.
 *   grams   N device pointers to the R x R float64 Grams; grams[mode] unused
 *   M       I x R float32 MTTKRP of `mode` (device)
 *   A       I x R float32 output (device): A = M V^+ with V the Hadamard
 *           product of the other Grams, columns scaled to unit 2-norm
 *   lambda  R float64 output (device): the column norms removed from A
 *   G_out   R x R float64 output (device): Gram of the new A (may be NULL)
 *   info    1 int32 (device): 0 if every Cholesky pivot of V exceeded
 *           R * eps * max_i V_ii (Cholesky solve), 1 otherwise (V numerically
 *           singular or indefinite: the eigen pseudo-inverse, eigenvalues
 *           with |w| <= max|w| * R * eps dropped)
 * R in 1..64; larger ranks return BLCO_ERR_UNSUPPORTED.
 */
blco_status blco_cpals_update(const double *const *grams, int N, int mode, int R, const float *M,
                              int64_t I, float *A, double *lambda, double *G_out, int32_t *info,
                              blco_stream stream);

/*
 * blco_cpals_update_noalloc: the same update as blco_cpals_update (same
 * arguments, same result) without allocating any device memory. The paper
 * has no counterpart; it exists for callers that cannot let a library
 * allocate during a call -- a process that reserved the GPU's memory up front
 * for its own pool, or a latency-critical loop that cannot afford the
 * device-wide synchronization of cudaFree. Its scratch (about 17 KB: the
 * float32 inverse of V and two per-column vectors) is one fixed array in
 * device memory that every GPU loading libblco.so holds until the process
 * exits. Limits and behaviour:
 *   - R must be in 1..64; larger ranks return BLCO_ERR_ARG (the size limit
 *     of the fixed scratch; blco_cpals_update reports the same limit as
 *     BLCO_ERR_UNSUPPORTED).
 *   - The first call in a device's context looks up the array's device
 *     address (cudaGetSymbolAddress) and caches it with the context's id;
 *     make that first call before capturing any stream work. A context that
 *     is destroyed and recreated (cudaDeviceReset) may hold the array at
 *     another address: the next call sees the new context id and looks the
 *     address up again (again a first call, outside any capture).
 *   - Every call on a device uses the same scratch, which keeps the last
 *     call's contents (the call clears what must start at zero). Calls whose
 *     GPU work overlaps -- on different streams without ordering -- race on
 *     it; order them on one stream or with events.
 */
blco_status blco_cpals_update_noalloc(const double *const *grams, int N, int mode, int R, const float *M,
                                      int64_t I, float *A, double *lambda, double *G_out, int32_t *info,
                                      blco_stream stream);

/*
 * blco_cpals_fit: fit = 1 - ||X - Xhat|| / ||X|| of the model (lambda, A_1..A_N)
 * from ||X||^2 (host value), all N Grams, lambda, and the last mode's M and A:
 *   ||Xhat||^2 = lambda^T (Hadamard product of all Grams) lambda
 *   <X, Xhat>  = sum_r lambda_r sum_i M[i, r] A_last[i, r]
 * fit: 1 float64 (device).
 */
blco_status blco_cpals_fit(double normX2, const double *const *grams, int N, int R,
                           const double *lambda, const float *M_last, const float *A_last,
                           int64_t I_last, double *fit, blco_stream stream);

/* sum_j vals[j]^2 in float64 over the stored values (device result). */
blco_status blco_norm2(blco_handle h, double *out, blco_stream stream);

/*
 * Kernel timing (measurement support; no counterpart in the paper). While
 * enabled, the handle records a CUDA event pair on the launching stream
 * around each kernel it launches. blco_profile_read waits for the recorded
 * events and returns one entry per kernel kind ("zero", "mttkrp", "sum_copies", "cp_fwd",
 * "norm2"; "upload" for the batch copies of a streamed store) with the
 * number of launches and their summed duration, then
 * clears the record. count receives the number of entries written (at most
 * capacity). Enabling costs two event records per launch.
 */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;
} blco_profile_entry;

blco_status blco_profile_enable(blco_handle h, int enable);
blco_status blco_profile_read(blco_handle h, blco_profile_entry *entries, int capacity, int *count);

/*
 * Host-side fault injection, for testing callers' error paths (no
 * counterpart in the paper). Arms the k-th next event of `kind`, counted from
 * this call, to fail as a real failure of that kind would; k = 0 disarms.
 * Nothing faults on the GPU: the library reports the failure and cleans up.
 *   BLCO_FAULT_ALLOC  a device allocation of the library (store, queue
 *                     reservations, construction scratch) -> BLCO_ERR_OOM;
 *                     the call releases what it had allocated.
 *   BLCO_FAULT_COPY   a batch copy of a streamed store -> BLCO_ERR_CUDA; the
 *                     work already queued by the call is joined into the
 *                     caller's stream, and the handle stays usable.
 * The armed state is per process. Returns BLCO_ERR_ARG for an unknown kind
 * or k < 0.
 */
typedef enum { BLCO_FAULT_ALLOC = 1, BLCO_FAULT_COPY = 2 } blco_fault_kind;

blco_status blco_inject_fault(int kind, int64_t k);

#ifdef __cplusplus
}
#endif

#endif /* BLCO_H */
