// Dense helpers around the sparse kernels: output zeroing, float32 ->
// 16-bit factor conversion, and the FP64 pieces of CP-ALS (Algorithm 1):
// Grams, the Hadamard product of Grams, its Cholesky (or eigen
// pseudo-inverse) solve, column normalization and the fit.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <mutex>

#include "internal.h"

namespace blco {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

unsigned grid_cap(int64_t n, int threads) {
    int64_t g = (n + threads - 1) / threads;
    const int64_t cap = (int64_t)sm_count() * 8;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

__global__ void k_zero4(float4 *p, int64_t n4) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}
__global__ void k_zero1(float *p, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 0.f;
}

__global__ void k_to_bf16(const float *__restrict__ s, __nv_bfloat16 *__restrict__ d, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = __float2bfloat16_rn(s[i]);
}
__global__ void k_to_f16(const float *__restrict__ s, __half *__restrict__ d, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        d[i] = __float2half_rn(s[i]);
}

template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) { return v; }
template <>
__device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }
template <>
__device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }

// G = A^T A. Each thread owns a 4 x 4 block of G in the upper triangle
// (diagonal blocks included) and accumulates its 16 dot products over its
// CTA's rows with Ogita, Rump and Oishi's Dot2 (SIAM J. Sci. Comput. 26(6),
// 2005): TwoProduct by FMA gives each float32 product exactly as p + e, and
// TwoSum carries the rounding error of every addition, so each partial is a
// float32 pair as accurate as a sum in twice the float32 precision. The pair
// is added in float64 (hi + lo), the CTA's thread groups are summed in
// shared memory in float64, and CTAs meet in float64 atomics (both halves of
// an off-diagonal block). This keeps the FP64 pipe, which is a small fraction
// of the FP32 rate on this GPU, off the O(I R^2) part of the work.
constexpr int kGramRows = 32;  // rows staged in shared memory per step
constexpr int kGramThreads = 256;

struct GramShape {
    int R4;      // R rounded up to 4 (padding columns are zero)
    int B;       // 4 x 4 blocks per side
    int nblk;    // blocks in the upper triangle
    int groups;  // thread groups per CTA that split the rows (nblk < 256)
};

__host__ __device__ inline GramShape gram_shape(int R) {
    GramShape g;
    g.R4 = (R + 3) & ~3;
    g.B = g.R4 / 4;
    g.nblk = g.B * (g.B + 1) / 2;
    g.groups = g.nblk >= kGramThreads ? 1 : kGramThreads / g.nblk;
    return g;
}

__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

template <typename T>
__global__ void __launch_bounds__(kGramThreads) k_gram(const T *__restrict__ A, int64_t I, int R, int64_t rows_per_cta,
                                                       double *__restrict__ G) {
    extern __shared__ __align__(16) unsigned char smem[];
    const GramShape sh = gram_shape(R);
    float *tile = reinterpret_cast<float *>(smem);                       // kGramRows x R4
    double *red = reinterpret_cast<double *>(tile + kGramRows * sh.R4);  // groups x nblk x 16
    const int tid = threadIdx.x;
    int blk, grp;
    if (sh.groups > 1) {
        blk = tid % sh.nblk;
        grp = tid / sh.nblk;
    } else {
        blk = blockIdx.y * kGramThreads + tid;
        grp = 0;
    }
    const bool active = blk < sh.nblk && grp < sh.groups;
    int br = 0, rem = active ? blk : 0;  // upper-triangle block -> (br, bc)
    while (rem >= sh.B - br) {
        rem -= sh.B - br;
        ++br;
    }
    const int bc = br + rem;
    float hi[16], lo[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) hi[k] = lo[k] = 0.f;
    const int64_t r0 = (int64_t)blockIdx.x * rows_per_cta;
    const int64_t r1 = r0 + rows_per_cta < I ? r0 + rows_per_cta : I;
    for (int64_t b0 = r0; b0 < r1; b0 += kGramRows) {
        const int nr = (int)((r1 - b0) < kGramRows ? (r1 - b0) : kGramRows);
        __syncthreads();
        for (int i = tid; i < kGramRows * sh.R4; i += kGramThreads) {
            const int row = i / sh.R4, col = i % sh.R4;
            tile[i] = (row < nr && col < R) ? to_f<T>(A[(b0 + row) * R + col]) : 0.f;
        }
        __syncthreads();
        if (!active) continue;
        for (int i = grp; i < nr; i += sh.groups) {
            const float4 x = *reinterpret_cast<const float4 *>(tile + i * sh.R4 + br * 4);
            const float4 y = *reinterpret_cast<const float4 *>(tile + i * sh.R4 + bc * 4);
            const float xa[4] = {x.x, x.y, x.z, x.w}, ya[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    const float p = __fmul_rn(xa[u], ya[v]);
                    const float e = __fmaf_rn(xa[u], ya[v], -p);  // x*y == p + e exactly
                    float sum, err;
                    two_sum(hi[u * 4 + v], p, sum, err);
                    hi[u * 4 + v] = sum;
                    lo[u * 4 + v] = __fadd_rn(lo[u * 4 + v], __fadd_rn(err, e));
                }
        }
    }
    // sum the thread groups of this CTA in float64, then one atomic per
    // entry. Shared slots are indexed by the block's local index: with thread
    // groups the block itself, else the thread (blockIdx.y picks the range).
    const int nloc = sh.groups > 1 ? sh.nblk : kGramThreads;  // local blocks per group
    const int lbl = sh.groups > 1 ? blk : tid;
    if (active)
#pragma unroll
        for (int k = 0; k < 16; ++k) red[(grp * nloc + lbl) * 16 + k] = (double)hi[k] + (double)lo[k];
    __syncthreads();
    const int nact = sh.groups > 1 ? sh.nblk : min(kGramThreads, sh.nblk - (int)blockIdx.y * kGramThreads);
    for (int i = tid; i < nact * 16; i += kGramThreads) {
        const int lb = i / 16, k = i % 16;
        double v = 0.0;
        for (int g2 = 0; g2 < sh.groups; ++g2) v += red[(g2 * nloc + lb) * 16 + k];
        const int gb = sh.groups > 1 ? lb : (int)blockIdx.y * kGramThreads + lb;
        int rr = 0, rm = gb;
        while (rm >= sh.B - rr) {
            rm -= sh.B - rr;
            ++rr;
        }
        const int r = rr * 4 + k / 4, c = (rr + rm) * 4 + k % 4;
        if (r >= R || c >= R) continue;
        atomicAdd(&G[(size_t)r * R + c], v);
        if (rr != rr + rm) atomicAdd(&G[(size_t)c * R + r], v);
    }
}

__global__ void k_zero_d(double *p, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = 0.0;
}

struct GramPtrs {
    const double *g[MAXN];
};

// -------------------------------------------------------------------------
// one CTA: V = Hadamard of Grams (k != mode); W = V^{-1} by Cholesky, or the
// eigen pseudo-inverse (cyclic Jacobi) when V is not positive definite.
// Output W as float32 (the apply step) and info.
// -------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_solve_small(const GramPtrs gp, int N, int mode, int R,
                                                     float *__restrict__ Wf, int32_t *__restrict__ info) {
    extern __shared__ __align__(16) unsigned char smem[];
    double *V = reinterpret_cast<double *>(smem);  // R x R: V, then W (or Jacobi vectors)
    double *L = V + R * R;                           // R x R work
    __shared__ int ok;
    const int tid = threadIdx.x;
    for (int p = tid; p < R * R; p += blockDim.x) {
        double v = 1.0;
        for (int k = 0; k < N; ++k)
            if (k != mode) v *= gp.g[k][p];
        V[p] = v;
        L[p] = v;
    }
    __shared__ double pd_tol;
    if (tid == 0) {
        ok = 1;
        // smallest pivot accepted as positive: R * eps * max_i V_ii; at or
        // below it V is treated as not positive definite (numerically
        // singular or indefinite) and the pseudo-inverse is used
        double m = 0.0;
        for (int i = 0; i < R; ++i) m = fmax(m, V[i * R + i]);
        pd_tol = (double)R * 2.220446049250313e-16 * m;
    }
    __syncthreads();
    // Cholesky, right-looking, in L (lower triangle)
    for (int j = 0; j < R; ++j) {
        if (tid == 0) {
            const double d = L[j * R + j];
            if (!(d > pd_tol)) ok = 0;
            L[j * R + j] = d > 0.0 ? sqrt(d) : 1.0;
        }
        __syncthreads();
        if (!ok) break;
        const double djj = L[j * R + j];
        for (int i = j + 1 + tid; i < R; i += blockDim.x) L[i * R + j] /= djj;
        __syncthreads();
        for (int p = tid; p < (R - j - 1) * (R - j - 1); p += blockDim.x) {
            const int i = j + 1 + p / (R - j - 1), k = j + 1 + p % (R - j - 1);
            if (k <= i) L[i * R + k] -= L[i * R + j] * L[k * R + j];
        }
        __syncthreads();
    }
    if (ok) {
        // W = L^{-T} L^{-1}, one column per thread, in place in V[:, c]
        __syncthreads();
        for (int c = tid; c < R; c += blockDim.x) {
            for (int i = 0; i < R; ++i) {  // forward: L x = e_c
                double sum = (i == c) ? 1.0 : 0.0;
                for (int k = 0; k < i; ++k) sum -= L[i * R + k] * V[k * R + c];
                V[i * R + c] = sum / L[i * R + i];
            }
            for (int i = R - 1; i >= 0; --i) {  // back: L^T w = x
                double sum = V[i * R + c];
                for (int k = i + 1; k < R; ++k) sum -= L[k * R + i] * V[k * R + c];
                V[i * R + c] = sum / L[i * R + i];
            }
        }
        __syncthreads();
        for (int p = tid; p < R * R; p += blockDim.x) Wf[p] = (float)V[p];
        if (tid == 0) *info = 0;
        return;
    }
    // ---- eigen pseudo-inverse: cyclic Jacobi rotations on L := V, Q := I
    double *Q = V;
    for (int p = tid; p < R * R; p += blockDim.x) {
        L[p] = V[p];
        Q[p] = (p / R == p % R) ? 1.0 : 0.0;
    }
    __syncthreads();
    __shared__ double cs[128][2];
    __shared__ int pairs_p[64], pairs_q[64];
    __shared__ double off;
    const int Rp = (R + 1) & ~1;  // even count for round-robin pairing (a dummy index when R is odd)
    for (int sweep = 0; sweep < 30; ++sweep) {
        if (tid == 0) off = 0.0;
        __syncthreads();
        for (int p = tid; p < R * R; p += blockDim.x)
            if (p / R != p % R) atomicAdd(&off, L[p] * L[p]);
        __syncthreads();
        double diag = 0.0;
        for (int i = 0; i < R; ++i) diag += L[i * R + i] * L[i * R + i];
        if (off <= 1e-30 * diag || off == 0.0) break;
        for (int round = 0; round < Rp - 1; ++round) {
            // round-robin schedule: position 0 fixed, the rest rotate
            if (tid < Rp / 2) {
                const int a = tid == 0 ? 0 : 1 + (tid - 1 + round) % (Rp - 1);
                const int b = 1 + (Rp - 2 - tid + round) % (Rp - 1);
                pairs_p[tid] = a < b ? a : b;
                pairs_q[tid] = a < b ? b : a;
            }
            __syncthreads();
            if (tid < Rp / 2) {
                const int p = pairs_p[tid], q = pairs_q[tid];
                double c = 1.0, s = 0.0;
                if (q < R && p != q) {
                    const double apq = L[p * R + q];
                    if (apq != 0.0) {
                        const double theta = (L[q * R + q] - L[p * R + p]) / (2.0 * apq);
                        const double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                        c = 1.0 / sqrt(t * t + 1.0);
                        s = t * c;
                    }
                }
                cs[tid][0] = c;
                cs[tid][1] = s;
            }
            __syncthreads();
            // rows: L <- J^T L
            for (int w = tid; w < (Rp / 2) * R; w += blockDim.x) {
                const int pr = w / R, col = w % R;
                const int p = pairs_p[pr], q = pairs_q[pr];
                if (q < R && p != q) {
                    const double c = cs[pr][0], s = cs[pr][1];
                    const double lp = L[p * R + col], lq = L[q * R + col];
                    L[p * R + col] = c * lp - s * lq;
                    L[q * R + col] = s * lp + c * lq;
                }
            }
            __syncthreads();
            // columns: L <- L J, Q <- Q J
            for (int w = tid; w < (Rp / 2) * R; w += blockDim.x) {
                const int pr = w / R, row = w % R;
                const int p = pairs_p[pr], q = pairs_q[pr];
                if (q < R && p != q) {
                    const double c = cs[pr][0], s = cs[pr][1];
                    const double lp = L[row * R + p], lq = L[row * R + q];
                    L[row * R + p] = c * lp - s * lq;
                    L[row * R + q] = s * lp + c * lq;
                    const double qp = Q[row * R + p], qq = Q[row * R + q];
                    Q[row * R + p] = c * qp - s * qq;
                    Q[row * R + q] = s * qp + c * qq;
                }
            }
            __syncthreads();
        }
    }
    // W = Q diag(1/w with cutoff) Q^T
    __shared__ double wmax;
    if (tid == 0) {
        double m = 0.0;
        for (int i = 0; i < R; ++i) m = fmax(m, fabs(L[i * R + i]));
        wmax = m;
    }
    __syncthreads();
    const double cut = wmax * R * 2.220446049250313e-16;
    for (int p = tid; p < R * R; p += blockDim.x) {
        const int i = p / R, j = p % R;
        double s = 0.0;
        for (int k = 0; k < R; ++k) {
            const double w = L[k * R + k];
            if (fabs(w) > cut) s += Q[i * R + k] * Q[j * R + k] / w;
        }
        Wf[p] = (float)s;
    }
    if (tid == 0) *info = 1;
}

// A = M W (float32, W in shared memory), one warp per row.
__global__ void __launch_bounds__(256) k_apply(const float *__restrict__ M, int64_t I, int R,
                                               const float *__restrict__ Wg, float *__restrict__ A) {
    extern __shared__ __align__(16) unsigned char smem[];
    float *W = reinterpret_cast<float *>(smem);
    float *rowbuf = W + R * R;  // 8 warps x R
    for (int p = threadIdx.x; p < R * R; p += blockDim.x) W[p] = Wg[p];
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float *rb = rowbuf + w * R;
    for (int64_t i = (int64_t)blockIdx.x * 8 + w; i < I; i += (int64_t)gridDim.x * 8) {
        for (int k = lane; k < R; k += 32) rb[k] = M[i * R + k];
        __syncwarp();
        for (int cidx = lane; cidx < R; cidx += 32) {
            float s = 0.f;
            for (int k = 0; k < R; ++k) s = fmaf(rb[k], W[k * R + cidx], s);
            A[i * R + cidx] = s;
        }
        __syncwarp();
    }
}

// column sums of squares (float64) -> colsq[R] via atomics
__global__ void __launch_bounds__(256) k_colsq(const float *__restrict__ A, int64_t I, int R, double *__restrict__ colsq) {
    // thread handles column c = threadIdx.x % R for rows strided
    const int lanes = 256 / R * R;  // threads used
    if (threadIdx.x >= lanes) return;
    const int c = threadIdx.x % R;
    const int sub = threadIdx.x / R, nsub = 256 / R;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * nsub + sub; i < I; i += (int64_t)gridDim.x * nsub) {
        const double v = A[i * R + c];
        s += v * v;
    }
    atomicAdd(&colsq[c], s);
}

__global__ void k_sqrt_lambda(const double *__restrict__ colsq, int R, double *__restrict__ lambda,
                              float *__restrict__ inv) {
    const int c = threadIdx.x;
    if (c < R) {
        const double l = sqrt(colsq[c]);
        lambda[c] = l;
        inv[c] = l > 0.0 ? (float)(1.0 / l) : 1.f;
    }
}

__global__ void k_scale_cols(float *__restrict__ A, int64_t I, int R, const float *__restrict__ inv) {
    const int64_t n = I * R;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += (int64_t)gridDim.x * blockDim.x)
        A[p] *= inv[p % R];
}

// <M, A> per column (float64) -> acc[R]
__global__ void __launch_bounds__(256) k_coldot(const float *__restrict__ M, const float *__restrict__ A, int64_t I,
                                                int R, double *__restrict__ acc) {
    const int lanes = 256 / R * R;
    if (threadIdx.x >= lanes) return;
    const int c = threadIdx.x % R;
    const int sub = threadIdx.x / R, nsub = 256 / R;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * nsub + sub; i < I; i += (int64_t)gridDim.x * nsub)
        s += (double)M[i * R + c] * (double)A[i * R + c];
    atomicAdd(&acc[c], s);
}

__global__ void k_fit_final(double normX2, const GramPtrs gp, int N, int R, const double *__restrict__ lambda,
                            const double *__restrict__ dots, double *__restrict__ fit) {
    __shared__ double part[256];
    double s = 0.0;
    for (int p = threadIdx.x; p < R * R; p += blockDim.x) {
        double v = 1.0;
        for (int k = 0; k < N; ++k) v *= gp.g[k][p];
        s += lambda[p / R] * v * lambda[p % R];
    }
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double xh2 = 0.0;
        for (int i = 0; i < (int)blockDim.x; ++i) xh2 += part[i];
        double inner = 0.0;
        for (int c = 0; c < R; ++c) inner += lambda[c] * dots[c];
        double r2 = normX2 + xh2 - 2.0 * inner;
        if (r2 < 0.0) r2 = 0.0;
        *fit = 1.0 - sqrt(r2) / sqrt(normX2);
    }
}

__global__ void __launch_bounds__(256) k_norm2(const float *__restrict__ v, int64_t n, double *__restrict__ out) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = v[i];
        s += x * x;
    }
    for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// out = sum of the private output copies (n floats each, n % 4 == 0,
// 16-byte aligned), one float4 per thread and step; copies summed in order.
__global__ void k_sum_copies(const float4 *__restrict__ copies, int ncopies, int64_t n4, float4 *__restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += (int64_t)gridDim.x * blockDim.x) {
        float4 a = copies[i];
        for (int c = 1; c < ncopies; ++c) {
            const float4 b = copies[(int64_t)c * n4 + i];
            a.x += b.x;
            a.y += b.y;
            a.z += b.z;
            a.w += b.w;
        }
        out[i] = a;
    }
}

}  // namespace

cudaError_t launch_sum_copies(const float *copies, int ncopies, int64_t n, float *out, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int64_t n4 = n / 4;
    k_sum_copies<<<grid_cap(n4, 256), 256, 0, s>>>(reinterpret_cast<const float4 *>(copies), ncopies, n4,
                                                    reinterpret_cast<float4 *>(out));
    return cudaGetLastError();
}

cudaError_t launch_zero(float *p, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if ((reinterpret_cast<uintptr_t>(p) & 15) == 0 && (n & 3) == 0) {
        k_zero4<<<grid_cap(n / 4, 256), 256, 0, s>>>(reinterpret_cast<float4 *>(p), n / 4);
    } else {
        k_zero1<<<grid_cap(n, 256), 256, 0, s>>>(p, n);
    }
    return cudaGetLastError();
}

cudaError_t launch_convert(const float *src, void *dst, blco_dtype dt, int64_t n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (dt == BLCO_BF16)
        k_to_bf16<<<grid_cap(n, 256), 256, 0, s>>>(src, static_cast<__nv_bfloat16 *>(dst), n);
    else if (dt == BLCO_F16)
        k_to_f16<<<grid_cap(n, 256), 256, 0, s>>>(src, static_cast<__half *>(dst), n);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_gram(const void *A, blco_dtype fdt, int64_t I, int R, double *G, cudaStream_t s) {
    k_zero_d<<<1, 256, 0, s>>>(G, R * R);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || I <= 0) return e;
    const GramShape sh = gram_shape(R);
    const int ny = sh.groups > 1 ? 1 : (sh.nblk + kGramThreads - 1) / kGramThreads;
    // three CTAs per SM in total (the register limit at 79 registers), each
    // over a contiguous range of rows
    const int64_t ctas_max = std::max<int64_t>(1, (int64_t)sm_count() * 3 / ny);
    int64_t rows = (I + ctas_max - 1) / ctas_max;
    rows = std::max<int64_t>(kGramRows, (rows + kGramRows - 1) / kGramRows * kGramRows);
    const int64_t ctas = (I + rows - 1) / rows;
    const size_t red_entries = (size_t)(sh.groups > 1 ? sh.groups * sh.nblk : kGramThreads) * 16;
    const size_t shm = sizeof(float) * kGramRows * sh.R4 + sizeof(double) * red_entries;
    const dim3 grid((unsigned)ctas, (unsigned)ny);
    switch (fdt) {
        case BLCO_F32:
            e = cudaFuncSetAttribute(k_gram<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
            if (e == cudaSuccess)
                k_gram<float><<<grid, kGramThreads, shm, s>>>(static_cast<const float *>(A), I, R, rows, G);
            break;
        case BLCO_BF16:
            e = cudaFuncSetAttribute(k_gram<__nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
            if (e == cudaSuccess)
                k_gram<__nv_bfloat16><<<grid, kGramThreads, shm, s>>>(static_cast<const __nv_bfloat16 *>(A), I, R,
                                                                        rows, G);
            break;
        case BLCO_F16:
            e = cudaFuncSetAttribute(k_gram<__half>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
            if (e == cudaSuccess)
                k_gram<__half><<<grid, kGramThreads, shm, s>>>(static_cast<const __half *>(A), I, R, rows, G);
            break;
    }
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

cudaError_t launch_cpals_update(const double *const *grams, int N, int mode, int R, const float *M, int64_t I,
                                float *A, double *lambda, double *G_out, int32_t *info, cudaStream_t s) {
    GramPtrs gp;
    for (int k = 0; k < MAXN; ++k) gp.g[k] = k < N ? grams[k] : nullptr;
    float *Wf = nullptr;
    double *colsq = nullptr;
    float *inv = nullptr;
    cudaError_t e = cudaMallocAsync(&Wf, sizeof(float) * R * R, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&colsq, sizeof(double) * R, s);
    if (e == cudaSuccess) e = cudaMallocAsync(&inv, sizeof(float) * R, s);
    if (e == cudaSuccess) {
        const size_t shm = sizeof(double) * 2 * R * R;
        e = cudaFuncSetAttribute(k_solve_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        if (e == cudaSuccess) {
            k_solve_small<<<1, 256, shm, s>>>(gp, N, mode, R, Wf, info);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess && I > 0) {
        const size_t shm = sizeof(float) * (R * R + 8 * R);
        e = cudaFuncSetAttribute(k_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        if (e == cudaSuccess) {
            k_apply<<<grid_cap(I, 8), 256, shm, s>>>(M, I, R, Wf, A);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        k_zero_d<<<1, 256, 0, s>>>(colsq, R);
        if (I > 0) k_colsq<<<grid_cap(I, 256 / R), 256, 0, s>>>(A, I, R, colsq);
        k_sqrt_lambda<<<1, 128, 0, s>>>(colsq, R, lambda, inv);
        if (I > 0) k_scale_cols<<<grid_cap(I * R, 256), 256, 0, s>>>(A, I, R, inv);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && G_out) e = launch_gram(A, BLCO_F32, I, R, G_out, s);
    if (Wf) cudaFreeAsync(Wf, s);
    if (colsq) cudaFreeAsync(colsq, s);
    if (inv) cudaFreeAsync(inv, s);
    return e;
}

cudaError_t launch_cpals_fit(double normX2, const double *const *grams, int N, int R, const double *lambda,
                             const float *M, const float *A, int64_t I, double *fit, cudaStream_t s) {
    GramPtrs gp;
    for (int k = 0; k < MAXN; ++k) gp.g[k] = k < N ? grams[k] : nullptr;
    double *dots = nullptr;
    cudaError_t e = cudaMallocAsync(&dots, sizeof(double) * R, s);
    if (e != cudaSuccess) return e;
    k_zero_d<<<1, 128, 0, s>>>(dots, R);
    if (I > 0) k_coldot<<<grid_cap(I, 256 / R), 256, 0, s>>>(M, A, I, R, dots);
    k_fit_final<<<1, 256, 0, s>>>(normX2, gp, N, R, lambda, dots, fit);
    e = cudaGetLastError();
    cudaFreeAsync(dots, s);
    return e;
}

cudaError_t launch_norm2(const float *v, int64_t n, double *out, cudaStream_t s) {
    k_zero_d<<<1, 32, 0, s>>>(out, 1);
    if (n > 0) k_norm2<<<grid_cap(n, 256), 256, 0, s>>>(v, n, out);
    return cudaGetLastError();
}

cudaError_t launch_norm2_acc(const float *v, int64_t n, double *out, cudaStream_t s) {
    if (n > 0) k_norm2<<<grid_cap(n, 256), 256, 0, s>>>(v, n, out);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// CP-ALS update without allocation.
//
// Some callers cannot let a library allocate device memory during a call:
// a process that reserved the GPU's memory up front for its own pool (a
// cudaMalloc would fail or escape its accounting), or a latency-critical loop
// where the device-wide synchronization of cudaFree is not acceptable. For
// them the update's scratch (the float32 inverse of V, the column sums of
// squares and their reciprocals) lives in one file-scope device array that
// every GPU which loads the library holds until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxRank = 64;
constexpr size_t kNoAllocWfBytes = sizeof(float) * kNoAllocMaxRank * kNoAllocMaxRank;
constexpr size_t kNoAllocColsqOff = (kNoAllocWfBytes + 255) & ~size_t(255);
constexpr size_t kNoAllocInvOff = kNoAllocColsqOff + ((sizeof(double) * kNoAllocMaxRank + 255) & ~size_t(255));
constexpr size_t kNoAllocScratchBytes = kNoAllocInvOff + sizeof(float) * kNoAllocMaxRank;

// Shared by every call on a device; holds the previous call's contents.
static __device__ __align__(256) unsigned char g_update_scratch[kNoAllocScratchBytes];

// The array's device address is looked up once per device and context
// (cudaGetSymbolAddress: the host-side name of the array is not a device
// address) and cached with the id of the context it belongs to. A context
// that is destroyed and recreated (cudaDeviceReset) reloads the module,
// possibly at another address; its new id makes the next call look the
// address up again instead of using a stale one.
typedef int (*CtxGetCurrentFn)(void **);
typedef int (*CtxGetIdFn)(void *, unsigned long long *);

struct ScratchCache {
    unsigned long long ctx_id = 0;  // 0: nothing cached
    void *addr = nullptr;
};

std::mutex g_scratch_mutex;
ScratchCache g_scratch[64];
CtxGetCurrentFn g_ctx_current = nullptr;
CtxGetIdFn g_ctx_id = nullptr;
bool g_driver_looked_up = false;

// Id of the calling thread's current context, 0 if unknown.
unsigned long long current_ctx_id() {
    if (!g_driver_looked_up) {
        g_driver_looked_up = true;
        void *f = nullptr, *g = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &g, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
            q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
            g_ctx_current = reinterpret_cast<CtxGetCurrentFn>(f);
            g_ctx_id = reinterpret_cast<CtxGetIdFn>(g);
        }
        cudaGetLastError();
    }
    if (!g_ctx_current || !g_ctx_id) return 0;
    void *ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_current(&ctx) != 0 || !ctx || g_ctx_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of g_update_scratch in the current device's context.
cudaError_t update_scratch(unsigned char **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    const unsigned long long id = current_ctx_id();
    ScratchCache &c = g_scratch[dev];
    if (id == 0 || c.ctx_id != id) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_update_scratch);  // also makes the primary context current
        if (e != cudaSuccess) return e;
        c.addr = p;
        c.ctx_id = current_ctx_id();  // 0 (no driver entry points): look up again on every call
    }
    *out = static_cast<unsigned char *>(c.addr);
    return cudaSuccess;
}

}  // namespace

int cpals_update_noalloc_max_rank() { return kNoAllocMaxRank; }

cudaError_t launch_cpals_update_noalloc(const double *const *grams, int N, int mode, int R, const float *M,
                                        int64_t I, float *A, double *lambda, double *G_out, int32_t *info,
                                        cudaStream_t s) {
    if (R < 1 || R > kNoAllocMaxRank) return cudaErrorInvalidValue;
    unsigned char *base = nullptr;
    cudaError_t e = update_scratch(&base);
    if (e != cudaSuccess) return e;
    float *Wf = reinterpret_cast<float *>(base);
    double *colsq = reinterpret_cast<double *>(base + kNoAllocColsqOff);
    float *inv = reinterpret_cast<float *>(base + kNoAllocInvOff);
    GramPtrs gp;
    for (int k = 0; k < MAXN; ++k) gp.g[k] = k < N ? grams[k] : nullptr;
    const size_t shm_solve = sizeof(double) * 2 * R * R;
    e = cudaFuncSetAttribute(k_solve_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_solve);
    if (e != cudaSuccess) return e;
    k_solve_small<<<1, 256, shm_solve, s>>>(gp, N, mode, R, Wf, info);
    e = cudaGetLastError();
    if (e == cudaSuccess && I > 0) {
        const size_t shm = sizeof(float) * (R * R + 8 * R);
        e = cudaFuncSetAttribute(k_apply, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        if (e == cudaSuccess) {
            k_apply<<<grid_cap(I, 8), 256, shm, s>>>(M, I, R, Wf, A);
            e = cudaGetLastError();
        }
    }
    if (e == cudaSuccess) {
        k_zero_d<<<1, 256, 0, s>>>(colsq, R);  // the shared scratch keeps the last call's sums
        if (I > 0) k_colsq<<<grid_cap(I, 256 / R), 256, 0, s>>>(A, I, R, colsq);
        k_sqrt_lambda<<<1, 128, 0, s>>>(colsq, R, lambda, inv);
        if (I > 0) k_scale_cols<<<grid_cap(I * R, 256), 256, 0, s>>>(A, I, R, inv);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess && G_out) e = launch_gram(A, BLCO_F32, I, R, G_out, s);
    return e;
}

}  // namespace blco
