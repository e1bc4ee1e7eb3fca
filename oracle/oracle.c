/*
 * FP64 CPU oracle for the BLCO sparse-MTTKRP path -- TEST INFRASTRUCTURE.
 *
 * Only the test suite, the package's smoke check and the benchmark's CPU
 * baseline load this library. The product path (libblco.so and its Python
 * binding) never links, loads or calls it, and it shares no code, header,
 * table or helper with the CUDA sources.
 *
 * Everything here is the plain definition, written as loops in the order the
 * paper states it, in double precision, single-threaded (orc_mttkrp_rows may
 * spread independent chunks and rows over OpenMP threads; every sum is still
 * the same additions in the same order):
 *
 *   orc_alto_layout   Section 4.1, Fig. 6a: the ALTO bit order of a linear
 *                     index (one bit per mode per level, round robin from the
 *                     least significant bit, lower mode numbers first).
 *   orc_alto_keys     the linear index of each coordinate under that layout,
 *                     as a (hi, lo) pair of 64-bit words.
 *   orc_build_store   Section 4.2 + Fig. 6b: stable sort by linear index,
 *                     block key = the bits above the encoding line, blocks
 *                     split at the nonzero cap, in-block key re-encoded as
 *                     concatenated per-mode fields (mode 1 lowest).
 *   orc_check_store   the same definition checked against a given store in
 *                     one pass (for stores too large to rebuild here).
 *   orc_check_store_at  the same checks at chosen store positions only (for
 *                     stores too large for a full pass), plus
 *   orc_is_permutation  whether a store's input positions are a permutation.
 *   orc_mttkrp        Eq. 1 evaluated per nonzero as in Fig. 3: fetch rows,
 *                     Hadamard product, scale by the value, accumulate into
 *                     row i_n; also S = sum of |terms| per output entry.
 *   orc_mttkrp_rows   the same, for a chosen subset of output rows.
 *   orc_cp_model      the CP model (Section 2.2, Fig. 2) at each nonzero:
 *                     xhat = sum_r prod_n A_n[i_n, r].
 *   orc_bf16_rne      IEEE binary32 -> bfloat16 rounding, nearest-even.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MAXN 16

/* b_n = ceil(log2 I_n), with b_n = 0 for a mode of length 1. */
static int orc_bits_of(int64_t dim) {
    int b = 0;
    while (b < 63 && ((int64_t)1 << b) < dim) b++;
    return b;
}

/*
 * ALTO layout. Key bit k (from the least significant bit) holds bit
 * key_level[k] of the index of mode key_mode[k]. Levels are visited from 0
 * upwards; within a level, every mode that still has bits contributes one,
 * lower mode numbers at lower positions. Returns B = sum_n b_n, or -1.
 */
int orc_alto_layout(int N, const int64_t *dims, int *bits, int *key_mode, int *key_level) {
    if (N < 1 || N > ORC_MAXN) return -1;
    int maxb = 0, B = 0;
    for (int n = 0; n < N; ++n) {
        if (dims[n] < 1) return -1;
        bits[n] = orc_bits_of(dims[n]);
        if (bits[n] > maxb) maxb = bits[n];
    }
    for (int l = 0; l < maxb; ++l)
        for (int n = 0; n < N; ++n)
            if (bits[n] > l) {
                if (B >= 128) return -1;
                key_mode[B] = n;
                key_level[B] = l;
                B++;
            }
    return B;
}

static void orc_key_of(int N, const uint32_t *c, int B, const int *km, const int *kl,
                       uint64_t *hi, uint64_t *lo) {
    uint64_t h = 0, l = 0;
    (void)N;
    for (int k = 0; k < B; ++k) {
        uint64_t bit = (uint64_t)((c[km[k]] >> kl[k]) & 1u);
        if (k < 64)
            l |= bit << k;
        else
            h |= bit << (k - 64);
    }
    *hi = h;
    *lo = l;
}

/* Returns 0, or -1 for a bad shape, or 1 + j for the first out-of-range row j. */
int64_t orc_alto_keys(int64_t nnz, int N, const uint32_t *coords, const int64_t *dims,
                      uint64_t *hi, uint64_t *lo) {
    int bits[ORC_MAXN], km[128], kl[128];
    int B = orc_alto_layout(N, dims, bits, km, kl);
    if (B < 0) return -1;
    for (int64_t j = 0; j < nnz; ++j) {
        const uint32_t *c = coords + j * N;
        for (int n = 0; n < N; ++n)
            if ((int64_t)c[n] >= dims[n]) return 1 + j;
        orc_key_of(N, c, B, km, kl, &hi[j], &lo[j]);
    }
    return 0;
}

/*
 * Block bits per mode: the top (B - line_bits) bits of the linear index are
 * the block key (Section 4.2). Because higher key positions hold higher
 * levels, the block bits of mode n are its k_n most significant bits; the
 * in-block field of mode n is its low w_n = b_n - k_n bits.
 */
static int orc_fields(int N, const int64_t *dims, int line_bits, int *bits, int *kbits,
                      int *width, int *shift, int *km, int *kl) {
    int B = orc_alto_layout(N, dims, bits, km, kl);
    if (B < 0) return -1;
    for (int n = 0; n < N; ++n) kbits[n] = 0;
    for (int k = line_bits; k < B; ++k) kbits[km[k]]++;
    int off = 0;
    for (int n = 0; n < N; ++n) {
        width[n] = bits[n] - kbits[n];
        shift[n] = off;
        off += width[n];
    }
    return B;
}

typedef struct {
    uint64_t hi, lo;
    int64_t pos;
} orc_rec;

static int orc_rec_cmp(const void *a, const void *b) {
    const orc_rec *x = (const orc_rec *)a, *y = (const orc_rec *)b;
    if (x->hi != y->hi) return x->hi < y->hi ? -1 : 1;
    if (x->lo != y->lo) return x->lo < y->lo ? -1 : 1;
    if (x->pos != y->pos) return x->pos < y->pos ? -1 : 1;
    return 0;
}

/* The block key of a linear index: the key shifted right by line_bits. */
static void orc_block_key(uint64_t hi, uint64_t lo, int line_bits, uint64_t *bh, uint64_t *bl) {
    if (line_bits >= 128) {
        *bh = 0;
        *bl = 0;
    } else if (line_bits >= 64) {
        *bh = 0;
        *bl = hi >> (line_bits - 64);
    } else if (line_bits == 0) {
        *bh = hi;
        *bl = lo;
    } else {
        *bl = (lo >> line_bits) | (hi << (64 - line_bits));
        *bh = hi >> line_bits;
    }
}

/*
 * Full reference build. Outputs (caller-allocated):
 *   skeys[nnz]  in-block keys, store order
 *   svals[nnz]  values, store order
 *   sperm[nnz]  input position of each store entry
 *   bstart[*nblocks + 1], bhigh[*nblocks * N]  (block table; capacity cap_blocks)
 * Blocks: runs of equal block key in sorted order; a run of c > max_nnz
 * entries is cut into pieces of ceil(c / ceil(c / max_nnz)) entries (the last
 * piece holds the rest). bhigh[b*N+n] = i_n >> w_n for every entry of block b.
 * Returns 0, -1 (bad arguments), -2 (block capacity) or 1 + j (coordinate j
 * out of range).
 */
int64_t orc_build_store(int64_t nnz, int N, const uint32_t *coords, const float *vals,
                        const int64_t *dims, int line_bits, int64_t max_nnz, uint64_t *skeys,
                        float *svals, int64_t *sperm, int64_t cap_blocks, int64_t *nblocks,
                        int64_t *bstart, uint32_t *bhigh) {
    int bits[ORC_MAXN], kbits[ORC_MAXN], width[ORC_MAXN], shift[ORC_MAXN], km[128], kl[128];
    if (line_bits < 1 || line_bits > 64 || max_nnz < 1) return -1;
    int B = orc_fields(N, dims, line_bits, bits, kbits, width, shift, km, kl);
    if (B < 0) return -1;
    orc_rec *rec = (orc_rec *)malloc(sizeof(orc_rec) * (size_t)(nnz > 0 ? nnz : 1));
    if (!rec) return -1;
    for (int64_t j = 0; j < nnz; ++j) {
        const uint32_t *c = coords + j * N;
        for (int n = 0; n < N; ++n)
            if ((int64_t)c[n] >= dims[n]) {
                free(rec);
                return 1 + j;
            }
        orc_key_of(N, c, B, km, kl, &rec[j].hi, &rec[j].lo);
        rec[j].pos = j;
    }
    qsort(rec, (size_t)nnz, sizeof(orc_rec), orc_rec_cmp);
    int64_t nb = 0;
    int64_t j = 0;
    while (j < nnz) {
        uint64_t bh0, bl0;
        orc_block_key(rec[j].hi, rec[j].lo, line_bits, &bh0, &bl0);
        int64_t e = j + 1;
        while (e < nnz) {
            uint64_t bh, bl;
            orc_block_key(rec[e].hi, rec[e].lo, line_bits, &bh, &bl);
            if (bh != bh0 || bl != bl0) break;
            e++;
        }
        int64_t cnt = e - j;
        int64_t pieces = (cnt + max_nnz - 1) / max_nnz;
        int64_t piece = (cnt + pieces - 1) / pieces;
        for (int64_t s = j; s < e; s += piece) {
            if (nb >= cap_blocks) {
                free(rec);
                return -2;
            }
            bstart[nb] = s;
            const uint32_t *c = coords + rec[s].pos * N;
            for (int n = 0; n < N; ++n) bhigh[nb * N + n] = (uint32_t)((uint64_t)c[n] >> width[n]);
            nb++;
        }
        j = e;
    }
    bstart[nb] = nnz;
    *nblocks = nb;
    for (int64_t s = 0; s < nnz; ++s) {
        const uint32_t *c = coords + rec[s].pos * N;
        uint64_t key = 0;
        for (int n = 0; n < N; ++n) {
            uint64_t low = width[n] >= 64 ? (uint64_t)c[n] : ((uint64_t)c[n] & ((1ull << width[n]) - 1));
            key |= low << shift[n];
        }
        skeys[s] = key;
        svals[s] = vals[rec[s].pos];
        sperm[s] = rec[s].pos;
    }
    free(rec);
    return 0;
}

/*
 * One-pass check that (skeys, svals, sperm, bstart, bhigh) is exactly the
 * store orc_build_store defines for (coords, vals). The sort order is checked
 * as: sperm is a permutation and (linear index, input position) strictly
 * increases along the store, which admits exactly one order. Returns 0 if
 * equal, else a code: 1 + s for the first bad store position s, or
 * -1 (arguments), -3 (sperm not a permutation), -4 (block table).
 */
int64_t orc_check_store(int64_t nnz, int N, const uint32_t *coords, const float *vals,
                        const int64_t *dims, int line_bits, int64_t max_nnz,
                        const uint64_t *skeys, const float *svals, const int64_t *sperm,
                        int64_t nblocks, const int64_t *bstart, const uint32_t *bhigh) {
    int bits[ORC_MAXN], kbits[ORC_MAXN], width[ORC_MAXN], shift[ORC_MAXN], km[128], kl[128];
    if (line_bits < 1 || line_bits > 64 || max_nnz < 1) return -1;
    int B = orc_fields(N, dims, line_bits, bits, kbits, width, shift, km, kl);
    if (B < 0) return -1;
    unsigned char *seen = (unsigned char *)calloc((size_t)(nnz > 0 ? nnz : 1), 1);
    if (!seen) return -1;
    for (int64_t s = 0; s < nnz; ++s) {
        int64_t p = sperm[s];
        if (p < 0 || p >= nnz || seen[p]) {
            free(seen);
            return -3;
        }
        seen[p] = 1;
    }
    free(seen);
    /* expected block starts, rebuilt from the (verified) order */
    int64_t b = 0;
    uint64_t phi = 0, plo = 0, pbh = 0, pbl = 0;
    int64_t run_start = 0, run_len = 0, piece = 0;
    for (int64_t s = 0; s < nnz; ++s) {
        const uint32_t *c = coords + sperm[s] * N;
        for (int n = 0; n < N; ++n)
            if ((int64_t)c[n] >= dims[n]) return 1 + s;
        uint64_t hi, lo, bh, bl;
        orc_key_of(N, c, B, km, kl, &hi, &lo);
        if (s > 0) {
            int less = (phi < hi) || (phi == hi && plo < lo) ||
                       (phi == hi && plo == lo && sperm[s - 1] < sperm[s]);
            if (!less) return 1 + s;
        }
        phi = hi;
        plo = lo;
        uint64_t key = 0;
        for (int n = 0; n < N; ++n) {
            uint64_t low = width[n] >= 64 ? (uint64_t)c[n] : ((uint64_t)c[n] & ((1ull << width[n]) - 1));
            key |= low << shift[n];
        }
        if (skeys[s] != key) return 1 + s;
        if (memcmp(&svals[s], &vals[sperm[s]], sizeof(float)) != 0) return 1 + s;
        orc_block_key(hi, lo, line_bits, &bh, &bl);
        int new_run = (s == 0) || bh != pbh || bl != pbl;
        if (new_run) {
            run_start = s;
            run_len = 1;
            int64_t e = s + 1;
            /* length of this run of equal block keys */
            while (e < nnz) {
                uint64_t h2, l2, bh2, bl2;
                orc_key_of(N, coords + sperm[e] * N, B, km, kl, &h2, &l2);
                orc_block_key(h2, l2, line_bits, &bh2, &bl2);
                if (bh2 != bh || bl2 != bl) break;
                e++;
            }
            run_len = e - s;
            int64_t pieces = (run_len + max_nnz - 1) / max_nnz;
            piece = (run_len + pieces - 1) / pieces;
        }
        pbh = bh;
        pbl = bl;
        if ((s - run_start) % piece == 0) {
            if (b >= nblocks || bstart[b] != s) return -4;
            for (int n = 0; n < N; ++n)
                if (bhigh[b * N + n] != (uint32_t)((uint64_t)c[n] >> width[n])) return -4;
            b++;
        }
    }
    if (b != nblocks || bstart[nblocks] != nnz) return -4;
    return 0;
}

/* 1 if p[0..n) is a permutation of 0..n-1, else 0. */
int orc_is_permutation(int64_t n, const int64_t *p) {
    unsigned char *seen = (unsigned char *)calloc((size_t)(n / 8 + 1), 1);
    if (!seen) return -1;
    int ok = 1;
    for (int64_t i = 0; i < n && ok; ++i) {
        int64_t v = p[i];
        if (v < 0 || v >= n || (seen[v >> 3] >> (v & 7)) & 1) ok = 0;
        else seen[v >> 3] |= (unsigned char)(1u << (v & 7));
    }
    free(seen);
    return ok;
}

/*
 * The checks of orc_check_store at the store positions pos[0..npos): the
 * entry is the re-encoded coordinate of its input row with that row's value;
 * (linear index, input position) increases from the entry to the next one;
 * the entry's block is the one bstart places it in, its high bits match, the
 * block holds one block key from its first to its last entry, and no block is
 * longer than the cap. Returns 0, or 1 + i for the first failing sample i, or
 * -1 for bad arguments.
 */
int64_t orc_check_store_at(int64_t nnz, int N, const uint32_t *coords, const float *vals,
                           const int64_t *dims, int line_bits, int64_t max_nnz,
                           const uint64_t *skeys, const float *svals, const int64_t *sperm,
                           int64_t nblocks, const int64_t *bstart, const uint32_t *bhigh,
                           int64_t npos, const int64_t *pos) {
    int bits[ORC_MAXN], kbits[ORC_MAXN], width[ORC_MAXN], shift[ORC_MAXN], km[128], kl[128];
    if (line_bits < 1 || line_bits > 64 || max_nnz < 1) return -1;
    int B = orc_fields(N, dims, line_bits, bits, kbits, width, shift, km, kl);
    if (B < 0) return -1;
    if (nblocks < 1 || bstart[0] != 0 || bstart[nblocks] != nnz) return -1;
    for (int64_t i = 0; i < npos; ++i) {
        const int64_t s = pos[i];
        if (s < 0 || s >= nnz) return 1 + i;
        const int64_t p = sperm[s];
        if (p < 0 || p >= nnz) return 1 + i;
        const uint32_t *c = coords + p * N;
        for (int n = 0; n < N; ++n)
            if ((int64_t)c[n] >= dims[n]) return 1 + i;
        uint64_t key = 0;
        for (int n = 0; n < N; ++n) {
            uint64_t low = width[n] >= 64 ? (uint64_t)c[n] : ((uint64_t)c[n] & ((1ull << width[n]) - 1));
            key |= low << shift[n];
        }
        if (skeys[s] != key) return 1 + i;
        if (memcmp(&svals[s], &vals[p], sizeof(float)) != 0) return 1 + i;
        uint64_t hi, lo;
        orc_key_of(N, c, B, km, kl, &hi, &lo);
        if (s + 1 < nnz) {
            uint64_t h2, l2;
            const uint32_t *c2 = coords + sperm[s + 1] * N;
            orc_key_of(N, c2, B, km, kl, &h2, &l2);
            int less = (hi < h2) || (hi == h2 && lo < l2) || (hi == h2 && lo == l2 && p < sperm[s + 1]);
            if (!less) return 1 + i;
        }
        /* block of s: the last b with bstart[b] <= s */
        int64_t a = 0, z = nblocks - 1;
        while (a < z) {
            int64_t m = (a + z + 1) / 2;
            if (bstart[m] <= s) a = m;
            else z = m - 1;
        }
        const int64_t b = a;
        if (bstart[b + 1] - bstart[b] > max_nnz || bstart[b + 1] <= bstart[b]) return 1 + i;
        for (int n = 0; n < N; ++n)
            if (bhigh[b * N + n] != (uint32_t)((uint64_t)c[n] >> width[n])) return 1 + i;
        uint64_t bh, bl, fh, fl, eh, el, h3, l3;
        orc_block_key(hi, lo, line_bits, &bh, &bl);
        orc_key_of(N, coords + sperm[bstart[b]] * N, B, km, kl, &h3, &l3);
        orc_block_key(h3, l3, line_bits, &fh, &fl);
        orc_key_of(N, coords + sperm[bstart[b + 1] - 1] * N, B, km, kl, &h3, &l3);
        orc_block_key(h3, l3, line_bits, &eh, &el);
        if (bh != fh || bl != fl || bh != eh || bl != el) return 1 + i;
    }
    return 0;
}

/*
 * Mode-`mode` MTTKRP (Eq. 1), per nonzero as in Fig. 3:
 *   M[i_n, r] += x * prod_{k != n} A_k[i_k, r]
 * and S[i_n, r] += |x * prod_{k != n} A_k[i_k, r]|, in input order, FP64.
 * factors[k] is I_k x R row-major (factors[mode] is not read).
 */
void orc_mttkrp(int64_t nnz, int N, const uint32_t *coords, const double *vals,
                const int64_t *dims, int R, const double *const *factors, int mode, double *M,
                double *S) {
    memset(M, 0, sizeof(double) * (size_t)dims[mode] * (size_t)R);
    if (S) memset(S, 0, sizeof(double) * (size_t)dims[mode] * (size_t)R);
    for (int64_t j = 0; j < nnz; ++j) {
        const uint32_t *c = coords + j * N;
        double *m = M + (int64_t)c[mode] * R;
        double *sa = S ? S + (int64_t)c[mode] * R : 0;
        for (int r = 0; r < R; ++r) {
            double t = vals[j];
            for (int k = 0; k < N; ++k)
                if (k != mode) t *= factors[k][(int64_t)c[k] * R + r];
            m[r] += t;
            if (sa) sa[r] += fabs(t);
        }
    }
}

/*
 * orc_mttkrp restricted to the output rows rows[0..nsel) (sorted ascending,
 * distinct): row rows[k] goes to Msel/Ssel row k (nsel x R, zeroed here).
 * Two passes over the nonzeros list, per chosen row and in input order, the
 * nonzeros that hit it (a bitmap filters, a binary search finds the row);
 * then each chosen row sums its own list in input order. Chunks of the
 * nonzeros, and the rows, are independent, so they may be handled by several
 * threads (OpenMP, when compiled with it): every row's sum is the same
 * sequence of additions as in a single-threaded loop.
 */
static int64_t orc_find_row(const int64_t *rows, int64_t nsel, int64_t i) {
    int64_t a = 0, z = nsel - 1;
    while (a < z) {
        const int64_t m = (a + z) / 2;
        if (rows[m] < i) a = m + 1;
        else z = m;
    }
    return a;
}

void orc_mttkrp_rows(int64_t nnz, int N, const uint32_t *coords, const double *vals,
                     const int64_t *dims, int R, const double *const *factors, int mode,
                     const int64_t *rows, int64_t nsel, double *Msel, double *Ssel) {
    memset(Msel, 0, sizeof(double) * (size_t)nsel * (size_t)R);
    memset(Ssel, 0, sizeof(double) * (size_t)nsel * (size_t)R);
    if (nsel <= 0) return;
    const int64_t I = dims[mode];
    /* The nonzeros are cut into NC consecutive chunks; chunk t's hits on row
     * k land after those of chunks 0..t-1, so every list stays in input
     * order whichever thread handles which chunk. */
    enum { NC = 64 };
    const int64_t per = (nnz + NC - 1) / NC;
    unsigned char *chosen = (unsigned char *)calloc((size_t)(I / 8 + 1), 1);
    int64_t *start = (int64_t *)calloc((size_t)nsel + 1, sizeof(int64_t));
    int64_t *at = (int64_t *)calloc((size_t)NC * (size_t)nsel, sizeof(int64_t)); /* [chunk][row] */
    int64_t *list = NULL;
    if (!chosen || !start || !at) goto done;
    for (int64_t k = 0; k < nsel; ++k) chosen[rows[k] >> 3] |= (unsigned char)(1u << (rows[k] & 7));
#pragma omp parallel for schedule(static)
    for (int t = 0; t < NC; ++t) {
        const int64_t j1 = (t + 1) * per < nnz ? (t + 1) * per : nnz;
        for (int64_t j = t * per; j < j1; ++j) {
            const int64_t i = coords[j * N + mode];
            if ((chosen[i >> 3] >> (i & 7)) & 1) at[(int64_t)t * nsel + orc_find_row(rows, nsel, i)]++;
        }
    }
    for (int64_t k = 0; k < nsel; ++k) {
        int64_t pos = start[k];
        for (int t = 0; t < NC; ++t) {
            const int64_t c = at[(int64_t)t * nsel + k];
            at[(int64_t)t * nsel + k] = pos;
            pos += c;
        }
        start[k + 1] = pos;
    }
    list = (int64_t *)malloc(sizeof(int64_t) * (size_t)(start[nsel] > 0 ? start[nsel] : 1));
    if (!list) goto done;
#pragma omp parallel for schedule(static)
    for (int t = 0; t < NC; ++t) {
        int64_t *fill = at + (int64_t)t * nsel;
        const int64_t j1 = (t + 1) * per < nnz ? (t + 1) * per : nnz;
        for (int64_t j = t * per; j < j1; ++j) {
            const int64_t i = coords[j * N + mode];
            if ((chosen[i >> 3] >> (i & 7)) & 1) list[fill[orc_find_row(rows, nsel, i)]++] = j;
        }
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t k = 0; k < nsel; ++k) {
        double *m = Msel + k * R;
        double *sa = Ssel + k * R;
        for (int64_t q = start[k]; q < start[k + 1]; ++q) {
            const int64_t j = list[q];
            const uint32_t *c = coords + j * N;
            for (int r = 0; r < R; ++r) {
                double t = vals[j];
                for (int kk = 0; kk < N; ++kk)
                    if (kk != mode) t *= factors[kk][(int64_t)c[kk] * R + r];
                m[r] += t;
                sa[r] += fabs(t);
            }
        }
    }
done:
    free(chosen);
    free(start);
    free(at);
    free(list);
}

/* CP model value at each nonzero: xhat_j = sum_r prod_n A_n[i_n^j, r]. */
void orc_cp_model(int64_t nnz, int N, const uint32_t *coords, int R,
                  const double *const *factors, double *xhat) {
    for (int64_t j = 0; j < nnz; ++j) {
        const uint32_t *c = coords + j * N;
        double acc = 0.0;
        for (int r = 0; r < R; ++r) {
            double t = 1.0;
            for (int k = 0; k < N; ++k) t *= factors[k][(int64_t)c[k] * R + r];
            acc += t;
        }
        xhat[j] = acc;
    }
}

/*
 * binary32 -> bfloat16 (kept in a binary32 container): keep the sign, the
 * exponent and the top 7 fraction bits; round the dropped 16 bits to nearest,
 * ties to the even kept value. NaN stays NaN (quiet), infinities stay.
 */
void orc_bf16_rne(int64_t n, const float *x, float *y) {
    for (int64_t i = 0; i < n; ++i) {
        uint32_t u;
        memcpy(&u, &x[i], 4);
        uint32_t exp = (u >> 23) & 0xFFu, frac = u & 0x7FFFFFu;
        uint32_t out;
        if (exp == 0xFFu && frac != 0) {
            out = (u & 0xFFFF0000u) | 0x00400000u; /* quiet NaN, sign kept */
        } else {
            uint32_t kept = u >> 16;      /* sign, exponent, 7 fraction bits */
            uint32_t dropped = u & 0xFFFFu;
            if (dropped > 0x8000u || (dropped == 0x8000u && (kept & 1u))) kept += 1u;
            out = kept << 16;
        }
        memcpy(&y[i], &out, 4);
    }
}
