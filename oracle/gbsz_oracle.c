/*
 * gbsz_oracle.c -- plain, slow, single-threaded CPU oracle of the cuSZ path
 * (Tian et al., PACT 2020, arXiv 2007.09625).
 *
 * TEST INFRASTRUCTURE ONLY: read by tests/, the smoke check and the
 * benchmark's CPU-baseline leg.  The CUDA library neither includes nor links
 * this file, and this file knows nothing of the CUDA library.
 *
 * Every step follows the paper in its own order and notation:
 *   S0  error bound (valrel footnote, Sec. 3.2.2)
 *   S1  prequantization d° = round(d / 2eb)            (Sec. 3.1.2)
 *       with the watchdog idea of Algorithm 1
 *   S2  Lorenzo prediction and postquantization          (Sec. 3.1.2, Alg. 2)
 *   S3  histogram of quant codes                         (Sec. 3.2.1)
 *   S4  Huffman tree -> code lengths -> canonical codes  (Sec. 3.2.2, 3.2.3)
 *   S5  encode + deflate per chunk                       (Sec. 3.2.4)
 *   S7  inflate with the canonical reverse codebook     (Sec. 3.3)
 *   S8  reversed dual-quantization, cascading            (Alg. 2, Sec. 3.3)
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - eb scalars: eb = (float)(rel * ((double)max - (double)min)) over finite
 *     values, (float)rel when the range is 0 or nothing is finite; 2eb is the
 *     float product eb*2; 1/(2eb) = (float)(1.0 / (double)(2eb)).
 *   - prequant: t = fl32(d * (1/(2eb))), q = round-half-even(t).  Accepted
 *     only if |d - fl32(2eb * fl32((float)q))| <= eb exactly; else q +- 1 is
 *     tried; else the value is a verbatim exception (raw float bits kept).
 *     Non-finite d, or |t| >= 2^30, is always an exception.
 *   - Lorenzo: one global predictor, zero outside the field; the sign of each
 *     term is (-1)^(|k|+1) as in the printed 2D example; delta = q - p as in
 *     the reconstruction (p + delta) * 2eb; arithmetic modulo 2^32.
 *   - postquant: code = delta + R when |delta| < R and the value is not an
 *     exception; otherwise code 0 and (idx, delta) joins the outlier list.
 *     Every exception is therefore also an outlier.
 *   - Huffman: leaves sorted by (frequency, symbol); the two-queue merge
 *     prefers the leaf queue on equal frequency; the first element popped is
 *     the left child; a single used symbol gets length 1.
 *   - canonical codes: symbols sorted by (length, symbol); first code 0;
 *     next = (prev + 1) << (len - prevlen); bits stored MSB-first.
 *
 * The only floating-point decisions (S1's watchdog) are evaluated exactly:
 * two floats whose difference is compared against eb differ by an amount that
 * double represents exactly whenever the comparison is close (the exponents
 * of d and its reconstruction are then within a few binades of each other);
 * when they are far apart the difference exceeds eb by orders of magnitude.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off (no fast-math).  An OpenMP build
 * of the same file is the multi-core CPU baseline: it runs the element-wise
 * loops marked below in parallel, and replaces the serial loops over chunks,
 * over the outlier list and over the reconstruction cascade with the
 * restatements in the "OpenMP build" section (each computes the same values
 * and statuses in independent pieces).  Both builds yield identical bytes;
 * the single-threaded build never compiles that section.
 */
#include "gbsz_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
/* the OpenMP build's restatements of serial steps (defined with S7 below) */
static void par_minmax(const float *x, uint64_t n, int *any_out, float *lo_out, float *hi_out);
static void par_postquant(const float *x, const int32_t *delta, const uint8_t *exc, uint64_t n,
                          uint32_t radius, uint16_t *codes, uint32_t *out_idx, int32_t *out_delta,
                          uint64_t *m, uint32_t *exc_idx, uint32_t *exc_raw, uint64_t *e);
static int par_histogram(const uint16_t *codes, uint64_t n, uint32_t nbins, uint32_t *hist);
static int par_deflate(const uint16_t *codes, uint64_t n, uint32_t chunk, const uint8_t *len,
                       const uint64_t *code, uint32_t *bits, uint32_t *stream, uint64_t stream_cap,
                       uint64_t *words);
#endif

/* ------------------------------------------------------------------------ */
/* archive layout (little-endian), written out independently of the CUDA side */

#define A_MAGIC 0x5A534247u /* bytes 'G','B','S','Z' */
#define A_VERSION 2u
#define A_HEADER 128u
#define A_MAXLEN 45u /* deepest Huffman leaf possible when n < 2^32 */
/* Chunk anchors (a section of this format, not of the paper): for a 1D field
 * with one order-1 predictor and chunks of at least A_ANCHOR_CHUNK symbols,
 * anchor[c] is the prequantized integer of the last point before chunk c
 * (0 for c = 0), i.e. the value the reconstruction (Alg. 2) reaches there,
 * modulo 2^32.  A decoder can then rebuild every chunk on its own; the
 * oracle only checks them against its own cascade. */
#define A_ANCHOR_CHUNK 1024u

static int anchored(const gbsz_ref_params *p)
{
    return p->ndim == 1 && (p->lorenzo_order <= 1) && p->lorenzo_block == 0 && p->chunk >= A_ANCHOR_CHUNK;
}

static uint64_t align16(uint64_t v) { return (v + 15u) & ~(uint64_t)15u; }

static void put_u16(uint8_t *b, size_t off, uint16_t v) { memcpy(b + off, &v, 2); }
static void put_u32(uint8_t *b, size_t off, uint32_t v) { memcpy(b + off, &v, 4); }
static void put_u64(uint8_t *b, size_t off, uint64_t v) { memcpy(b + off, &v, 8); }
static void put_f32(uint8_t *b, size_t off, float v) { memcpy(b + off, &v, 4); }
static void put_f64(uint8_t *b, size_t off, double v) { memcpy(b + off, &v, 8); }
static uint16_t get_u16(const uint8_t *b, size_t off) { uint16_t v; memcpy(&v, b + off, 2); return v; }
static uint32_t get_u32(const uint8_t *b, size_t off) { uint32_t v; memcpy(&v, b + off, 4); return v; }
static uint64_t get_u64(const uint8_t *b, size_t off) { uint64_t v; memcpy(&v, b + off, 8); return v; }
static float get_f32(const uint8_t *b, size_t off) { float v; memcpy(&v, b + off, 4); return v; }
static double get_f64(const uint8_t *b, size_t off) { double v; memcpy(&v, b + off, 8); return v; }

static uint64_t field_size(uint32_t ndim, const uint64_t dims[3])
{
    uint64_t n = 1;
    for (uint32_t i = 0; i < ndim; i++) n *= dims[i];
    return n;
}

static int check_params(const gbsz_ref_params *p, uint64_t *n_out)
{
    if (!p || p->ndim < 1 || p->ndim > 4) return REF_ERR_INVALID_ARG;
    uint64_t n = 1;
    for (uint32_t i = 0; i < 4; i++) {
        uint64_t d = i < p->ndim ? p->dims[i] : 1;
        if (d == 0 || d >= (1ull << 32)) return REF_ERR_INVALID_ARG;
        n *= d;
        if (n >= (1ull << 32)) return REF_ERR_INVALID_ARG;
    }
    if (!(p->eb > 0.0) || !isfinite(p->eb)) return REF_ERR_INVALID_ARG;
    if (p->eb_mode != REF_EB_ABS && p->eb_mode != REF_EB_REL) return REF_ERR_INVALID_ARG;
    if (p->radius < 2 || p->radius > 32768) return REF_ERR_INVALID_ARG;
    if (p->chunk < 64 || p->chunk > 65536 || (p->chunk & (p->chunk - 1)))
        return REF_ERR_INVALID_ARG;
    if (p->lorenzo_block > 1 || p->lorenzo_order > 3) return REF_ERR_INVALID_ARG;
    if (p->lorenzo_block && p->lorenzo_order > 1) return REF_ERR_INVALID_ARG;
    *n_out = n;
    return REF_OK;
}

/* The predictor's geometry: a 4D field is predicted as 3D with its two
 * slowest extents folded into one (dims[2] * dims[3]). */
static uint32_t lorenzo_geometry(const gbsz_ref_params *p, uint64_t d[3])
{
    d[0] = d[1] = d[2] = 1;
    for (uint32_t i = 0; i < p->ndim && i < 3; i++) d[i] = p->dims[i];
    if (p->ndim == 4) d[2] *= p->dims[3];
    return p->ndim == 4 ? 3u : p->ndim;
}

static uint32_t lorenzo_order(const gbsz_ref_params *p)
{
    return p->lorenzo_order ? p->lorenzo_order : 1u;
}

/* ------------------------------------------------------------------------ */
/* S0: error bound relative to the value range (footnote in Sec. 3.2.2)      */

int gbsz_ref_error_bound(const float *x, uint64_t n, uint32_t eb_mode,
                         double eb, float out[3])
{
    if (!(eb > 0.0) || !isfinite(eb)) return REF_ERR_INVALID_ARG;
    float e;
    if (eb_mode == REF_EB_REL) {
        int any = 0;
        float lo = 0.0f, hi = 0.0f;
#ifdef _OPENMP
        par_minmax(x, n, &any, &lo, &hi);
#else
        for (uint64_t i = 0; i < n; i++) {
            if (!isfinite(x[i])) continue;
            if (!any) { lo = hi = x[i]; any = 1; }
            if (x[i] < lo) lo = x[i];
            if (x[i] > hi) hi = x[i];
        }
#endif
        double range = (double)hi - (double)lo;
        if (!any || range == 0.0) e = (float)eb;
        else e = (float)(eb * range);
    } else if (eb_mode == REF_EB_ABS) {
        e = (float)eb;
    } else {
        return REF_ERR_INVALID_ARG;
    }
    float e2 = e * 2.0f;
    float inv = (float)(1.0 / (double)e2);
    if (!(e > 0.0f) || !isfinite(e) || !isfinite(e2) || !isfinite(inv) || !(inv > 0.0f))
        return REF_ERR_INVALID_ARG;
    out[0] = e;
    out[1] = e2;
    out[2] = inv;
    return REF_OK;
}

/* ------------------------------------------------------------------------ */
/* S1: prequantization, d° = round(d / (2 eb)), with a watchdog              */

/* the value the decompressor will produce for integer q: fl(2eb * fl(q)) */
static float recon_value(int32_t q, float ebx2)
{
    float qf = (float)q;
    return ebx2 * qf;
}

/* |d - r| <= eb, decided exactly (see the header comment) */
static int within_bound(float d, float r, float eb)
{
    double diff = fabs((double)d - (double)r);
    return diff <= (double)eb;
}

int gbsz_ref_prequant_one(float d, const float sc[3], int32_t *q_out)
{
    const float eb = sc[0], ebx2 = sc[1], inv2eb = sc[2];
    if (!isfinite(d)) {
        *q_out = 0;
        return 1;
    }
    float t = d * inv2eb; /* d / (2 eb) as one rounded FP32 multiply */
    if (!(fabsf(t) < 1073741824.0f)) {
        *q_out = t > 0.0f ? (int32_t)1073741824 : -(int32_t)1073741824;
        return 1;
    }
    int32_t q = (int32_t)nearbyintf(t); /* round half to even */
    float r = recon_value(q, ebx2);
    if (within_bound(d, r, eb)) {
        *q_out = q;
        return 0;
    }
    int32_t q2 = d > r ? q + 1 : q - 1;
    if (within_bound(d, recon_value(q2, ebx2), eb)) {
        *q_out = q2;
        return 0;
    }
    *q_out = q;
    return 1;
}

/* ------------------------------------------------------------------------ */
/* S2: Lorenzo predictor with binomial coefficients, order n                 */

static uint64_t binom(uint32_t n, uint32_t k)
{
    uint64_t r = 1;
    for (uint32_t i = 1; i <= k; i++) r = r * (n - k + i) / i;
    return r;
}

uint32_t gbsz_ref_lorenzo_block_extent(uint32_t ndim)
{
    return ndim == 1 ? 32u : ndim == 2 ? 16u : 8u;
}

/* Position of coordinate c inside its block: c itself over the whole field,
 * c mod the block extent in the per-block mode.  A neighbour k steps back
 * exists (is not padding) iff k <= that position. */
static uint64_t in_block(uint64_t c, uint32_t ndim, uint32_t lblock)
{
    return lblock ? c % gbsz_ref_lorenzo_block_extent(ndim) : c;
}

/* The order-n prediction of point (x, y, z) from q (Sec. 3.1.2, "Lorenzo
 * Predictor with Binomial Coefficients"): the sum over every offset k != 0
 * with 0 <= k_j <= n of c(k) q[x - k], where c(k) is the product of the
 * binomials C(n, k_j) times (-1)^(k_x + k_y + k_z + 1).  This is the
 * coefficient of the shift by k in 1 - prod_j (1 - S_j)^n, so the residual
 * q - p is the n-th difference along every dimension and the coefficients
 * sum to 1.  (The printed formula puts one factor (-1)^(k_j + 1) per
 * dimension; for an even number of dimensions that flips every sign, which
 * contradicts its own 2D example and unit weight.)  Points outside the field,
 * or outside the point's block in the per-block mode, count as zero.
 * Arithmetic modulo 2^32. */
static uint32_t lorenzo_predict(const int32_t *q, const uint64_t d[3], uint32_t ndim, uint32_t order,
                                uint32_t lblock, uint64_t x, uint64_t y, uint64_t z)
{
    const uint32_t kz_max = ndim >= 3 ? order : 0;
    const uint32_t ky_max = ndim >= 2 ? order : 0;
    const uint64_t bx = in_block(x, ndim, lblock), by = in_block(y, ndim, lblock),
                   bz = in_block(z, ndim, lblock);
    uint32_t p = 0;
    for (uint32_t kz = 0; kz <= kz_max; kz++)
        for (uint32_t ky = 0; ky <= ky_max; ky++)
            for (uint32_t kx = 0; kx <= order; kx++) {
                if (kx == 0 && ky == 0 && kz == 0) continue;
                if (kx > bx || ky > by || kz > bz) continue;
                uint64_t j = (x - kx) + d[0] * ((y - ky) + d[1] * (z - kz));
                uint64_t c = binom(order, kx) * binom(order, ky) * binom(order, kz);
                int neg = ((kx + ky + kz) % 2) == 0;
                uint32_t term = (uint32_t)c * (uint32_t)q[j];
                p = neg ? p - term : p + term;
            }
    return p;
}

int gbsz_ref_lorenzo_delta_blocked(const int32_t *q, uint32_t ndim,
                                   const uint64_t dims[3], uint32_t order,
                                   uint32_t lblock, int32_t *delta)
{
    if (ndim < 1 || ndim > 3 || order < 1 || order > 4 || lblock > 1) return REF_ERR_INVALID_ARG;
    uint64_t d[3] = {1, 1, 1};
    for (uint32_t i = 0; i < ndim; i++) d[i] = dims[i];
    /* every residual reads only q: rows (or, in 1D, runs of 65536 points)
     * are independent */
    const uint64_t rows = d[1] * d[2], run = 65536;
    const int64_t parts = rows > 1 ? (int64_t)rows : (int64_t)((d[0] + run - 1) / run);
#pragma omp parallel for schedule(static)
    for (int64_t r = 0; r < parts; r++) {
        const uint64_t y = rows > 1 ? (uint64_t)r % d[1] : 0, z = rows > 1 ? (uint64_t)r / d[1] : 0;
        const uint64_t x0 = rows > 1 ? 0 : (uint64_t)r * run;
        const uint64_t x1 = rows > 1 ? d[0] : (x0 + run < d[0] ? x0 + run : d[0]);
        for (uint64_t x = x0; x < x1; x++) {
            uint64_t i = x + d[0] * (y + d[1] * z);
            delta[i] = (int32_t)((uint32_t)q[i] - lorenzo_predict(q, d, ndim, order, lblock, x, y, z));
        }
    }
    return REF_OK;
}

int gbsz_ref_lorenzo_delta(const int32_t *q, uint32_t ndim,
                           const uint64_t dims[3], uint32_t order,
                           int32_t *delta)
{
    return gbsz_ref_lorenzo_delta_blocked(q, ndim, dims, order, 0, delta);
}

/* ------------------------------------------------------------------------ */
/* S1 + S2: dual-quantization of the field (Algorithm 2, compression)         */

int gbsz_ref_dualquant_ex(const float *x, uint32_t ndim,
                          const uint64_t dims[3], const float sc[3],
                          uint32_t radius, uint32_t lblock, uint32_t order,
                          uint16_t *codes, uint32_t *out_idx,
                          int32_t *out_delta, uint64_t *m,
                          uint32_t *exc_idx, uint32_t *exc_raw,
                          uint64_t *e, int32_t *q_keep)
{
    if (ndim < 1 || ndim > 3 || radius < 2 || radius > 32768 || lblock > 1) return REF_ERR_INVALID_ARG;
    if (order < 1 || order > 3 || (lblock && order > 1)) return REF_ERR_INVALID_ARG;
    uint64_t n = field_size(ndim, dims);
    int32_t *q = (int32_t *)malloc(n * sizeof(int32_t) + 1);
    int32_t *delta = (int32_t *)malloc(n * sizeof(int32_t) + 1);
    uint8_t *exc = (uint8_t *)malloc(n + 1);
    if (!q || !delta || !exc) {
        free(q); free(delta); free(exc);
        return REF_ERR_OOM;
    }
    /* prequant: every point independently (the barrier in Algorithm 2) */
#pragma omp parallel for
    for (int64_t i = 0; i < (int64_t)n; i++) exc[i] = (uint8_t)gbsz_ref_prequant_one(x[i], sc, &q[i]);
    /* prediction on the prequantized integers, then postquant */
    gbsz_ref_lorenzo_delta_blocked(q, ndim, dims, order, lblock, delta);
    uint64_t nm = 0, ne = 0;
#ifdef _OPENMP
    par_postquant(x, delta, exc, n, radius, codes, out_idx, out_delta, &nm, exc_idx, exc_raw, &ne);
#else
    for (uint64_t i = 0; i < n; i++) {
        int32_t dl = delta[i];
        int in_cap = dl > -(int32_t)radius && dl < (int32_t)radius;
        if (in_cap && !exc[i]) {
            codes[i] = (uint16_t)(dl + (int32_t)radius);
        } else {
            codes[i] = 0;
            out_idx[nm] = (uint32_t)i;
            out_delta[nm] = dl;
            nm++;
        }
        if (exc[i]) {
            uint32_t raw;
            memcpy(&raw, &x[i], 4);
            exc_idx[ne] = (uint32_t)i;
            exc_raw[ne] = raw;
            ne++;
        }
    }
#endif
    *m = nm;
    *e = ne;
    if (q_keep) memcpy(q_keep, q, n * sizeof(int32_t));
    free(q); free(delta); free(exc);
    return REF_OK;
}

int gbsz_ref_dualquant(const float *x, uint32_t ndim, const uint64_t dims[3],
                       const float sc[3], uint32_t radius, uint16_t *codes,
                       uint32_t *out_idx, int32_t *out_delta, uint64_t *m,
                       uint32_t *exc_idx, uint32_t *exc_raw, uint64_t *e,
                       int32_t *q_keep)
{
    return gbsz_ref_dualquant_ex(x, ndim, dims, sc, radius, 0, 1, codes, out_idx, out_delta, m,
                                      exc_idx, exc_raw, e, q_keep);
}

/* ------------------------------------------------------------------------ */
/* S3: histogram                                                              */

int gbsz_ref_histogram(const uint16_t *codes, uint64_t n, uint32_t nbins,
                       uint32_t *hist)
{
    memset(hist, 0, nbins * sizeof(uint32_t));
#ifdef _OPENMP
    return par_histogram(codes, n, nbins, hist);
#endif
    for (uint64_t i = 0; i < n; i++) {
        if (codes[i] >= nbins) return REF_ERR_INVALID_ARG;
        hist[codes[i]]++;
    }
    return REF_OK;
}

/* ------------------------------------------------------------------------ */
/* S4a: Huffman tree by two queues, then leaf depths                         */

typedef struct { uint64_t f; uint32_t sym; } leaf_t;

static int leaf_cmp(const void *a, const void *b)
{
    const leaf_t *u = (const leaf_t *)a, *v = (const leaf_t *)b;
    if (u->f != v->f) return u->f < v->f ? -1 : 1;
    return u->sym < v->sym ? -1 : (u->sym > v->sym);
}

int gbsz_ref_huffman_lengths(const uint32_t *hist, uint32_t nbins,
                             uint8_t *len, uint32_t *maxlen)
{
    memset(len, 0, nbins);
    uint32_t k = 0;
    for (uint32_t s = 0; s < nbins; s++) k += hist[s] > 0;
    *maxlen = 0;
    if (k == 0) return REF_ERR_INVALID_ARG;
    leaf_t *leaf = (leaf_t *)malloc(k * sizeof(leaf_t));
    uint64_t *f = (uint64_t *)malloc((2 * (size_t)k) * sizeof(uint64_t));
    uint32_t *parent = (uint32_t *)malloc((2 * (size_t)k) * sizeof(uint32_t));
    uint32_t *depth = (uint32_t *)malloc((2 * (size_t)k) * sizeof(uint32_t));
    if (!leaf || !f || !parent || !depth) {
        free(leaf); free(f); free(parent); free(depth);
        return REF_ERR_OOM;
    }
    for (uint32_t s = 0, j = 0; s < nbins; s++)
        if (hist[s]) { leaf[j].f = hist[s]; leaf[j].sym = s; j++; }
    qsort(leaf, k, sizeof(leaf_t), leaf_cmp);
    if (k == 1) {
        len[leaf[0].sym] = 1;
        *maxlen = 1;
        free(leaf); free(f); free(parent); free(depth);
        return REF_OK;
    }
    /* nodes 0..k-1: leaves in sorted order; k..2k-2: internal, FIFO order */
    for (uint32_t i = 0; i < k; i++) f[i] = leaf[i].f;
    uint32_t lh = 0, ih = k, next = k;
    for (uint32_t step = 0; step + 1 < k; step++) {
        uint32_t pick[2];
        for (int t = 0; t < 2; t++) {
            int take_leaf = lh < k && (ih >= next || f[lh] <= f[ih]);
            pick[t] = take_leaf ? lh++ : ih++;
        }
        f[next] = f[pick[0]] + f[pick[1]];
        parent[pick[0]] = next;
        parent[pick[1]] = next;
        next++;
    }
    uint32_t root = 2 * k - 2;
    depth[root] = 0;
    for (int64_t i = (int64_t)root - 1; i >= 0; i--) depth[i] = depth[parent[i]] + 1;
    uint32_t mx = 0;
    for (uint32_t i = 0; i < k; i++) {
        len[leaf[i].sym] = (uint8_t)depth[i];
        if (depth[i] > mx) mx = depth[i];
    }
    *maxlen = mx;
    free(leaf); free(f); free(parent); free(depth);
    return mx <= A_MAXLEN ? REF_OK : REF_ERR_INVALID_ARG;
}

/* ------------------------------------------------------------------------ */
/* S4b: canonization                                                          */

typedef struct { uint32_t len, sym; } lsym_t;

static int lsym_cmp(const void *a, const void *b)
{
    const lsym_t *u = (const lsym_t *)a, *v = (const lsym_t *)b;
    if (u->len != v->len) return u->len < v->len ? -1 : 1;
    return u->sym < v->sym ? -1 : (u->sym > v->sym);
}

int gbsz_ref_canonical_codes(const uint8_t *len, uint32_t nbins, uint64_t *code)
{
    memset(code, 0, nbins * sizeof(uint64_t));
    uint32_t k = 0;
    for (uint32_t s = 0; s < nbins; s++) k += len[s] > 0;
    if (k == 0) return REF_OK;
    lsym_t *v = (lsym_t *)malloc(k * sizeof(lsym_t));
    if (!v) return REF_ERR_OOM;
    for (uint32_t s = 0, j = 0; s < nbins; s++)
        if (len[s]) { v[j].len = len[s]; v[j].sym = s; j++; }
    qsort(v, k, sizeof(lsym_t), lsym_cmp);
    uint64_t c = 0;
    for (uint32_t j = 0; j < k; j++) {
        if (j > 0) c = (c + 1) << (v[j].len - v[j - 1].len);
        code[v[j].sym] = c;
    }
    free(v);
    return REF_OK;
}

/* ------------------------------------------------------------------------ */
/* S5: encode + deflate, one chunk after another                              */

static uint64_t nchunks(uint64_t n, uint32_t chunk) { return (n + chunk - 1) / chunk; }

int gbsz_ref_deflate(const uint16_t *codes, uint64_t n, uint32_t chunk,
                     const uint8_t *len, const uint64_t *code,
                     uint32_t *bits, uint32_t *stream, uint64_t stream_cap,
                     uint64_t *words)
{
#ifdef _OPENMP
    return par_deflate(codes, n, chunk, len, code, bits, stream, stream_cap, words);
#endif
    uint64_t nc = nchunks(n, chunk);
    uint64_t w = 0;
    for (uint64_t c = 0; c < nc; c++) {
        uint64_t lo = c * chunk, hi = lo + chunk < n ? lo + chunk : n;
        uint64_t pos = 0; /* bit position inside the chunk */
        for (uint64_t i = lo; i < hi; i++) {
            uint32_t l = len[codes[i]];
            if (l == 0) return REF_ERR_INVALID_ARG; /* symbol absent from the codebook */
            for (int b = (int)l - 1; b >= 0; b--) { /* MSB first */
                uint64_t word = w + pos / 32;
                if (word >= stream_cap) return REF_ERR_CAPACITY;
                if (pos % 32 == 0) stream[word] = 0;
                if ((code[codes[i]] >> b) & 1u) stream[word] |= 1u << (31 - pos % 32);
                pos++;
            }
        }
        bits[c] = (uint32_t)pos;
        w += (pos + 31) / 32;
    }
    *words = w;
    return REF_OK;
}

/* ------------------------------------------------------------------------ */
/* S7: inflate with the canonical reverse codebook                            */

typedef struct {
    uint32_t maxlen;
    uint64_t first[64];  /* first canonical code of each length */
    uint32_t count[64];  /* number of codes of each length */
    uint32_t start[64];  /* index of the first of them in `sorted` */
    uint32_t *sorted;    /* symbols in (length, symbol) order */
} revbook_t;

static int revbook_build(const uint8_t *len, uint32_t nbins, revbook_t *rb)
{
    memset(rb, 0, sizeof(*rb));
    uint32_t k = 0;
    for (uint32_t s = 0; s < nbins; s++) {
        if (len[s] > A_MAXLEN) return REF_ERR_CORRUPT;
        if (len[s]) { rb->count[len[s]]++; k++; if (len[s] > rb->maxlen) rb->maxlen = len[s]; }
    }
    if (k == 0) return REF_ERR_CORRUPT;
    rb->sorted = (uint32_t *)malloc(k * sizeof(uint32_t));
    if (!rb->sorted) return REF_ERR_OOM;
    uint32_t pos = 0;
    uint64_t c = 0;
    for (uint32_t l = 1; l <= rb->maxlen; l++) {
        rb->start[l] = pos;
        rb->first[l] = c;
        for (uint32_t s = 0; s < nbins; s++)
            if (len[s] == l) rb->sorted[pos++] = s;
        c = (c + rb->count[l]) << 1;
    }
    /* Kraft: a valid length table never overflows its code space */
    uint64_t used = 0;
    for (uint32_t l = 1; l <= rb->maxlen; l++) used += (uint64_t)rb->count[l] << (rb->maxlen - l);
    if (used > (1ull << rb->maxlen)) { free(rb->sorted); rb->sorted = NULL; return REF_ERR_CORRUPT; }
    return REF_OK;
}

/* ------------------------------------------------------------------------ */
/* OpenMP build: serial steps restated in independent pieces               */
/*
 * Compiled only with -fopenmp.  Each function computes exactly what the
 * serial loop it replaces computes (same values, same status), splitting the
 * work where the step itself has independent parts:
 *   par_minmax     S0: min / max of finite values, per range, then merged
 *                  (min and max do not depend on the order);
 *   par_postquant  S2: codes per range, then each range writes its outliers
 *                  and exceptions at offsets from a prefix sum of the counts
 *                  (index order is kept);
 *   par_histogram  S3: per-thread histograms added together;
 *   par_deflate    S5: bits of every chunk, word offsets by a prefix sum,
 *                  then every chunk packs its own words (chunks are
 *                  independent by construction of the format);
 *   par_inflate    S7: word offsets by a prefix sum, then every chunk decodes
 *                  on its own;
 *   par_cascade    S8: the cascade of Algorithm 2, each point predicted from
 *                  points already rebuilt, but in an order that lets threads
 *                  work at once: blocks of the per-block mode are
 *                  independent; a 1D field's order-1 cascade restarts every
 *                  range from the prefix sum of the residuals before it
 *                  (q[i-1] is exactly that sum); 2D and 3D fields go in
 *                  wavefronts of rows (3D: row (y, z) needs only rows of
 *                  smaller y + z) or of row pieces (2D: piece (b, y) needs
 *                  only pieces of smaller b + y).
 */
#ifdef _OPENMP
static void par_minmax(const float *x, uint64_t n, int *any_out, float *lo_out, float *hi_out)
{
    int any = 0;
    float lo = 0.0f, hi = 0.0f;
#pragma omp parallel
    {
        int a = 0;
        float l = 0.0f, h = 0.0f;
#pragma omp for schedule(static) nowait
        for (int64_t i = 0; i < (int64_t)n; i++) {
            if (!isfinite(x[i])) continue;
            if (!a) { l = h = x[i]; a = 1; }
            if (x[i] < l) l = x[i];
            if (x[i] > h) h = x[i];
        }
#pragma omp critical
        if (a) {
            if (!any) { lo = l; hi = h; any = 1; }
            if (l < lo) lo = l;
            if (h > hi) hi = h;
        }
    }
    *any_out = any;
    *lo_out = lo;
    *hi_out = hi;
}

/* index ranges for the two-pass steps: about 64k points each */
static uint64_t par_parts(uint64_t n) { return n / 65536 + 1; }
static uint64_t part_lo(uint64_t n, uint64_t p, uint64_t parts) { return n * p / parts; }

static void par_postquant(const float *x, const int32_t *delta, const uint8_t *exc, uint64_t n,
                          uint32_t radius, uint16_t *codes, uint32_t *out_idx, int32_t *out_delta,
                          uint64_t *m, uint32_t *exc_idx, uint32_t *exc_raw, uint64_t *e)
{
    const uint64_t P = par_parts(n);
    uint64_t *cm = (uint64_t *)calloc(P + 1, sizeof(uint64_t));
    uint64_t *ce = (uint64_t *)calloc(P + 1, sizeof(uint64_t));
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < (int64_t)P; p++) {
        uint64_t nm = 0, ne = 0;
        for (uint64_t i = part_lo(n, p, P); i < part_lo(n, p + 1, P); i++) {
            int32_t dl = delta[i];
            int in_cap = dl > -(int32_t)radius && dl < (int32_t)radius;
            codes[i] = (in_cap && !exc[i]) ? (uint16_t)(dl + (int32_t)radius) : 0;
            nm += codes[i] == 0;
            ne += exc[i] != 0;
        }
        cm[p + 1] = nm;
        ce[p + 1] = ne;
    }
    for (uint64_t p = 0; p < P; p++) {
        cm[p + 1] += cm[p];
        ce[p + 1] += ce[p];
    }
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < (int64_t)P; p++) {
        uint64_t nm = cm[p], ne = ce[p];
        for (uint64_t i = part_lo(n, p, P); i < part_lo(n, p + 1, P); i++) {
            if (codes[i] == 0) {
                out_idx[nm] = (uint32_t)i;
                out_delta[nm] = delta[i];
                nm++;
            }
            if (exc[i]) {
                uint32_t raw;
                memcpy(&raw, &x[i], 4);
                exc_idx[ne] = (uint32_t)i;
                exc_raw[ne] = raw;
                ne++;
            }
        }
    }
    *m = cm[P];
    *e = ce[P];
    free(cm);
    free(ce);
}

static int par_histogram(const uint16_t *codes, uint64_t n, uint32_t nbins, uint32_t *hist)
{
    int bad = 0;
#pragma omp parallel reduction(| : bad)
    {
        uint32_t *h = (uint32_t *)calloc(nbins, sizeof(uint32_t));
        if (!h) bad = 2;
#pragma omp for schedule(static)
        for (int64_t i = 0; i < (int64_t)n; i++) {
            if (!h) continue;
            if (codes[i] >= nbins) bad = 1;
            else h[codes[i]]++;
        }
        if (h) {
#pragma omp critical
            for (uint32_t s = 0; s < nbins; s++) hist[s] += h[s];
        }
        free(h);
    }
    return bad & 2 ? REF_ERR_OOM : bad ? REF_ERR_INVALID_ARG : REF_OK;
}

static int par_deflate(const uint16_t *codes, uint64_t n, uint32_t chunk, const uint8_t *len,
                       const uint64_t *code, uint32_t *bits, uint32_t *stream, uint64_t stream_cap,
                       uint64_t *words)
{
    const uint64_t nc = nchunks(n, chunk);
    uint64_t *cb = (uint64_t *)malloc(nc * sizeof(uint64_t)); /* bits, or bits before an absent symbol */
    uint64_t *off = (uint64_t *)malloc(nc * sizeof(uint64_t));
    uint8_t *absent = (uint8_t *)malloc(nc);
    if (!cb || !off || !absent) {
        free(cb); free(off); free(absent);
        return REF_ERR_OOM;
    }
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t c = 0; c < (int64_t)nc; c++) {
        uint64_t lo = (uint64_t)c * chunk, hi = lo + chunk < n ? lo + chunk : n, pos = 0;
        absent[c] = 0;
        for (uint64_t i = lo; i < hi; i++) {
            if (len[codes[i]] == 0) { absent[c] = 1; break; }
            pos += len[codes[i]];
        }
        cb[c] = pos;
    }
    /* statuses in the order the serial loop meets them: a bit past the
     * capacity, or a symbol without a code, whichever comes first */
    uint64_t w = 0;
    int st = REF_OK;
    for (uint64_t c = 0; c < nc && st == REF_OK; c++) {
        if (cb[c] > 0 && w + (cb[c] - 1) / 32 >= stream_cap) st = REF_ERR_CAPACITY;
        else if (absent[c]) st = REF_ERR_INVALID_ARG;
        off[c] = w;
        w += (cb[c] + 31) / 32;
    }
    if (st == REF_OK) {
#pragma omp parallel for schedule(dynamic, 64)
        for (int64_t c = 0; c < (int64_t)nc; c++) {
            uint64_t lo = (uint64_t)c * chunk, hi = lo + chunk < n ? lo + chunk : n, pos = 0;
            for (uint64_t i = lo; i < hi; i++) {
                uint32_t l = len[codes[i]];
                for (int b = (int)l - 1; b >= 0; b--) { /* MSB first */
                    uint64_t word = off[c] + pos / 32;
                    if (pos % 32 == 0) stream[word] = 0;
                    if ((code[codes[i]] >> b) & 1u) stream[word] |= 1u << (31 - pos % 32);
                    pos++;
                }
            }
            bits[c] = (uint32_t)pos;
        }
        *words = w;
    }
    free(cb); free(off); free(absent);
    return st;
}

static int par_inflate(const uint32_t *stream, uint64_t words, const uint32_t *bits, uint64_t n,
                       uint32_t chunk, const revbook_t *rb, uint16_t *codes)
{
    const uint64_t nc = nchunks(n, chunk);
    uint64_t *off = (uint64_t *)malloc(nc * sizeof(uint64_t) + 8);
    if (!off) return REF_ERR_OOM;
    uint64_t w = 0;
    int st = REF_OK;
    for (uint64_t c = 0; c < nc; c++) {
        off[c] = w;
        w += ((uint64_t)bits[c] + 31) / 32;
        if (w > words) { st = REF_ERR_CORRUPT; break; }
    }
    if (st == REF_OK) {
        int bad = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(| : bad)
        for (int64_t c = 0; c < (int64_t)nc; c++) {
            uint64_t lo = (uint64_t)c * chunk, hi = lo + chunk < n ? lo + chunk : n;
            uint64_t nb = bits[c], pos = 0;
            int ok = 1;
            for (uint64_t i = lo; i < hi && ok; i++) {
                uint64_t v = 0;
                uint32_t l = 0;
                for (;;) {
                    if (pos >= nb || l >= rb->maxlen) { ok = 0; break; }
                    uint32_t bit = (stream[off[c] + pos / 32] >> (31 - pos % 32)) & 1u;
                    v = (v << 1) | bit;
                    pos++;
                    l++;
                    if (v - rb->first[l] < rb->count[l]) {
                        codes[i] = (uint16_t)rb->sorted[rb->start[l] + (uint32_t)(v - rb->first[l])];
                        break;
                    }
                }
            }
            if (!ok || pos != nb) bad = 1;
        }
        if (bad) st = REF_ERR_CORRUPT;
    }
    free(off);
    return st;
}

/* one point of the cascade: q = p + delta (mod 2^32) */
static void cascade_point(int32_t *q, const int32_t *dl, const uint64_t d[3], uint32_t ndim, uint32_t order,
                          uint32_t lblock, uint64_t x, uint64_t y, uint64_t z)
{
    const uint64_t i = x + d[0] * (y + d[1] * z);
    q[i] = (int32_t)(lorenzo_predict(q, d, ndim, order, lblock, x, y, z) + (uint32_t)dl[i]);
}

static int par_cascade(const uint16_t *codes, uint32_t ndim, const uint64_t d[3], uint32_t radius,
                       uint32_t lblock, uint32_t order, const uint32_t *out_idx, const int32_t *out_delta,
                       uint64_t m, int32_t *q)
{
    const uint64_t n = d[0] * d[1] * d[2];
    const uint64_t P = par_parts(n);
    int32_t *dl = (int32_t *)malloc(n * sizeof(int32_t) + 4);
    uint64_t *cz = (uint64_t *)calloc(P + 1, sizeof(uint64_t));
    if (!dl || !cz) {
        free(dl); free(cz);
        return REF_ERR_OOM;
    }
    /* The serial loop takes the outliers in index order: the r-th code-0
     * point takes entry r.  It succeeds exactly when there are m code-0
     * points and entry r names the r-th of them (then no entry can name a
     * point whose code is not 0). */
#pragma omp parallel for schedule(static)
    for (int64_t p = 0; p < (int64_t)P; p++) {
        uint64_t z0 = 0;
        for (uint64_t i = part_lo(n, p, P); i < part_lo(n, p + 1, P); i++) z0 += codes[i] == 0;
        cz[p + 1] = z0;
    }
    for (uint64_t p = 0; p < P; p++) cz[p + 1] += cz[p];
    int bad = cz[P] != m;
    if (!bad) {
#pragma omp parallel for schedule(static) reduction(| : bad)
        for (int64_t p = 0; p < (int64_t)P; p++) {
            uint64_t r = cz[p];
            for (uint64_t i = part_lo(n, p, P); i < part_lo(n, p + 1, P); i++) {
                if (codes[i] != 0) {
                    dl[i] = (int32_t)codes[i] - (int32_t)radius;
                } else {
                    if (out_idx[r] != i) bad = 1;
                    dl[i] = out_delta[r++];
                }
            }
        }
    }
    free(cz);
    if (bad) {
        free(dl);
        return REF_ERR_CORRUPT;
    }
    if (lblock) {
        /* every block of the per-block mode is a field of its own */
        const uint64_t B = gbsz_ref_lorenzo_block_extent(ndim);
        const uint64_t nb0 = (d[0] + B - 1) / B, nb1 = ndim >= 2 ? (d[1] + B - 1) / B : 1,
                       nb2 = ndim >= 3 ? (d[2] + B - 1) / B : 1;
#pragma omp parallel for schedule(dynamic, 256)
        for (int64_t b = 0; b < (int64_t)(nb0 * nb1 * nb2); b++) {
            const uint64_t bx = (uint64_t)b % nb0, by = ((uint64_t)b / nb0) % nb1, bz = (uint64_t)b / (nb0 * nb1);
            const uint64_t Bz = ndim >= 3 ? B : 1, By = ndim >= 2 ? B : 1;
            for (uint64_t z = bz * Bz; z < d[2] && z < (bz + 1) * Bz; z++)
                for (uint64_t y = by * By; y < d[1] && y < (by + 1) * By; y++)
                    for (uint64_t x = bx * B; x < d[0] && x < (bx + 1) * B; x++)
                        cascade_point(q, dl, d, ndim, order, lblock, x, y, z);
        }
    } else if (ndim == 1 && order == 1) {
        /* range p starts from the sum of every residual before it, which is
         * q at the point before the range */
        uint32_t *carry = (uint32_t *)calloc(P + 1, sizeof(uint32_t));
        if (!carry) { free(dl); return REF_ERR_OOM; }
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < (int64_t)P; p++) {
            uint32_t sum = 0;
            for (uint64_t i = part_lo(n, p, P); i < part_lo(n, p + 1, P); i++) sum += (uint32_t)dl[i];
            carry[p + 1] = sum;
        }
        for (uint64_t p = 0; p < P; p++) carry[p + 1] += carry[p];
#pragma omp parallel for schedule(static)
        for (int64_t p = 0; p < (int64_t)P; p++) {
            const uint64_t lo = part_lo(n, p, P), hi = part_lo(n, p + 1, P);
            if (lo == hi) continue;
            q[lo] = (int32_t)(carry[p] + (uint32_t)dl[lo]);
            for (uint64_t x = lo + 1; x < hi; x++) cascade_point(q, dl, d, ndim, order, lblock, x, 0, 0);
        }
        free(carry);
    } else if (ndim == 1) {
        for (uint64_t x = 0; x < d[0]; x++) cascade_point(q, dl, d, ndim, order, lblock, x, 0, 0);
    } else {
        /* tasks (b, y, z): x in [b W, (b+1) W) of row (y, z); a point's
         * neighbours lie in tasks of smaller b + y + z, or earlier in its own
         * task (W >= order) */
        const uint64_t W = ndim == 2 ? 128 : d[0];
        const uint64_t nbx = (d[0] + W - 1) / W;
        const uint64_t kmax = (nbx - 1) + (d[1] - 1) + (d[2] - 1);
        for (uint64_t k = 0; k <= kmax; k++) {
            /* tasks of wavefront k: z from zlo, y = k - b - z */
            const uint64_t zlo = k > (nbx - 1) + (d[1] - 1) ? k - (nbx - 1) - (d[1] - 1) : 0;
            const uint64_t zhi = k < d[2] - 1 ? k : d[2] - 1;
            const uint64_t nz = zhi - zlo + 1;
#pragma omp parallel for schedule(dynamic, 1) collapse(2)
            for (int64_t zi = 0; zi < (int64_t)nz; zi++)
                for (int64_t b = 0; b < (int64_t)nbx; b++) {
                    const uint64_t z = zlo + (uint64_t)zi;
                    if ((uint64_t)b + z > k || k - (uint64_t)b - z > d[1] - 1) continue;
                    const uint64_t y = k - (uint64_t)b - z;
                    for (uint64_t x = (uint64_t)b * W; x < d[0] && x < ((uint64_t)b + 1) * W; x++)
                        cascade_point(q, dl, d, ndim, order, lblock, x, y, z);
                }
        }
    }
    free(dl);
    return REF_OK;
}
#endif /* _OPENMP */

int gbsz_ref_inflate(const uint32_t *stream, uint64_t words,
                     const uint32_t *bits, uint64_t n, uint32_t chunk,
                     const uint8_t *len, uint32_t nbins, uint16_t *codes)
{
    revbook_t rb;
    int st = revbook_build(len, nbins, &rb);
    if (st) return st;
#ifdef _OPENMP
    st = par_inflate(stream, words, bits, n, chunk, &rb, codes);
    free(rb.sorted);
    return st;
#endif
    uint64_t nc = nchunks(n, chunk), w = 0;
    for (uint64_t c = 0; c < nc && st == REF_OK; c++) {
        uint64_t lo = c * chunk, hi = lo + chunk < n ? lo + chunk : n;
        uint64_t nb = bits[c], cw = (nb + 31) / 32;
        if (w + cw > words) { st = REF_ERR_CORRUPT; break; }
        uint64_t pos = 0;
        for (uint64_t i = lo; i < hi && st == REF_OK; i++) {
            uint64_t v = 0;
            uint32_t l = 0;
            for (;;) {
                if (pos >= nb || l >= rb.maxlen) { st = REF_ERR_CORRUPT; break; }
                uint32_t bit = (stream[w + pos / 32] >> (31 - pos % 32)) & 1u;
                v = (v << 1) | bit;
                pos++;
                l++;
                if (v - rb.first[l] < rb.count[l]) { /* unsigned: v >= first */
                    codes[i] = (uint16_t)rb.sorted[rb.start[l] + (uint32_t)(v - rb.first[l])];
                    break;
                }
            }
        }
        if (st == REF_OK && pos != nb) st = REF_ERR_CORRUPT;
        w += cw;
    }
    free(rb.sorted);
    return st;
}

/* ------------------------------------------------------------------------ */
/* S8: reversed dual-quantization, reconstructed cascadingly (Algorithm 2)   */

/* The cascade of Alg. 2; with anchors (na entries, chunk C), every anchor
 * must equal the reconstructed integer of the point before its chunk (0 for
 * the first chunk), else the archive is corrupt. */
static int reconstruct_anchored(const uint16_t *codes, uint32_t ndim,
                                const uint64_t dims[3], uint32_t radius,
                                uint32_t lblock, uint32_t order,
                                const uint32_t *out_idx,
                                const int32_t *out_delta, uint64_t m,
                                const uint32_t *exc_idx,
                                const uint32_t *exc_raw, uint64_t e,
                                float ebx2, float *xr,
                                const uint32_t *anchors, uint64_t na, uint32_t chunk)
{
    if (ndim < 1 || ndim > 3 || lblock > 1) return REF_ERR_INVALID_ARG;
    if (order < 1 || order > 3 || (lblock && order > 1)) return REF_ERR_INVALID_ARG;
    uint64_t d[3] = {1, 1, 1};
    for (uint32_t i = 0; i < ndim; i++) d[i] = dims[i];
    uint64_t n = d[0] * d[1] * d[2];
    int32_t *q = (int32_t *)malloc(n * sizeof(int32_t) + 1);
    if (!q) return REF_ERR_OOM;
#ifdef _OPENMP
    {
        const int pst = par_cascade(codes, ndim, d, radius, lblock, order, out_idx, out_delta, m, q);
        if (pst) { free(q); return pst; }
    }
#else
    uint64_t j = 0; /* next outlier */
    for (uint64_t z = 0; z < d[2]; z++)
        for (uint64_t y = 0; y < d[1]; y++)
            for (uint64_t x = 0; x < d[0]; x++) {
                uint64_t i = x + d[0] * (y + d[1] * z);
                int32_t dl;
                if (codes[i] != 0) {
                    dl = (int32_t)codes[i] - (int32_t)radius;
                    if (j < m && out_idx[j] == i) { free(q); return REF_ERR_CORRUPT; }
                } else {
                    if (j >= m || out_idx[j] != i) { free(q); return REF_ERR_CORRUPT; }
                    dl = out_delta[j++];
                }
                /* p = l(q of the reconstructed points before this one) */
                const uint32_t p = lorenzo_predict(q, d, ndim, order, lblock, x, y, z);
                q[i] = (int32_t)(p + (uint32_t)dl);
            }
    if (j != m) { free(q); return REF_ERR_CORRUPT; }
#endif
    {
        int bad = 0;
#pragma omp parallel for reduction(| : bad)
        for (int64_t c = 0; c < (int64_t)na; c++) {
            const uint32_t want = c == 0 ? 0u : (uint32_t)q[(uint64_t)c * chunk - 1];
            if (anchors[c] != want) bad = 1;
        }
        if (bad) { free(q); return REF_ERR_CORRUPT; }
    }
#pragma omp parallel for
    for (int64_t i = 0; i < (int64_t)n; i++) xr[i] = recon_value(q[i], ebx2);
    for (uint64_t t = 0; t < e; t++) {
        if (exc_idx[t] >= n || (t > 0 && exc_idx[t] <= exc_idx[t - 1])) { free(q); return REF_ERR_CORRUPT; }
        memcpy(&xr[exc_idx[t]], &exc_raw[t], 4);
    }
    free(q);
    return REF_OK;
}

int gbsz_ref_reconstruct_ex(const uint16_t *codes, uint32_t ndim,
                            const uint64_t dims[3], uint32_t radius,
                            uint32_t lblock, uint32_t order,
                            const uint32_t *out_idx,
                            const int32_t *out_delta, uint64_t m,
                            const uint32_t *exc_idx,
                            const uint32_t *exc_raw, uint64_t e,
                            float ebx2, float *xr)
{
    return reconstruct_anchored(codes, ndim, dims, radius, lblock, order, out_idx, out_delta, m, exc_idx,
                                exc_raw, e, ebx2, xr, NULL, 0, 0);
}

int gbsz_ref_reconstruct(const uint16_t *codes, uint32_t ndim,
                         const uint64_t dims[3], uint32_t radius,
                         const uint32_t *out_idx, const int32_t *out_delta,
                         uint64_t m, const uint32_t *exc_idx,
                         const uint32_t *exc_raw, uint64_t e, float ebx2,
                         float *xr)
{
    return gbsz_ref_reconstruct_ex(codes, ndim, dims, radius, 0, 1, out_idx, out_delta, m,
                                        exc_idx, exc_raw, e, ebx2, xr);
}

/* ------------------------------------------------------------------------ */
/* whole path                                                                 */

/* threads the parallel loops of this build use (1 in the single-threaded
 * build) */
int gbsz_ref_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

size_t gbsz_ref_compress_bound(const gbsz_ref_params *p)
{
    uint64_t n;
    if (check_params(p, &n)) return 0;
    uint64_t nc = nchunks(n, p->chunk);
    uint64_t words_max = nc + (A_MAXLEN * n + 31) / 32;
    return (size_t)(208 + 2ull * p->radius + 12 * nc + 16 * n + 4 * words_max);
}

int gbsz_ref_compress(const float *x, const gbsz_ref_params *p, void *archive,
                      size_t capacity, size_t *out_bytes)
{
    uint64_t n;
    int st = check_params(p, &n);
    if (st) return st;
    float sc[3];
    st = gbsz_ref_error_bound(x, n, p->eb_mode, p->eb, sc);
    if (st) return st;
    const uint32_t R = p->radius, nbins = 2 * R, C = p->chunk;
    const uint64_t nc = nchunks(n, C);
    uint64_t dims[3];
    const uint32_t gnd = lorenzo_geometry(p, dims);

    uint16_t *codes = (uint16_t *)malloc(n * 2 + 2);
    uint32_t *oidx = (uint32_t *)malloc(n * 4 + 4);
    int32_t *odel = (int32_t *)malloc(n * 4 + 4);
    uint32_t *eidx = (uint32_t *)malloc(n * 4 + 4);
    uint32_t *eraw = (uint32_t *)malloc(n * 4 + 4);
    uint32_t *hist = (uint32_t *)malloc(nbins * 4);
    uint8_t *len = (uint8_t *)malloc(nbins);
    uint64_t *code = (uint64_t *)malloc(nbins * 8);
    uint32_t *bits = (uint32_t *)malloc(nc * 4);
    uint64_t scap = nc + (A_MAXLEN * n + 31) / 32;
    uint32_t *stream = (uint32_t *)malloc(scap * 4 + 4);
    uint64_t m = 0, e = 0, w = 0;
    uint32_t maxlen = 0;
    if (!codes || !oidx || !odel || !eidx || !eraw || !hist || !len || !code || !bits || !stream) {
        st = REF_ERR_OOM;
        goto done;
    }
    st = gbsz_ref_dualquant_ex(x, gnd, dims, sc, R, p->lorenzo_block, lorenzo_order(p), codes, oidx, odel,
                               &m, eidx, eraw, &e, NULL);
    if (st) goto done;
    st = gbsz_ref_histogram(codes, n, nbins, hist);
    if (st) goto done;
    st = gbsz_ref_huffman_lengths(hist, nbins, len, &maxlen);
    if (st) goto done;
    st = gbsz_ref_canonical_codes(len, nbins, code);
    if (st) goto done;
    st = gbsz_ref_deflate(codes, n, C, len, code, bits, stream, scap, &w);
    if (st) goto done;
    {
        const uint64_t na = anchored(p) ? nc : 0;
        uint64_t off_len = A_HEADER;
        uint64_t off_bits = align16(off_len + nbins);
        uint64_t off_anc = align16(off_bits + 4 * nc);
        uint64_t off_out = align16(off_anc + 4 * na);
        uint64_t off_exc = off_out + 8 * m;
        uint64_t off_str = align16(off_exc + 8 * e);
        uint64_t total = off_str + 4 * w;
        *out_bytes = (size_t)total;
        if (total > capacity) { st = REF_ERR_CAPACITY; goto done; }
        uint8_t *a = (uint8_t *)archive;
        memset(a, 0, (size_t)total);
        put_u32(a, 0, A_MAGIC);
        put_u16(a, 4, (uint16_t)A_VERSION);
        put_u16(a, 6, (uint16_t)A_HEADER);
        put_u32(a, 8, p->ndim);
        put_u32(a, 12, p->eb_mode);
        put_u64(a, 16, p->dims[0]);
        put_u64(a, 24, p->ndim >= 2 ? p->dims[1] : 1);
        put_u64(a, 32, p->ndim >= 3 ? p->dims[2] : 1);
        put_u64(a, 40, n);
        put_f64(a, 48, p->eb);
        put_f32(a, 56, sc[0]);
        put_f32(a, 60, sc[1]);
        put_f32(a, 64, sc[2]);
        put_u32(a, 68, R);
        put_u32(a, 72, C);
        put_u32(a, 76, (uint32_t)nc);
        put_u64(a, 80, m);
        put_u64(a, 88, e);
        put_u64(a, 96, w);
        put_u32(a, 104, maxlen);
        put_u32(a, 108, p->lorenzo_block); /* 0: one predictor; 1: per block */
        put_u64(a, 112, total);
        put_u32(a, 120, lorenzo_order(p));
        put_u32(a, 124, p->ndim == 4 ? (uint32_t)p->dims[3] : 1u); /* below 2^32 as n is */
        memcpy(a + off_len, len, nbins);
#pragma omp parallel for
        for (int64_t c = 0; c < (int64_t)nc; c++) put_u32(a, off_bits + 4 * c, bits[c]);
        /* anchors: the prequantized integer of the point before each chunk */
#pragma omp parallel for
        for (int64_t c = 1; c < (int64_t)na; c++) {
            int32_t qa;
            gbsz_ref_prequant_one(x[(uint64_t)c * C - 1], sc, &qa);
            put_u32(a, off_anc + 4 * c, (uint32_t)qa);
        }
#pragma omp parallel for
        for (int64_t t = 0; t < (int64_t)m; t++) {
            put_u32(a, off_out + 8 * t, oidx[t]);
            put_u32(a, off_out + 8 * t + 4, (uint32_t)odel[t]);
        }
        for (uint64_t t = 0; t < e; t++) {
            put_u32(a, off_exc + 8 * t, eidx[t]);
            put_u32(a, off_exc + 8 * t + 4, eraw[t]);
        }
#pragma omp parallel for
        for (int64_t t = 0; t < (int64_t)w; t++) put_u32(a, off_str + 4 * t, stream[t]);
    }
done:
    free(codes); free(oidx); free(odel); free(eidx); free(eraw);
    free(hist); free(len); free(code); free(bits); free(stream);
    return st;
}

typedef struct {
    gbsz_ref_params p;
    uint64_t n, nc, m, e, w, total;
    float sc[3];
    uint32_t maxlen;
    uint64_t off_len, off_bits, off_anc, off_out, off_exc, off_str;
    uint64_t na; /* anchors: nc or 0 */
} hdr_t;

static int parse_header(const uint8_t *a, size_t bytes, hdr_t *h)
{
    if (!a || bytes < A_HEADER) return REF_ERR_CORRUPT;
    if (get_u32(a, 0) != A_MAGIC || get_u16(a, 4) != A_VERSION || get_u16(a, 6) != A_HEADER)
        return REF_ERR_CORRUPT;
    memset(h, 0, sizeof(*h));
    h->p.ndim = get_u32(a, 8);
    h->p.eb_mode = get_u32(a, 12);
    for (int i = 0; i < 3; i++) h->p.dims[i] = get_u64(a, 16 + 8 * i);
    h->p.dims[3] = get_u32(a, 124);
    h->p.lorenzo_order = get_u32(a, 120);
    h->p.lorenzo_block = get_u32(a, 108);
    h->n = get_u64(a, 40);
    h->p.eb = get_f64(a, 48);
    h->sc[0] = get_f32(a, 56);
    h->sc[1] = get_f32(a, 60);
    h->sc[2] = get_f32(a, 64);
    h->p.radius = get_u32(a, 68);
    h->p.chunk = get_u32(a, 72);
    h->nc = get_u32(a, 76);
    h->m = get_u64(a, 80);
    h->e = get_u64(a, 88);
    h->w = get_u64(a, 96);
    h->maxlen = get_u32(a, 104);
    h->total = get_u64(a, 112);
    uint64_t n;
    if (check_params(&h->p, &n) || n != h->n) return REF_ERR_CORRUPT;
    for (uint32_t i = h->p.ndim; i < 4; i++)
        if (h->p.dims[i] != 1) return REF_ERR_CORRUPT;
    if (h->p.lorenzo_order < 1) return REF_ERR_CORRUPT; /* written as 1..3 */
    if (h->nc != nchunks(n, h->p.chunk)) return REF_ERR_CORRUPT;
    if (!(h->sc[0] > 0.0f) || !isfinite(h->sc[0]) || h->sc[1] != h->sc[0] * 2.0f ||
        !isfinite(h->sc[1]))
        return REF_ERR_CORRUPT;
    if (h->m > n || h->e > h->m || h->maxlen < 1 || h->maxlen > A_MAXLEN) return REF_ERR_CORRUPT;
    if (h->w > h->nc + (A_MAXLEN * n + 31) / 32) return REF_ERR_CORRUPT;
    h->off_len = A_HEADER;
    h->off_bits = align16(h->off_len + 2ull * h->p.radius);
    h->na = anchored(&h->p) ? h->nc : 0;
    h->off_anc = align16(h->off_bits + 4 * h->nc);
    h->off_out = align16(h->off_anc + 4 * h->na);
    h->off_exc = h->off_out + 8 * h->m;
    h->off_str = align16(h->off_exc + 8 * h->e);
    if (h->total != h->off_str + 4 * h->w || h->total > bytes) return REF_ERR_CORRUPT;
    return REF_OK;
}

int gbsz_ref_archive_info(const void *archive, size_t bytes,
                          gbsz_ref_params *p, uint64_t *n)
{
    hdr_t h;
    int st = parse_header((const uint8_t *)archive, bytes, &h);
    if (st) return st;
    if (p) *p = h.p;
    if (n) *n = h.n;
    return REF_OK;
}

int gbsz_ref_decompress(const void *archive, size_t bytes, float *x,
                        uint64_t capacity_elems)
{
    hdr_t h;
    const uint8_t *a = (const uint8_t *)archive;
    int st = parse_header(a, bytes, &h);
    if (st) return st;
    if (h.n > capacity_elems) return REF_ERR_CAPACITY;
    const uint32_t nbins = 2 * h.p.radius;
    const uint8_t *len = a + h.off_len;
    uint32_t mx = 0;
    for (uint32_t s = 0; s < nbins; s++) mx = len[s] > mx ? len[s] : mx;
    if (mx != h.maxlen) return REF_ERR_CORRUPT;
    uint32_t *bits = (uint32_t *)malloc(h.nc * 4 + 4);
    uint32_t *stream = (uint32_t *)malloc(h.w * 4 + 4);
    uint32_t *oidx = (uint32_t *)malloc(h.m * 4 + 4);
    int32_t *odel = (int32_t *)malloc(h.m * 4 + 4);
    uint32_t *eidx = (uint32_t *)malloc(h.e * 4 + 4);
    uint32_t *eraw = (uint32_t *)malloc(h.e * 4 + 4);
    uint16_t *codes = (uint16_t *)malloc(h.n * 2 + 2);
    uint32_t *anc = (uint32_t *)malloc(h.na * 4 + 4);
    if (!bits || !stream || !oidx || !odel || !eidx || !eraw || !codes || !anc) {
        st = REF_ERR_OOM;
        goto done;
    }
    {
        uint64_t wsum = 0;
        for (uint64_t c = 0; c < h.nc; c++) {
            bits[c] = get_u32(a, h.off_bits + 4 * c);
            wsum += (bits[c] + 31u) / 32u;
        }
        if (wsum != h.w) { st = REF_ERR_CORRUPT; goto done; }
    }
#pragma omp parallel for
    for (int64_t t = 0; t < (int64_t)h.w; t++) stream[t] = get_u32(a, h.off_str + 4 * t);
    {
        int bad = 0; /* outlier indices: in range and strictly ascending */
#pragma omp parallel for reduction(| : bad)
        for (int64_t t = 0; t < (int64_t)h.m; t++) {
            oidx[t] = get_u32(a, h.off_out + 8 * t);
            odel[t] = (int32_t)get_u32(a, h.off_out + 8 * t + 4);
            if (oidx[t] >= h.n || (t > 0 && oidx[t] <= get_u32(a, h.off_out + 8 * (t - 1)))) bad = 1;
        }
        if (bad) { st = REF_ERR_CORRUPT; goto done; }
    }
    for (uint64_t t = 0; t < h.e; t++) {
        eidx[t] = get_u32(a, h.off_exc + 8 * t);
        eraw[t] = get_u32(a, h.off_exc + 8 * t + 4);
    }
    for (uint64_t c = 0; c < h.na; c++) anc[c] = get_u32(a, h.off_anc + 4 * c);
    st = gbsz_ref_inflate(stream, h.w, bits, h.n, h.p.chunk, len, nbins, codes);
    if (st) goto done;
    {
        uint64_t dims[3];
        const uint32_t gnd = lorenzo_geometry(&h.p, dims);
        st = reconstruct_anchored(codes, gnd, dims, h.p.radius, h.p.lorenzo_block, h.p.lorenzo_order, oidx,
                                  odel, h.m, eidx, eraw, h.e, h.sc[1], x, anc, h.na, h.p.chunk);
    }
done:
    free(bits); free(stream); free(oidx); free(odel); free(eidx); free(eraw); free(codes); free(anc);
    return st;
}
