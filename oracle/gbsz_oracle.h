/*
 * gbsz_oracle.h -- plain CPU oracle of the cuSZ dual-quantization + Huffman
 * path (Tian et al., "cuSZ: An Efficient GPU-Based Error-Bounded Lossy
 * Compression Framework for Scientific Data", PACT 2020).
 *
 * TEST INFRASTRUCTURE ONLY.  This library exists so that tests, the smoke
 * check and the CPU-baseline leg of the benchmark can check the CUDA library
 * against an independent, slow, obviously correct restatement of the paper.
 * The product path never links, loads or calls it.  It shares no code, header
 * or constant with the CUDA library: the archive layout below is written out
 * here a second time on purpose.
 *
 * Every function takes HOST pointers.  Return value 0 = success; otherwise one
 * of the REF_ERR_* codes.  Numeric values of the status codes equal the CUDA
 * library's so the tests can compare them, but they are defined here anew.
 */
#ifndef GBSZ_ORACLE_H
#define GBSZ_ORACLE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    REF_OK = 0,
    REF_ERR_INVALID_ARG = 1,
    REF_ERR_CAPACITY = 2,
    REF_ERR_CORRUPT = 3,
    REF_ERR_OOM = 4
};

enum { REF_EB_ABS = 0, REF_EB_REL = 1 };

typedef struct {
    uint32_t ndim;    /* 1, 2, 3, or 4 (predicted as 3D over dims[0],
                         dims[1] and dims[2]*dims[3]: the two slowest extents
                         folded into one) */
    uint64_t dims[4]; /* dims[0] varies fastest; unused dims are 1 */
    double eb;        /* absolute bound, or value-range-relative bound */
    uint32_t eb_mode; /* REF_EB_ABS or REF_EB_REL */
    uint32_t radius;  /* R: in-cap residuals satisfy |delta| < R; 2R bins */
    uint32_t chunk;   /* Huffman chunk in symbols, power of two 64..65536 */
    uint32_t lorenzo_block; /* 0: one predictor over the whole field; 1: the
                               paper's blocks (Sec. 3.1.1, 32 / 16x16 / 8x8x8)
                               with a zero padding layer around each block */
    uint32_t lorenzo_order; /* n of the Lorenzo predictor with binomial
                               coefficients (Sec. 3.1.2): 0 or 1 = first
                               order, 2, 3; orders above 1 need
                               lorenzo_block = 0 */
} gbsz_ref_params;

/* Block extent of the per-block Lorenzo mode along every dimension
 * (Sec. 3.1.1, "Chunking and Padding"): 32 in 1D, 16 in 2D, 8 in 3D. */
uint32_t gbsz_ref_lorenzo_block_extent(uint32_t ndim);

/* Threads the parallel loops use: omp_get_max_threads() in the OpenMP
 * build, 1 in the single-threaded one. */
int gbsz_ref_threads(void);

/* S0 -- error bound scalars (value-range-relative bound, footnote of Sec.
 * 3.2.2).  out[0] = eb, out[1] = 2*eb, out[2] = 1/(2*eb), all FP32. */
int gbsz_ref_error_bound(const float *x, uint64_t n, uint32_t eb_mode,
                         double eb, float out[3]);

/* S1 -- prequantization of one value (Sec. 3.1.2, Eq. for D-circle) with the
 * watchdog of Algorithm 1.  Returns 1 if the value becomes a verbatim
 * exception, 0 otherwise; *q receives the integer. */
int gbsz_ref_prequant_one(float x, const float sc[3], int32_t *q);

/* S2 -- Lorenzo residual delta = q - l(q) of order `order` (Sec. 3.1.2,
 * "Lorenzo Predictor with Binomial Coefficients"), zero outside the field,
 * arithmetic modulo 2^32. */
int gbsz_ref_lorenzo_delta(const int32_t *q, uint32_t ndim,
                           const uint64_t dims[3], uint32_t order,
                           int32_t *delta);

/* The same inside the paper's blocks when lblock = 1: a neighbour outside the
 * point's block counts as zero (the zero padding layer of Sec. 3.1.1). */
int gbsz_ref_lorenzo_delta_blocked(const int32_t *q, uint32_t ndim,
                                   const uint64_t dims[3], uint32_t order,
                                   uint32_t lblock, int32_t *delta);

/* S1+S2 -- dual-quantization of a whole field (Algorithm 2, compression
 * loop).  codes[n]; outliers (idx, delta) and exceptions (idx, raw bits) in
 * ascending idx.  Capacities are in entries; *m and *e get the counts.  q may
 * be NULL; if not, it receives the prequantized integers. */
int gbsz_ref_dualquant(const float *x, uint32_t ndim, const uint64_t dims[3],
                       const float sc[3], uint32_t radius, uint16_t *codes,
                       uint32_t *out_idx, int32_t *out_delta, uint64_t *m,
                       uint32_t *exc_idx, uint32_t *exc_raw, uint64_t *e,
                       int32_t *q);
/* The same with the per-block mode (lblock = 1) and a Lorenzo predictor of
 * order `order` (1..3; above 1 only with lblock = 0). */
int gbsz_ref_dualquant_ex(const float *x, uint32_t ndim,
                          const uint64_t dims[3], const float sc[3],
                          uint32_t radius, uint32_t lblock, uint32_t order,
                          uint16_t *codes, uint32_t *out_idx,
                          int32_t *out_delta, uint64_t *m,
                          uint32_t *exc_idx, uint32_t *exc_raw,
                          uint64_t *e, int32_t *q);

/* S3 -- histogram of quant codes (Sec. 3.2.1). */
int gbsz_ref_histogram(const uint16_t *codes, uint64_t n, uint32_t nbins,
                       uint32_t *hist);

/* S4a -- Huffman code lengths by the two-queue construction with the
 * (frequency, symbol) tie rule (Sec. 3.2.2).  len[nbins]; *maxlen. */
int gbsz_ref_huffman_lengths(const uint32_t *hist, uint32_t nbins,
                             uint8_t *len, uint32_t *maxlen);

/* S4b -- canonical codewords from lengths (Sec. 3.2.3). code[nbins]. */
int gbsz_ref_canonical_codes(const uint8_t *len, uint32_t nbins,
                             uint64_t *code);

/* S5 -- chunked encode + deflate (Sec. 3.2.4).  bits[nchunk]; stream words
 * are written MSB-first, each chunk starting on a word.  *words = total. */
int gbsz_ref_deflate(const uint16_t *codes, uint64_t n, uint32_t chunk,
                     const uint8_t *len, const uint64_t *code,
                     uint32_t *bits, uint32_t *stream, uint64_t stream_cap,
                     uint64_t *words);

/* S7 -- inflate (Sec. 3.3): canonical decode of every chunk. */
int gbsz_ref_inflate(const uint32_t *stream, uint64_t words,
                     const uint32_t *bits, uint64_t n, uint32_t chunk,
                     const uint8_t *len, uint32_t nbins, uint16_t *codes);

/* S8 -- reversed dual-quantization (Algorithm 2, decompression loop): every
 * point is predicted from the already reconstructed points before it. */
int gbsz_ref_reconstruct(const uint16_t *codes, uint32_t ndim,
                         const uint64_t dims[3], uint32_t radius,
                         const uint32_t *out_idx, const int32_t *out_delta,
                         uint64_t m, const uint32_t *exc_idx,
                         const uint32_t *exc_raw, uint64_t e, float ebx2,
                         float *xr);
int gbsz_ref_reconstruct_ex(const uint16_t *codes, uint32_t ndim,
                            const uint64_t dims[3], uint32_t radius,
                            uint32_t lblock, uint32_t order,
                            const uint32_t *out_idx,
                            const int32_t *out_delta, uint64_t m,
                            const uint32_t *exc_idx,
                            const uint32_t *exc_raw, uint64_t e,
                            float ebx2, float *xr);

/* Whole path: archive bytes and back.  Archive version 2: a 128-byte header,
 * then 16-byte aligned sections len[2R] (u8), bits[nchunk] (u32), anchors
 * (u32, nchunk entries for 1D fields with one order-1 predictor and chunks of
 * at least 1024 symbols, else none: anchor[c] is the prequantized integer of
 * the point before chunk c, 0 for c = 0), outliers[M] {u32 idx, i32 delta},
 * exceptions[E] {u32 idx, u32 raw}, stream[W] (u32).  Decompression checks
 * every anchor against the reconstructed integers (a mismatch is
 * REF_ERR_CORRUPT). */
size_t gbsz_ref_compress_bound(const gbsz_ref_params *p);
int gbsz_ref_compress(const float *x, const gbsz_ref_params *p, void *archive,
                      size_t capacity, size_t *out_bytes);
int gbsz_ref_decompress(const void *archive, size_t bytes, float *x,
                        uint64_t capacity_elems);
int gbsz_ref_archive_info(const void *archive, size_t bytes,
                          gbsz_ref_params *p, uint64_t *n);

#ifdef __cplusplus
}
#endif
#endif
