/*
 * gbsz.h -- C ABI of the GB300 (sm_103a) error-bounded lossy compressor for
 * FP32 fields that implements the dual-quantization + Huffman path of cuSZ
 * (Tian et al., PACT 2020, arXiv 2007.09625).
 *
 * Pipeline (paper section in brackets):
 *   compress   : error bound from the value range [Sec. 3.2.2 footnote]
 *                -> prequant + Lorenzo + postquant, outliers [Sec. 3.1, Alg. 2]
 *                -> histogram [Sec. 3.2.1] -> Huffman lengths and canonical
 *                codebook [Sec. 3.2.2-3.2.3] -> chunked encode + deflate
 *                [Sec. 3.2.4] -> archive bytes
 *   decompress : inflate [Sec. 3.3] -> reversed dual-quantization as a
 *                d-dimensional integer prefix sum [Alg. 2, Sec. 3.3]
 *
 * Archive (version 2, little-endian): a 128-byte header, then 16-byte
 * aligned sections -- code lengths (u8 per bin), bits per chunk (u32),
 * chunk anchors, outliers {u32 index, i32 residual}, exceptions {u32 index,
 * u32 raw float bits}, the bitstream (u32 words).  The anchors (this
 * format's own section; the paper has none) exist for 1D fields with one
 * order-1 predictor in chunks of at least 1024 symbols: one u32 per chunk,
 * the prequantized integer of the point before it (0 for the first), which
 * lets the decoder rebuild each chunk on its own.  Decompression checks
 * every anchor against the integers it reconstructs.
 *
 * Conventions shared by every entry point:
 *   - Pointers named d_* are CUDA device pointers on the context's device;
 *     h_* are host pointers.  The caller owns every buffer it passes; the
 *     library never frees, keeps or aliases them beyond the call (stream-
 *     ordered work on them may still be pending when an async call returns).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *   - Fields are FP32, row-major with dims[0] varying fastest.
 *   - Errors are return codes; no call aborts the process or throws.  Device
 *     side errors (corrupt archive, exhausted capacity, bounded waits that
 *     ran out) are recorded in a device status word and reported by the call
 *     that synchronises.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef GBSZ_H
#define GBSZ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbsz_ctx gbsz_ctx;

typedef enum {
    GBSZ_OK = 0,
    GBSZ_ERR_INVALID_ARG = 1, /* bad pointer, size, dims, eb, radius or chunk */
    GBSZ_ERR_CAPACITY = 2,    /* output buffer too small; needed size reported */
    GBSZ_ERR_CORRUPT = 3,     /* archive fails a consistency check */
    GBSZ_ERR_OOM = 4,         /* device or pinned allocation failed */
    GBSZ_ERR_CUDA = 5,        /* a CUDA runtime call failed */
    GBSZ_ERR_TIMEOUT = 6,     /* a bounded device wait ran out (a look-back of the warp decoder
                                 or of a scan waited more than 1 s) */
    GBSZ_ERR_UNSUPPORTED = 7, /* device is not sm_103 or feature absent */
    GBSZ_ERR_BOUNDS = 8       /* bounds-checking build only (-DGBSZ_BOUNDS_CHECK): a kernel's
                                 index check failed and the access was skipped */
} gbsz_status;

typedef enum { GBSZ_EB_ABS = 0, GBSZ_EB_REL = 1 } gbsz_eb_mode;

/* Compression parameters.
 *   ndim     1, 2, 3 (Lorenzo predictor dimensionality, Sec. 3.1.2) or 4:
 *            a 4D field (the QMCPACK shape of Sec. 4) is predicted as 3D
 *            over dims[0], dims[1] and dims[2]*dims[3]
 *   dims     extents, dims[0] fastest; entries >= ndim must be 1;
 *            product n in [1, 2^32)
 *   eb       error bound: absolute (GBSZ_EB_ABS) or relative to the value
 *            range max-min over finite values (GBSZ_EB_REL, the paper's
 *            "valrel"); every reconstructed value satisfies |d - d'| <= eb
 *            as FP32 eb, non-finite values are kept verbatim
 *   radius   R in [2, 32768]: residuals with |delta| < R get code delta+R,
 *            others are outliers with code 0; 2R Huffman symbols
 *            (Sec. 3.1.2 "cap"; 512 = the paper's 1024 bins)
 *   chunk    Huffman chunk in symbols, power of two in [64, 65536]
 *            (Sec. 3.2.4); 0 = choose automatically from n
 *   lorenzo_block  0: one Lorenzo predictor over the whole field (values
 *            outside the field are 0); 1: the paper's blocks (Sec. 3.1.1,
 *            "Chunking and Padding": 32 in 1D, 16x16 in 2D, 8x8x8 in 3D),
 *            each surrounded by a padding layer of zeros, so every block is
 *            predicted and reconstructed on its own.  Stored in the archive.
 *   lorenzo_order  n of the Lorenzo predictor with binomial coefficients
 *            (Sec. 3.1.2): 0 or 1 = first order (the default), 2 or 3; the
 *            residual is then the n-th difference along every dimension.
 *            Orders above 1 need lorenzo_block = 0.  Stored in the archive
 *            (as 1..3). */
typedef struct {
    uint32_t ndim;
    uint64_t dims[4];
    double eb;
    uint32_t eb_mode;
    uint32_t radius;
    uint32_t chunk;
    uint32_t lorenzo_block;
    uint32_t lorenzo_order;
} gbsz_params;

/* Creates a context on CUDA device `device` (must be compute capability
 * 10.3, GB300).  The context owns device scratch (grown on demand and kept
 * across calls), pinned staging and CUDA events.
 * Errors: INVALID_ARG (out NULL), UNSUPPORTED (wrong device), CUDA, OOM. */
gbsz_status gbsz_create(gbsz_ctx **out, int device);

/* Frees everything the context owns.  Waits for its pending work.  NULL ok. */
void gbsz_destroy(gbsz_ctx *ctx);

/* Context options: knobs of the kernels that never change archive bytes.
 *   GBSZ_OPT_CODEWORD_BITS  width of the (bitwidth, codeword) table entries
 *     the encoder reads.  0 (default) = the paper's adaptive choice (Sec.
 *     3.2.2): 32-bit entries when the longest code has at most 24 bits, else
 *     64; 64 = always 64-bit entries (the "enc.64" column of the paper's
 *     encode/deflate table, for comparison).
 * Errors: INVALID_ARG (NULL context, unknown option or value). */
#define GBSZ_OPT_CODEWORD_BITS 1
/*   GBSZ_OPT_BATCH_MODE  how gbsz_compress_batch and gbsz_decompress_batch
 *     run a batch: 0 (default) = one launch per stage (per kernel variant)
 *     for all fields, each field owning a range of the grid's blocks (its
 *     tiles, units or chunks), when the batch has at least two fields, all
 *     of Lorenzo order 1, averaging at most 2^21 points; otherwise every
 *     field's own launches on up to 8 slot streams; 1 = always the slot
 *     streams (for comparison).  The results are the same bytes either
 *     way. */
#define GBSZ_OPT_BATCH_MODE 3
/*   GBSZ_OPT_DECODER  which Huffman decoder (S7) runs.  Thread: one thread
 *     walks each chunk.  Warp: the 32 lanes of a warp decode 32 ranges of a
 *     chunk's bits and re-synchronise; for 1D fields of order-1 whole-field
 *     Lorenzo under 2^30 points it also reconstructs the values (S8) in the
 *     same kernel.  Chunks of more than 4096 symbols always take the thread
 *     decoder, and so do 1D order-1 fields of 2^30 points or more.
 *     With an anchored 1D archive (see the archive format above) whose codes
 *     fit the complete table (at most 15 bits), the thread decoder writes
 *     the values itself, each chunk from its anchor.
 *     0 (default) = warp for fields of at most 32 chunks per SM in chunks
 *     of at least 1024 symbols, else thread; 1 = thread always; 2 = warp
 *     wherever it applies; 3 = thread always, writing the codes for a
 *     separate reconstruction pass even where the anchors allow the fused
 *     one.  The results and statuses are the same either way. */
#define GBSZ_OPT_DECODER 4
/*   GBSZ_OPT_LORENZO_SLAB  extent of a dual-quant tile along its swept
 *     dimension (S1+S2, Sec. 3.1): rows for 2D fields (tiles of 512 x slab
 *     points), planes for 3D (tiles of 32 x 32 x slab).  0 (default) = the
 *     autotuner's choice for the field's key, else the built-in rule (8 rows;
 *     planes halved from the full depth until there are 8 tiles per SM or 4
 *     planes); 1..65536 = that extent.  The archive is the same either way
 *     (the tile boundaries only decide which threads compute which points). */
#define GBSZ_OPT_LORENZO_SLAB 5
/*   GBSZ_OPT_TEST_HOLD_CHUNK  test hook for the warp decoder's bounded wait:
 *     -1 (default) = off; k >= 0 = chunk k never publishes its look-back
 *     word, so the next chunk's wait runs out (after 1 s) and a fused 1D
 *     decompress returns GBSZ_ERR_TIMEOUT; the context stays usable.  No
 *     effect on the other decoders. */
#define GBSZ_OPT_TEST_HOLD_CHUNK 6
gbsz_status gbsz_set_option(gbsz_ctx *ctx, int option, int64_t value);

/* Worst-case archive size in bytes for these parameters (0 if invalid).
 * Host-only, no device work. */
size_t gbsz_compress_bound(const gbsz_params *p);

/* Chunk size that chunk = 0 resolves to for these parameters (a fixed rule
 * of n: the smallest power of two in 64..4096 whose chunks fit in one wave of
 * 1024 decoding threads per SM on a 152-SM GB300). */
uint32_t gbsz_auto_chunk(const gbsz_params *p);

/* Measured choice of the Huffman chunk (Sec. 3.2.4; the paper tunes it by
 * hand, Sec. 4.2) and of two knobs that leave the bytes alone.  On `stream`
 * (CUDA events, best of two runs after a warm-up each):
 *   1. compress + decompress of the field at d_field for chunk sizes
 *      256..4096 and the rule's choice; *out = *p with the fastest chunk;
 *   2. at that chunk (if at most 4096), decompress with the thread-per-chunk
 *      and the warp-per-chunk decoders (GBSZ_OPT_DECODER 1 and 2);
 *   3. for 2D and 3D fields of Lorenzo order 1, compress with dual-quant
 *      tiles of 4..64 rows / planes and the built-in rule
 *      (GBSZ_OPT_LORENZO_SLAB).
 * The choices are remembered per context for the key (ndim, dims, radius,
 * lorenzo_block, lorenzo_order): later calls with the same key return the
 * chunk without measuring, so every single or batched call given *out
 * produces the same archive, and calls on fields of the key use the tuned
 * decoder (for archives of the tuned chunk) and tile extent while the
 * context's options for them are 0.  *ms (may be NULL) gets the measured
 * compress + decompress time of the chosen chunk (0 when remembered).
 * Allocates scratch for one archive and one field.  Errors: INVALID_ARG,
 * OOM, CUDA, and any error of the compress/decompress calls it makes. */
gbsz_status gbsz_autotune(gbsz_ctx *ctx, const float *d_field, const gbsz_params *p,
                          gbsz_params *out, float *ms, void *stream);

/* What gbsz_autotune chose for the key of *p: knobs[0] = chunk, knobs[1] =
 * decoder (1 thread, 2 warp per chunk; 0 = not measured: chunk above 4096),
 * knobs[2] = dual-quant tile extent (0 = the built-in rule).  Host-only.
 * Errors: INVALID_ARG (NULL argument, or no choice remembered for the key). */
gbsz_status gbsz_tuned_knobs(gbsz_ctx *ctx, const gbsz_params *p, uint32_t knobs[3]);

/* Compresses n = prod(dims) floats at d_field into the archive at d_archive
 * (device memory, 16-byte aligned, `capacity` bytes).  Stages: S0 error
 * bound, S1-S3 dual-quant + histogram, S4 codebook, S5 encode/deflate and
 * archive assembly, all as sm_103a kernels on `stream`.  Synchronises the
 * stream once to return the archive size in *out_bytes (host).
 * Errors: INVALID_ARG, CAPACITY (*out_bytes = bytes needed; archive
 * contents unspecified), OOM, CUDA, TIMEOUT. */
gbsz_status gbsz_compress(gbsz_ctx *ctx, const float *d_field,
                          const gbsz_params *p, void *d_archive,
                          size_t capacity, size_t *out_bytes, void *stream);

/* Decompresses the archive at d_archive (`bytes` bytes, device memory,
 * 16-byte aligned) into d_field (room for capacity_elems floats, 16-byte
 * aligned).  Stages: S7 decode, S8 outlier scatter + prefix-sum
 * reconstruction + exception patch (for anchored 1D archives S8 runs inside
 * the decoder: each chunk from its anchor).  Reads the 128-byte header to the host
 * first and synchronises at the end to report device-side checks.
 * Errors: INVALID_ARG, CORRUPT, CAPACITY (field larger than capacity),
 * OOM, CUDA, TIMEOUT. */
gbsz_status gbsz_decompress(gbsz_ctx *ctx, const void *d_archive, size_t bytes,
                            float *d_field, uint64_t capacity_elems,
                            void *stream);

/* Batched compression of `count` independent fields (host arrays of
 * length count: device pointers, parameters, capacities; outputs out_bytes
 * and per-field statuses).  The fields' stages are spread over up to eight
 * internal streams forked from `stream` and joined back into it, so small
 * fields' kernels overlap on the GPU; the call synchronises once at the end.
 * Every archive is byte-identical to what gbsz_compress gives for that field
 * alone.  Returns GBSZ_OK if every field succeeded, else the first field's
 * error (see statuses[]).  This is the batching the paper's block-by-block
 * processing of many fields (Sec. 4.1) calls for, done concurrently. */
gbsz_status gbsz_compress_batch(gbsz_ctx *ctx, uint32_t count,
                                const float *const *d_fields,
                                const gbsz_params *params,
                                void *const *d_archives,
                                const size_t *capacities, size_t *out_bytes,
                                gbsz_status *statuses, void *stream);

/* Batched decompression; the counterpart of gbsz_compress_batch.  Reads all
 * headers to the host with one synchronisation, then decodes every field
 * concurrently as above.  Per-field statuses as for gbsz_decompress. */
gbsz_status gbsz_decompress_batch(gbsz_ctx *ctx, uint32_t count,
                                  const void *const *d_archives,
                                  const size_t *bytes, float *const *d_fields,
                                  const uint64_t *capacities,
                                  gbsz_status *statuses, void *stream);

/* Host-buffer variants: the field (or archive) is copied from host memory to
 * context-owned device staging, processed, and the result copied back to
 * host memory, all inside the call (pinned host buffers copy fastest).
 * Same errors as the device variants. */
gbsz_status gbsz_compress_host(gbsz_ctx *ctx, const float *h_field,
                               const gbsz_params *p, void *h_archive,
                               size_t capacity, size_t *out_bytes,
                               void *stream);
gbsz_status gbsz_decompress_host(gbsz_ctx *ctx, const void *h_archive,
                                 size_t bytes, float *h_field,
                                 uint64_t capacity_elems, void *stream);

/* Asynchronous form of gbsz_decompress_host, for pipelines that upload the
 * next field while this one downloads: parses the header from h_archive,
 * enqueues the archive upload, the decompression and the field download on
 * `stream`, and returns without waiting.  The call uses scratch of its own,
 * so other calls on the context may run meanwhile (on other streams); one
 * asynchronous call may be pending per context.  h_archive and h_field must
 * stay valid and unmodified until gbsz_async_wait returns.  Pinned host
 * buffers are needed for the copies to overlap other work.
 * Errors at the call: INVALID_ARG (NULL, or a call already pending),
 * CORRUPT (header), CAPACITY, OOM, CUDA.  Device-side checks are reported
 * by gbsz_async_wait. */
gbsz_status gbsz_decompress_host_async(gbsz_ctx *ctx, const void *h_archive,
                                       size_t bytes, float *h_field,
                                       uint64_t capacity_elems, void *stream);

/* Waits for the pending asynchronous call, if any, and returns its status
 * (GBSZ_OK when nothing is pending): CORRUPT, CUDA or TIMEOUT as for
 * gbsz_decompress. */
gbsz_status gbsz_async_wait(gbsz_ctx *ctx);

/* Serving loop (continuous batching).  A server owns `workers` threads, each
 * with its own context and stream.  Submitted requests wait in a FIFO queue;
 * a free worker takes the oldest requests, at most `max_batch`, and runs them
 * with gbsz_compress_batch / gbsz_decompress_batch, so batches of different
 * workers overlap on the GPU.  `mem_budget` bounds the device memory the
 * workers' contexts hold (gbsz_memory_usage), idle or busy: a batch is
 * admitted only if an upper bound of its worker's memory after it
 * (gbsz_scratch_bytes of every request plus any new slot) keeps the sum over
 * workers within the budget; after the batch the worker's measured memory
 * is counted; a worker that cannot admit the oldest request releases its
 * scratch first (gbsz_release_scratch).  The caller's fields and archives are
 * not counted.  Every result is the same bytes as the single-field call's.
 * The paper has no serving layer; this is the batching its block-wise design
 * allows, for many independent fields.
 *   gbsz_server_create   workers in [1, 64], max_batch in [1, 1024],
 *                        mem_budget > 0.  Errors: INVALID_ARG, OOM, and the
 *                        errors of gbsz_create.
 *   gbsz_server_destroy  runs every queued request, then frees the server.
 *   gbsz_server_submit_* queue one request and return its ticket (> 0).  The
 *                        device buffers belong to the caller and must stay
 *                        valid until the request is done; the input must be
 *                        complete on the device when submitted (a
 *                        decompress reads the archive's 128-byte header at
 *                        submission, synchronously).  Errors: INVALID_ARG,
 *                        CORRUPT (header), CAPACITY (the request alone needs
 *                        more than mem_budget; it is not queued).
 *   gbsz_server_poll     *done = 1 and *status / *out_bytes (archive bytes for
 *                        a compress, field bytes for a decompress) once the
 *                        request is done; the ticket is then released.
 *                        INVALID_ARG for an unknown or released ticket.
 *   gbsz_server_wait     the same, waiting up to timeout_s seconds (< 0: no
 *                        limit); TIMEOUT if still pending.
 *   gbsz_server_stats    out6 = {completed requests, p50 latency ms, p99
 *                        latency ms, mean batch size, input GB/s over the
 *                        span, span s from first arrival to last completion}.
 */
typedef struct gbsz_server gbsz_server;
gbsz_status gbsz_server_create(gbsz_server **out, int device, uint32_t workers,
                               uint32_t max_batch, uint64_t mem_budget);
void gbsz_server_destroy(gbsz_server *s);
gbsz_status gbsz_server_submit_compress(gbsz_server *s, const float *d_field,
                                        const gbsz_params *p, void *d_archive,
                                        size_t capacity, uint64_t *ticket);
gbsz_status gbsz_server_submit_decompress(gbsz_server *s,
                                          const void *d_archive, size_t bytes,
                                          float *d_field,
                                          uint64_t capacity_elems,
                                          uint64_t *ticket);
gbsz_status gbsz_server_poll(gbsz_server *s, uint64_t ticket, int *done,
                             gbsz_status *status, size_t *out_bytes);
gbsz_status gbsz_server_wait(gbsz_server *s, uint64_t ticket,
                             double timeout_s, gbsz_status *status,
                             size_t *out_bytes);
gbsz_status gbsz_server_stats(gbsz_server *s, double *out6);
/* out4 = {device bytes counted against the budget now, their peak, scratch
 * releases to admit requests, batches after which a worker held more than
 * its bound (0 unless the bound is wrong)}.  Errors: INVALID_ARG. */
gbsz_status gbsz_server_memory(gbsz_server *s, uint64_t *out4);

/* Device memory of a context.  The paper has no counterpart: these serve
 * callers that budget device memory (the serving loop above).
 *   gbsz_memory_usage     *device_bytes = bytes of device memory the context
 *                         holds now (every slot's scratch and tables, staging
 *                         of the host-buffer calls); *slots (may be NULL) =
 *                         its scratch slots (1 .. 8).  Host-only.
 *   gbsz_release_scratch  waits for the device, then frees every slot's
 *                         scratch sized by field, every slot but the first,
 *                         and all staging; drops captured graphs.  The next
 *                         call reallocates what it needs.  INVALID_ARG while
 *                         an asynchronous host decompress is pending.
 *   gbsz_scratch_bytes    *field_bytes = scratch one field with parameters p
 *                         adds to a slot (for_decompress: p as the archive
 *                         states it); *slot_bytes = the fixed tables of one
 *                         slot.  Host-only.  Either pointer may be NULL.
 * Errors: INVALID_ARG (NULL context or invalid p), CUDA. */
gbsz_status gbsz_memory_usage(gbsz_ctx *ctx, uint64_t *device_bytes,
                              uint32_t *slots);
gbsz_status gbsz_release_scratch(gbsz_ctx *ctx);
gbsz_status gbsz_scratch_bytes(const gbsz_params *p, int for_decompress,
                               uint64_t *field_bytes, uint64_t *slot_bytes);

/* Parses a host copy of an archive header (at least 128 bytes; `bytes` is
 * the archive's full size, used for the size check).  Fills *out and *n.
 * Host-only.  Errors: INVALID_ARG (NULL), CORRUPT. */
gbsz_status gbsz_archive_info(const void *h_archive, size_t bytes,
                              gbsz_params *out, uint64_t *n);

/* Static description of a status code. */
const char *gbsz_status_str(gbsz_status s);

/* Copies an internal buffer of the last compress/decompress on this context
 * to host memory, for stage-by-stage checks.  `which`:
 *   0 quant codes of the last compress (uint16[n])
 *   1 histogram of the last compress (uint32[2R])
 *   2 error-bound scalars of the last compress (float[3]: eb, 2eb, 1/(2eb))
 *   3 quant codes decoded by the last decompress (uint16[n]; INVALID_ARG
 *     when it took the fused 1D decoder, whose codes never leave the chip)
 *   4 canonical codewords of the last compress (uint64[2R]: code, no length)
 *   5 batch graph counters (uint64[4]: compress captures, compress replays,
 *     decompress captures, decompress replays)
 *   6 the same for single-field calls (gbsz_compress / gbsz_decompress
 *     repeated with the same buffers and parameters on a capturable stream
 *     are replayed as CUDA graphs)
 * `bytes` must equal the buffer's size.  Synchronises the context's last
 * stream.  Errors: INVALID_ARG, CUDA. */
gbsz_status gbsz_debug_copy(gbsz_ctx *ctx, int which, void *h_dst,
                            size_t bytes);

/* Stage timing.  While enabled, every compress/decompress records CUDA
 * events around each stage on its stream; calls replayed as CUDA graphs
 * record them through the graph's own event nodes, and the call collects
 * those times after it synchronises.  gbsz_profile_read synchronises,
 * adds up the stage durations recorded since the last read, and returns
 * them with the count of kernel launches.  Stage indices:
 *   0 error bound, 1 dual-quant+histogram, 2 codebook,
 *   3 encode: bit counts, 4 encode: offset scan, 5 encode: pack (deflate),
 *   6 decode tables, 7 decode: chunk offset scan, 8 decode: symbols,
 *   9 reconstruct (scatter+scan+patch), 10 other (reserved)
 * ms[nstage], calls[nstage] may be NULL.  Errors: INVALID_ARG, CUDA. */
#define GBSZ_NSTAGE 11
gbsz_status gbsz_profile_enable(gbsz_ctx *ctx, int enable);
gbsz_status gbsz_profile_read(gbsz_ctx *ctx, double *ms, uint64_t *calls,
                              uint64_t *kernel_launches);

/* Huffman codebook from a histogram without allocating device memory.  The
 * paper has no counterpart: it exists for callers that cannot call
 * cudaMalloc -- host frameworks that own all device memory through their
 * own pool and forbid driver allocations, and processes under a fixed
 * device-memory budget that a library allocating on its own could exceed.
 * It runs the compressor's codebook kernel (S4) with its scratch in a fixed
 * device array that the library defines (sized for 65536 symbols, about
 * 4 MB, held on every GPU that loads the library until exit).
 *   d_hist   device uint32[nbins] symbol frequencies (nbins in [1, 65536];
 *            at least one nonzero; their total below 2^32)
 *   d_len    device uint8[nbins] out: code lengths (0 = symbol absent)
 *   d_code   device uint64[nbins] out: canonical codewords, right-aligned
 *   maxlen   host out (may be NULL): longest code length
 * Runs on the current CUDA device; its first call on a device looks up the
 * array's device address, so make that first call before any stream
 * capture.  All calls share the array and it keeps the last call's contents:
 * calls whose work overlaps on the GPU race, so serialise them.  Synchronises
 * `stream` to report errors.  Allocates nothing (no cudaMalloc, cudaFree or
 * allocating library routine).
 * Errors: INVALID_ARG (bad sizes, NULL, all-zero histogram, total of the
 * frequencies >= 2^32), CUDA. */
gbsz_status gbsz_codebook_noalloc(const uint32_t *d_hist, uint32_t nbins,
                                  uint8_t *d_len, uint64_t *d_code,
                                  uint32_t *maxlen, void *stream);

#ifdef __cplusplus
}
#endif
#endif
