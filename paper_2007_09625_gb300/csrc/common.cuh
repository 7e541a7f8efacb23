// common.cuh -- definitions shared by the sm_103a kernels of the compressor.
//
// Archive format (version 2), little-endian, sections 16-byte aligned:
//   [0,128)          header (field offsets below)
//   len[2R]          Huffman code length per quant code (uint8)
//   bits[nchunk]     deflated bits per chunk (uint32)
//   anchors          1D fields with one order-1 predictor and chunks of at
//                    least kAnchorChunk symbols: nchunk uint32, the
//                    prequantized integer of the point before each chunk (0
//                    for the first), so each chunk can be rebuilt on its own;
//                    no entries otherwise
//   outliers[M]      {uint32 idx, int32 delta}, ascending idx
//   exceptions[E]    {uint32 idx, uint32 raw float bits}, ascending idx
//   stream[W]        uint32 words; each chunk starts on a word, MSB first
#pragma once

#include <cstdint>
#include <cuda_runtime.h>
#include <functional>
#include <vector>

namespace gbsz {

constexpr uint32_t kMagic = 0x5A534247u;  // "GBSZ"
constexpr uint16_t kVersion = 2;
constexpr uint32_t kAnchorChunk = 1024;  // smallest chunk whose 1D archives carry anchors
constexpr uint32_t kHeaderBytes = 128;
// Deepest possible Huffman leaf for n < 2^32 symbols: a leaf at depth d needs
// a total weight >= Fibonacci(d + 2), and Fibonacci(48) > 2^32.
constexpr uint32_t kMaxLen = 45;
constexpr uint32_t kMaxBins = 65536;

// header byte offsets
enum : uint32_t {
    H_MAGIC = 0, H_VERSION = 4, H_HDRBYTES = 6, H_NDIM = 8, H_EBMODE = 12,
    H_DIMS = 16, H_N = 40, H_EB = 48, H_EBF = 56, H_EBX2 = 60, H_INV2EB = 64,
    H_RADIUS = 68, H_CHUNK = 72, H_NCHUNK = 76, H_M = 80, H_E = 88, H_W = 96,
    H_MAXLEN = 104, H_LBLOCK = 108, H_TOTAL = 112, H_ORDER = 120, H_DIM3 = 124
};

__host__ __device__ inline uint64_t align16(uint64_t v) { return (v + 15) & ~uint64_t(15); }

struct Layout {
    uint64_t len, bits, anch, outl, exc, stream, total;
    uint64_t nanch;  // anchor entries (nchunk or 0)
};

// whether a field's archive carries chunk anchors (ndim as in the header; order 0 reads as 1)
__host__ __device__ inline bool anchored(uint32_t ndim, uint32_t order, uint32_t lblock, uint32_t chunk)
{
    return ndim == 1 && order <= 1 && lblock == 0 && chunk >= kAnchorChunk;
}

__host__ __device__ inline Layout make_layout(uint32_t radius, uint64_t nchunk, uint64_t m,
                                              uint64_t e, uint64_t w, bool anchors)
{
    Layout L;
    L.len = kHeaderBytes;
    L.bits = align16(L.len + 2ull * radius);
    L.anch = align16(L.bits + 4 * nchunk);
    L.nanch = anchors ? nchunk : 0;
    L.outl = align16(L.anch + 4 * L.nanch);
    L.exc = L.outl + 8 * m;
    L.stream = align16(L.exc + 8 * e);
    L.total = L.stream + 4 * w;
    return L;
}

// device status bits (Control::error)
enum : uint32_t {
    DERR_CAPACITY = 1u, DERR_CORRUPT = 2u, DERR_TIMEOUT = 4u, DERR_EB = 8u, DERR_INTERNAL = 16u,
    DERR_RANGE = 32u,  // an input outside what the kernel supports (codebook: histogram total >= 2^32)
    DERR_BOUNDS = 64u,  // bounds-checking build: an index check failed
    // decompress planned from the header its context kept from the compress
    // into the same buffer, and the archive's header is no longer that one
    // (the host runs the call again from the archive's own header)
    DERR_STALE = 128u
};

// Per-call device control block.  Zeroed by one memset at the start of each
// compress / decompress.
struct Control {
    uint32_t max_key;      // S0: max ordered key over finite values (0 = none)
    uint32_t min_key_inv;  // S0: max of ~key, i.e. the min (0 = none)
    uint32_t s0_done;      // S0: finished blocks
    uint32_t error;        // DERR_* bits
    float eb, ebx2, inv2eb;
    uint32_t maxlen;
    unsigned long long n_out;  // outliers (code 0), counted by the dual-quant kernel
    unsigned long long n_exc;  // verbatim exceptions
    uint32_t nsym;             // codebook: symbols with nonzero frequency
    unsigned long long words;  // encode: total stream words
    unsigned long long total;  // encode: archive bytes
    unsigned long long zeros;  // decode: code-0 symbols decoded
    unsigned long long out_chk; // encode: outliers emitted (check)
    unsigned long long exc_chk; // encode: exceptions emitted (check)
    uint32_t ticket;            // warp decoder: next chunk to take
};

// Bounds-checking build (compiled with -DGBSZ_BOUNDS_CHECK): GBSZ_CHECK(cond,
// ctl) guards an access at an index a kernel computed -- true when cond
// holds; otherwise it records DERR_BOUNDS in ctl and is false, and the caller
// skips the access.  In the normal build it is the constant true and cond is
// not evaluated.
#ifdef GBSZ_BOUNDS_CHECK
__device__ __forceinline__ bool bounds_hold(bool c, Control *ctl)
{
    if (!c) atomicOr(&ctl->error, DERR_BOUNDS);
    return c;
}
#define GBSZ_CHECK(cond, ctl) (::gbsz::bounds_hold((cond), (ctl)))
#else
#define GBSZ_CHECK(cond, ctl) true
#endif

struct EbScalars {
    float eb, ebx2, inv2eb;
};

// ---------------------------------------------------------------------------
// Prequantization (Sec. 3.1.2): d° = round(d / 2eb) as t = fl(d * 1/(2eb)),
// round half to even, accepted only if the value the decompressor rebuilds,
// fl(2eb * fl(q)), is within eb of d (the watchdog of Algorithm 1); else
// q +- 1; else the value is kept verbatim (exception).

__device__ __forceinline__ float recon_value(int32_t q, float ebx2)
{
    return __fmul_rn(ebx2, __int2float_rn(q));
}

// |d - r| <= eb, decided exactly.  The rounded difference decides unless it
// equals eb; then Knuth's TwoSum gives the exact residual of the subtraction.
__device__ __forceinline__ bool within_bound(float d, float r, float eb)
{
    const float s = __fsub_rn(d, r);
    const float a = fabsf(s);
    if (a < eb) return true;
    if (!(a == eb)) return false;
    const float nr = -r;
    const float bp = __fsub_rn(s, d);
    const float ap = __fsub_rn(s, bp);
    const float e = __fadd_rn(__fsub_rn(d, ap), __fsub_rn(nr, bp));
    return s > 0.0f ? e <= 0.0f : e >= 0.0f;
}

__device__ __forceinline__ int32_t prequant_full(float d, const EbScalars &s, bool &exc)
{
    if ((__float_as_uint(d) & 0x7F800000u) == 0x7F800000u) {  // NaN or Inf
        exc = true;
        return 0;
    }
    const float t = __fmul_rn(d, s.inv2eb);
    if (!(fabsf(t) < 1073741824.0f)) {
        exc = true;
        return t > 0.0f ? (1 << 30) : -(1 << 30);
    }
    const int32_t q = __float2int_rn(t);
    const float r = recon_value(q, s.ebx2);
    if (within_bound(d, r, s.eb)) {
        exc = false;
        return q;
    }
    const int32_t q2 = d > r ? q + 1 : q - 1;
    if (within_bound(d, recon_value(q2, s.ebx2), s.eb)) {
        exc = false;
        return q2;
    }
    exc = true;
    return q;
}

// Common case of prequant_full without int/float conversions: for |t| < 2^22,
// t + 1.5*2^23 lands in [2^23, 2^24) where floats are the integers, so the
// one rounding of that addition is round-half-even of t (1.5*2^23 is even);
// subtracting it back is exact, and the integer is the float's bit pattern
// minus that of 1.5*2^23 offset by 2^22.  Accepted only when the rounded
// |d - fl(2eb * q)| is strictly below eb (then the exact value is too);
// every other case (NaN, Inf, large |t|, near-ties) takes the full path,
// which gives the same q for the cases accepted here.
// The fast path alone: ok = false when it cannot decide (then the value must
// go through prequant_full).
__device__ __forceinline__ int32_t prequant_fast(float d, const EbScalars &s, bool &ok)
{
    const float t = __fmul_rn(d, s.inv2eb);
    const float tm = __fadd_rn(t, 12582912.0f);
    const float r = __fmul_rn(s.ebx2, __fsub_rn(tm, 12582912.0f));
    // one predicate for both tests (NaN and Inf fail the first)
    ok = (fabsf(t) < 4194304.0f) & (fabsf(__fsub_rn(d, r)) < s.eb);
    return __float_as_int(tm) - 0x4B400000;
}

__device__ __forceinline__ int32_t prequant(float d, const EbScalars &s, bool &exc)
{
    bool ok;
    const int32_t q = prequant_fast(d, s, ok);
    if (ok) {
        exc = false;
        return q;
    }
    return prequant_full(d, s, exc);
}

__device__ __forceinline__ EbScalars load_scalars(const Control *ctl)
{
    EbScalars s;
    s.eb = ctl->eb;
    s.ebx2 = ctl->ebx2;
    s.inv2eb = ctl->inv2eb;
    return s;
}

// code for residual delta (postquant, Algorithm 2): delta + R if in cap and
// not an exception, else 0 (outlier marker)
__device__ __forceinline__ uint32_t postquant(uint32_t delta, bool exc, int32_t R)
{
    const int32_t dl = (int32_t)delta;
    return (!exc && dl > -R && dl < R) ? (uint32_t)(dl + R) : 0u;
}

// ---------------------------------------------------------------------------
// small warp / block helpers

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

__device__ __forceinline__ unsigned long long warp_incl_scan64(unsigned long long v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// Block-wide exclusive scan of one uint32 per thread; `sh` needs
// blockDim.x/32 + 1 entries.  Returns the exclusive prefix; *total gets the
// block total.  Contains __syncthreads; all threads must call.
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *sh, uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? sh[lane] : 0;
        uint32_t wi = warp_incl_scan(w);
        if (lane < nw) sh[lane] = wi - w;
        if (lane == nw - 1) sh[nw] = wi;
    }
    __syncthreads();
    uint32_t r = sh[warp] + inc - v;
    *total = sh[nw];
    __syncthreads();
    return r;
}

// The same without the closing barrier: sh may be written again only after
// every thread has passed another barrier (callers alternate two arrays).
__device__ __forceinline__ uint32_t block_excl_scan_nb(uint32_t v, uint32_t *sh, uint32_t *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t inc = warp_incl_scan(v);
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? sh[lane] : 0;
        uint32_t wi = warp_incl_scan(w);
        if (lane < nw) sh[lane] = wi - w;
        if (lane == nw - 1) sh[nw] = wi;
    }
    __syncthreads();
    *total = sh[nw];
    return sh[warp] + inc - v;
}

__device__ __forceinline__ unsigned long long block_excl_scan64(unsigned long long v,
                                                                unsigned long long *sh,
                                                                unsigned long long *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned long long inc = warp_incl_scan64(v);
    if (lane == 31) sh[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        unsigned long long w = lane < nw ? sh[lane] : 0;
        unsigned long long wi = warp_incl_scan64(w);
        if (lane < nw) sh[lane] = wi - w;
        if (lane == nw - 1) sh[nw] = wi;
    }
    __syncthreads();
    unsigned long long r = sh[warp] + inc - v;
    *total = sh[nw];
    __syncthreads();
    return r;
}

__device__ __forceinline__ uint32_t block_max(uint32_t v, uint32_t *sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        uint32_t w = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) w = max(w, __shfl_xor_sync(0xffffffffu, w, o));
        if (lane == 0) sh[nw] = w;
    }
    __syncthreads();
    uint32_t r = sh[nw];
    __syncthreads();
    return r;
}


// ---------------------------------------------------------------------------
// Grouped launches.  A kernel body sees its block index and grid size
// through a VGrid, so the same body runs as a launch of its own or as one
// field's share of a grouped launch that covers many fields of a batch: item
// i owns the blocks [first[i], first[i+1]) of the grid and runs the body
// with blocks 0 .. first[i+1] - first[i] - 1 of its own virtual grid.
struct VGrid {
    uint32_t bid, nb;
};

__device__ __forceinline__ VGrid vgrid_self() { return VGrid{blockIdx.x, gridDim.x}; }

// The item that owns this block (all threads; contains a barrier).
__device__ __forceinline__ uint32_t group_item(const uint32_t *first, uint32_t nitems, VGrid &vg)
{
    __shared__ uint32_t s_item;
    if (threadIdx.x == 0) {
        uint32_t lo = 0, hi = nitems;  // first[lo] <= blockIdx.x < first[hi]
        while (hi - lo > 1) {
            const uint32_t m = (lo + hi) >> 1;
            if (first[m] <= blockIdx.x) lo = m;
            else hi = m;
        }
        s_item = lo;
    }
    __syncthreads();
    const uint32_t i = s_item;
    vg = VGrid{blockIdx.x - first[i], first[i + 1] - first[i]};
    return i;
}

// ---------------------------------------------------------------------------
// launch wrappers implemented in the kernel translation units

struct QuantArgs {
    const float *x;
    uint64_t dims[3];
    uint32_t ndim;
    uint32_t radius;
    uint16_t *codes;
    int2 *dscr;      // {residual, is exception} of every code-0 point, by point
    uint32_t *hist;  // 2R bins, zeroed by the caller
    uint32_t *unit_exc;   // exceptions per encoder unit (zeroed by the caller)
    uint32_t unit_shift;  // log2 of the encoder unit in points
    uint32_t lblock;      // 1: Lorenzo inside the paper's blocks (zero padding layer)
    uint32_t order;       // Lorenzo order n (1..3)
    int32_t *qint;        // order > 1: prequantized integers (scratch, n entries)
    uint32_t *excm;       // order > 1: exception bit per point (zeroed, n/32 + 1 words)
    Control *ctl;
    int num_sms;
    uint32_t slab;  // rows (2D) or planes (3D) each tile sweeps; 0 = the built-in rule
    // 1D fields whose archive carries chunk anchors: the archive's anchor
    // section (anchors[c] = prequantized integer of point c * chunk - 1,
    // anchors[0] = 0), else nullptr
    uint32_t *anchors;
    uint32_t chunk;
};
__host__ __device__ inline uint64_t npoints(const QuantArgs &a) { return a.dims[0] * a.dims[1] * a.dims[2]; }
// block extent of the per-block Lorenzo mode (Sec. 3.1.1): 32, 16x16, 8x8x8
__host__ __device__ constexpr uint32_t lorenzo_block_extent(uint32_t ndim)
{
    return ndim == 1 ? 32u : ndim == 2 ? 16u : 8u;
}

void launch_minmax_eb(const float *x, uint64_t n, Control *ctl, double eb, uint32_t mode,
                      int num_sms, cudaStream_t st);
// sets DERR_STALE unless the kHeaderBytes at arc (4-byte aligned) equal expect
void launch_header_check(const void *arc, const uint8_t *expect, Control *ctl, cudaStream_t st);
int launch_dualquant(const QuantArgs &a, cudaStream_t st);  // returns kernels launched

// grouped S0-S3 (items and block tables in device memory)
struct MinmaxItem {
    const float *x;
    uint64_t n;
    Control *ctl;
    double eb;
    uint32_t mode;
};
struct QuantItem {
    QuantArgs a;
    uint32_t t[4];  // tiles: 1D {ntiles}; 2D {ntx, nty}; 3D {ntx, nty, ntz, z planes per tile}
};
// blocks of one field's S0 in a grouped launch
uint32_t minmax_blocks(uint64_t n, uint32_t mode, int num_sms);
// one order-1 field's S1-S3: its blocks, tile parameters, kernel variant
// (D * 4 + VEC * 2 + WIN) and dynamic shared memory
uint32_t dualquant_plan(const QuantArgs &a, uint32_t t[4], int *variant, size_t *smem);
void launch_minmax_group(const MinmaxItem *items, const uint32_t *first, uint32_t ni, uint32_t blocks, bool vec,
                         cudaStream_t st);
void launch_dualquant_group(int variant, const QuantItem *items, const uint32_t *first, uint32_t ni,
                            uint32_t blocks, size_t smem, cudaStream_t st);

struct CodebookArgs {
    const uint32_t *hist;  // for compress; NULL for the decode-table build
    const uint8_t *len_in; // for decode: lengths from the archive
    uint32_t nbins;
    uint8_t *len_out;      // compress: lengths (written into the archive)
    uint64_t *cw64;        // (len << 56) | code
    uint32_t *cw32;        // (len << 24) | code, valid when maxlen <= 24
    uint64_t *codes_only;  // plain codewords (debug copy)
    // decode tables
    uint32_t *lut;         // 1 << kLutBits entries: (sym << 8) | len, 0 = long code;
                           // then the second level (kLut2Words words, see kLut2Prefixes)
    unsigned long long *first;   // [kMaxLen + 2] first canonical code per length
    uint32_t *count;       // [kMaxLen + 2]
    uint32_t *start;       // [kMaxLen + 2]
    uint16_t *sorted;      // symbols in (len, sym) order
    void *lutf;            // complete table over fast_bits-bit prefixes (see kFastLutMax)
    uint32_t fast_bits;    // 0: no complete table
    uint32_t fast_pair;    // the table resolves two codes per entry
    uint32_t expect_maxlen;  // decode: header's maxlen
    // scratch (global, kMaxBins-sized or 2x)
    unsigned long long *keyA, *keyB;
    uint32_t *nodef, *parent, *distA, *distB, *parA, *parB;
    Control *ctl;
};
constexpr int kLutBits = 12;
// Second level of the decode table: for the kLut2Prefixes 12-bit prefixes
// from the smallest one that starts a longer code (canonical codes put all
// of them at the top), the code under each prefix and each value of the
// next kLut2Bits bits, as 16-bit entries (sym << 5) | len when that code has
// at most 12 + kLut2Bits bits and the symbol is below 2048, else 0.  Stored
// after the 4096 first-level entries: the first prefix (one word), then the
// entries.
constexpr uint32_t kLut2Bits = 4, kLut2Prefixes = 128;
constexpr uint32_t kLut2Entries = kLut2Prefixes << kLut2Bits;
constexpr uint32_t kLut2Words = 1 + kLut2Entries / 2;
// When every code is at most kFastLutMax bits and symbols fit 12 bits, the
// decoder uses one complete table indexed by B = maxlen bits.  Up to
// kPairLutMax bits an entry resolves the first code of its prefix and, when
// it also fits, the second: 32-bit entries len1 | len2 << 4 | sym1 << 8 |
// sym2 << 20 (len2 = 0: the second code is longer than the bits left).
// Above that, 16-bit entries (sym << 4) | len.  Length 0: no code matches.
constexpr uint32_t kFastLutMax = 15;
constexpr uint32_t kPairLutMax = 14;
constexpr size_t kFastLutBytes = 4u << kPairLutMax;  // also 2 << kFastLutMax
__host__ __device__ inline uint32_t fast_lut_bits(uint32_t maxlen, uint32_t nbins)
{
    return (maxlen >= 1 && maxlen <= kFastLutMax && nbins <= 4096) ? maxlen : 0u;
}

void launch_codebook(const CodebookArgs &a, cudaStream_t st);
void launch_codebook_group(const CodebookArgs *items, uint32_t count, cudaStream_t st);  // one CTA per field
void launch_decode_tables(const CodebookArgs &a, cudaStream_t st);

struct EncodeArgs {
    const uint16_t *codes;
    const float *x;
    const int2 *dscr;
    // code-0 bitmap (bit i of byte b: point 8b + i has code 0), or nullptr;
    // when set, the count phase writes it for the points below n and pack
    // leaves the outlier and exception records to k_encode_outliers
    uint32_t *zbits;
    uint64_t n;
    uint32_t chunk, radius, nbins;
    const uint64_t *cw64;
    const uint32_t *cw32;
    uint8_t *archive;
    uint64_t capacity;
    uint32_t *lane_bits;    // bits of every lane (S symbols) of every round
    const uint32_t *unit_exc;  // exceptions per unit, counted by the dual-quant kernels
    ulonglong2 *unit_tot;   // per unit: {words, outliers | exceptions << 32}
    ulonglong2 *unit_off;   // their exclusive prefix sums
    ulonglong2 *scan_part;  // scan scratch
    Control *ctl;
    uint32_t cw64_only;     // 1: read 64-bit codeword entries whatever the longest code
    // header fields (the field's own shape; 4D is not folded here)
    uint32_t ndim, eb_mode, lblock, order;
    uint64_t dims[4];
    double eb;
    int num_sms;
};
// phase 0: count, 1: scan of the unit totals, 2: pack (and, with a code-0
// bitmap, the outlier records); returns kernels launched
int launch_encode(const EncodeArgs &a, cudaStream_t st, int phase);

// grouped S5 (items and block tables in device memory)
struct EncodeItem {
    EncodeArgs a;
    uint64_t nunits;
    uint32_t use_smem;
};
// exclusive scan of one field's unit totals (words, outliers | exceptions << 32)
struct UnitScan {
    using T = ulonglong2;
    const ulonglong2 *tot;
    ulonglong2 *off;
    __device__ T load(uint64_t i) const { return tot[i]; }
    __device__ void store(uint64_t i, T v) const { off[i] = v; }
    __device__ void total(T) const {}
};
template <typename Op> struct ScanItem {
    using OpT = Op;
    Op o;
    uint64_t n;
    typename Op::T *partial;
    __device__ const Op &op() const { return o; }
};
// one field's S5 in a grouped launch: its item, the blocks of count (0) and
// pack (1), their dynamic shared memory, and the units to scan
void encode_plan(const EncodeArgs &a, EncodeItem *it, uint32_t blocks[2], size_t smem[2], uint64_t *scan_items);
void launch_encode_group(int phase, const EncodeItem *items, const uint32_t *first, uint32_t ni, uint32_t blocks,
                         size_t smem, cudaStream_t st);  // phase 0: count, 1: pack
int launch_unit_scan_group(const ScanItem<UnitScan> *items, const uint32_t *first, uint32_t ni, uint32_t blocks,
                           cudaStream_t st);
void launch_decode_tables_group(const CodebookArgs *items, uint32_t count, cudaStream_t st);  // one CTA per field
uint64_t encode_units(uint64_t n, uint32_t chunk);        // units (per-unit totals) of the encoder
uint32_t encode_unit_shift(uint32_t chunk);                // log2 of the encoder unit in points

struct DecodeArgs {
    const uint8_t *archive;
    uint64_t n;
    uint32_t chunk, nchunk, radius, maxlen;
    uint64_t words;
    uint64_t off_bits, off_stream;
    const uint32_t *lut;
    const unsigned long long *first;
    const uint32_t *count, *start;
    const uint16_t *sorted;
    const void *lutf;          // complete table when fast_bits != 0
    uint32_t fast_bits, fast_pair, num_sms;
    unsigned long long *chunk_off;  // scratch nchunk
    unsigned long long *scan_partial;  // scratch for the offset scan
    uint32_t *tile_sums;  // 1D: residual sum per 4096-point tile (zeroed), else NULL
    uint16_t *codes;
    Control *ctl;
    // 1D reconstruction inside the complete-table decoder (anchored archives,
    // launch_decode phase 2): the values, fl(2eb * q) with q from the chunk's
    // anchor; the outlier list and each chunk's first entry in it (ostart,
    // nchunk + 1 entries)
    float *out;
    float ebx2;
    const uint32_t *anchors;
    const uint2 *outl;
    const uint32_t *ostart;
    uint64_t m;
};
constexpr uint32_t kRecon1DTile = 512;  // 1D reconstruction tile (points): one warp of the value kernel
// phase 0: chunk word offsets (scan), 1: symbols, 2: values (fused S7-S8 of
// an anchored 1D archive with a complete table; d.out, d.anchors, d.outl,
// d.ostart set); returns kernels launched
int launch_decode(const DecodeArgs &a, cudaStream_t st, int phase);
// each chunk's first outlier: ostart[c] = first entry of the index-ordered
// list with idx >= c * chunk, c = 0 .. nchunk (ostart[nchunk] = m); a list
// out of order or out of range marks the archive corrupt; returns kernels
// launched
int launch_outlier_chunk_starts(const uint2 *outl, uint64_t m, uint64_t n, uint32_t chunk, uint32_t nchunk,
                                uint32_t *ostart, Control *ctl, cudaStream_t st);

// S7 with one warp per chunk (k_decode_warp.cu).  fuse = 0: the chunk's codes
// go to d.codes; 1: 1D order-1 fields only, S8 in the same pass: the values
// go to out, the codes stay on chip (needs n < 2^30, d.fast_bits != 0,
// d.chunk <= kWarpMaxChunk).  look: nchunk zeroed words; odp: exclusive
// prefix sums of the outliers' residuals (m + 1 entries).
constexpr uint32_t kWarpMaxChunk = 4096;
struct WarpDecodeArgs {
    DecodeArgs d;
    const uint2 *outl;  // outlier list: (index, residual) in index order
    const uint32_t *odp;
    uint64_t m;
    float ebx2;
    float *out;
    unsigned long long *look;
    uint32_t hold_chunk;  // test hook: this chunk's look-back word is never published (~0u: none)
    const uint32_t *anchors;  // anchored archives (fused only): checked against every chunk's last integer
};
// kernels launched (one)
int launch_decode_warp(const WarpDecodeArgs &w, bool fuse, cudaStream_t st);
// exclusive prefix sums of the outliers' residuals into odp[0..m] (m + 1
// entries; partial: scan_partials(m + 1) entries); returns kernels launched
int launch_outlier_prefix(const uint2 *outl, uint64_t m, uint32_t *odp, uint32_t *partial, Control *ctl,
                          cudaStream_t st);

// chunk word offsets: the exclusive prefix sum of ceil(bits / 32) over the
// archive's chunk table; a count above the longest chunk, or a total other
// than the header's, marks the archive corrupt
struct ChunkWords {
    using T = unsigned long long;
    const uint32_t *bits;
    unsigned long long *off;
    unsigned long long words, maxbits;
    Control *ctl;
    __device__ T load(uint64_t i) const
    {
        const uint32_t b = bits[i];
        if (b > maxbits) {
            atomicOr(&ctl->error, DERR_CORRUPT);
            return 0;
        }
        return (b + 31ull) / 32;
    }
    __device__ void store(uint64_t i, T v) const { off[i] = v; }
    __device__ void total(T t) const
    {
        if (t != words) atomicOr(&ctl->error, DERR_CORRUPT);
    }
};
inline ChunkWords chunk_words_op(const DecodeArgs &a)
{
    ChunkWords op;
    op.bits = reinterpret_cast<const uint32_t *>(a.archive + a.off_bits);
    op.off = a.chunk_off;
    op.words = a.words;
    op.maxbits = (unsigned long long)a.chunk * kMaxLen;
    op.ctl = a.ctl;
    return op;
}

// grouped S7 (items and block tables in device memory)
struct DecodeItem {
    DecodeArgs a;
    uint32_t sorted_in_smem;
};
// one field's decoder launch: blocks, variant (2: complete-table decoder,
// + 1: tiles of several chunks) and dynamic shared memory
unsigned decode_plan(const DecodeArgs &a, DecodeItem *it, int *variant, size_t *dyn);
void launch_decode_group(int variant, const DecodeItem *items, const uint32_t *first, uint32_t ni, uint32_t blocks,
                         size_t dyn, cudaStream_t st);
int launch_offsets_scan_group(const ScanItem<ChunkWords> *items, const uint32_t *first, uint32_t ni, uint32_t blocks,
                              cudaStream_t st);

struct ReconArgs {
    const uint16_t *codes;
    const uint8_t *archive;
    uint64_t off_outl, off_exc;
    uint64_t m, e;
    uint32_t ndim;
    uint64_t dims[3];
    uint32_t radius;
    float ebx2;
    int32_t *dscr;
    uint32_t lblock;      // 1: block-local reconstruction (the paper's blocks)
    uint32_t order;       // Lorenzo order n (1..3)
    uint32_t *faces;      // carry scratch; 1D: the tile sums left by the decoder
    uint64_t faces_cap;   // entries
    uint32_t *scan_partial;  // scratch for the 1D carry scan (order > 1: scan_partials(n) entries)
    float *out;
    Control *ctl;
    int num_sms;
    const uint32_t *anchors;  // anchored 1D archives: checked against the reconstructed integers
    uint32_t chunk;
};
uint64_t recon_faces_entries(uint32_t ndim, const uint64_t dims[3]);
void launch_reconstruct(const ReconArgs &a, cudaStream_t st, int *launches);
// the verbatim exceptions on top of the values (codes NULL: not checked
// against code 0); returns kernels launched
int launch_exceptions(const ReconArgs &a, cudaStream_t st);

// A launch of a grouped plan: given the plan's device address, enqueues its
// kernels on st and returns how many.
using GroupLaunch = std::function<int(const uint8_t *, cudaStream_t)>;
// Appends the grouped S8 of `count` order-1 fields to `plan` (host bytes,
// copied to the device before the launches run) and its launches, in stage
// order, to `launches`.
void plan_reconstruct_group(const ReconArgs *ra, uint32_t count, std::vector<uint8_t> &plan,
                            std::vector<GroupLaunch> &launches);

}  // namespace gbsz
