// k_decode.cu -- S7: Huffman decode (inflate, Sec. 3.3).
//
// Chunk word offsets are the exclusive prefix sum of ceil(bits/32) over the
// archive's chunk table (one single-pass scan kernel).  Decoding is
// sequential inside a chunk, as in the paper; one thread decodes one chunk.
// Each thread keeps a ring of its chunk's stream words in shared memory, fed
// by cp.async ahead of the decode, and a bit window of four registers
// advanced with selects instead of branches.  Three decoders:
//   k_decode          any code length: a 4096-entry table resolves codes of
//                     at most 12 bits, a second level those of 13-16 bits,
//                     the canonical per-length tables the rest;
//   k_decode_fast     codes of at most 15 bits: a lane-replicated table of
//                     the window's top byte gives one or two codes per
//                     lookup, the complete table the longer ones;
//   k_decode_fast_values  the same decode for anchored 1D archives (every
//                     chunk starts from its anchor) writing the values
//                     fl(2eb * q) instead of the codes: the reconstruction
//                     (Alg. 2) happens in the decoder.
// Codes leave in 16-byte stores, values in 32-byte stores.  Every chunk must
// consume exactly its recorded bit count and every code must exist in the
// codebook; anything else marks the archive corrupt.  For 1D fields the code
// decoders also accumulate the residual sum of every 512-point tile (in-cap
// codes only; outliers are added by the reconstruction), which the separate
// value pass scans instead of making another pass over the codes.
#include "common.cuh"
#include "scan.cuh"

#include <algorithm>
#include <atomic>
#include <cstring>

namespace gbsz {

namespace {

constexpr int kDecThreads = 256;
constexpr uint32_t kSortedSmemMax = 8192;  // symbols whose table is copied to shared memory



constexpr uint32_t kRing = 32;       // stream words per thread in shared memory (any code length)
constexpr uint32_t kRingFast = 16;   // the same for codes of at most kFastLutMax bits
constexpr int kDecFastThreads = 512;
constexpr int kFastValuesMaxThreads = 1024;  // k_decode_fast_values: one block per SM of up to 32 warps
constexpr uint32_t kBatch = 8;       // symbols between refill checks

// 4-byte cp.async of which src_bytes (4 or 0) are read and the rest of the
// word zero-filled: no branch around words past the end of the stream
__device__ __forceinline__ void cp_async4_fill(uint32_t *dst, const uint32_t *src, uint32_t src_bytes)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// A thread's view of its chunk: word v of the chunk lives in ring slot
// v mod RW; a warp's rings are interleaved (slot j of lane l at j * 32 + l),
// so the 32 lanes of a warp read 32 different banks whatever their
// positions.  Quarter q (words Q*q .. Q*q+Q-1, Q = RW/4) is loaded into the
// slots that quarter q - 4 used.  Before each batch the quarters up to the
// one after next of the current word have landed: at least 2Q+1 words
// ahead, which covers a batch's consumption plus the four-word look-ahead
// (RW = 32: 8 codes of up to 45 bits, at most 12 words; RW = 16: 8 codes of
// up to 15 bits, at most 4 words).
template <uint32_t RW>
struct Ring {
    static constexpr uint32_t Q = RW / 4;
    uint32_t *r;          // slot 0 of this lane
    const uint32_t *src;  // the chunk's first word
    uint64_t avail;       // stream words from src to the end of the stream
    uint32_t qnext;
    __device__ __forceinline__ uint32_t &at(uint32_t v) const { return r[(v & (RW - 1)) * 32]; }
    __device__ __forceinline__ void load_quarter()
    {
#pragma unroll
        for (uint32_t i = 0; i < Q; i++) {
            const uint32_t v = qnext * Q + i;
            const bool in = v < avail;  // past the end: a zero word (src stays a valid address)
            cp_async4_fill(&at(v), in ? src + v : src, in ? 4u : 0u);
        }
        cp_async_commit();
        qnext++;
    }
    // ring: this warp's ring block (RW * 32 words); lane: the lane's column
    __device__ __forceinline__ void start(uint32_t *warp_ring, uint32_t lane, const uint32_t *chunk_src,
                                          uint64_t words_left)
    {
        r = warp_ring + lane;
        src = chunk_src;
        avail = words_left;
        qnext = 0;
        for (int q = 0; q < 4; q++) load_quarter();
        cp_async_wait<0>();
    }
    // before a batch that starts at word v
    __device__ __forceinline__ void refill(uint32_t v)
    {
        if (v / Q + 3 >= qnext) {
            do {
                load_quarter();
            } while (v / Q + 3 >= qnext);
            cp_async_wait<1>();
        }
    }
};

// A ring fed a few words at a time (RW words per lane, interleaved as in
// Ring), used by the decoder that writes the values: instead of a quarter at
// a time whenever a lane runs low -- a branch some lane of the warp takes in
// almost every batch -- every batch requests up to K next words, each
// predicated on a free slot, so the ring stays full without divergence.
// (Measured on the 2^28 walk: fused decode 0.492 -> 0.464 ms.  The decoder
// writing codes, in two 512-thread blocks per SM, measured 0.489 -> 0.506 ms
// with it, and the general decoder on a 512^3 lognormal field at rel eb 1e-4,
// whose codes average 7.8 bits, 0.405 -> 0.532 ms with K = 4: both keep
// Ring.  One word a batch measured the same as two here; a copy of the
// complete table in shared memory, which helps the fused decoder, made the
// codes decoder slower too, 0.489 -> 0.503 ms, by taking L1 from its rings.)  Before a batch at word v, every word requested in an
// earlier batch has landed (wait_group 1 leaves only this batch's pending);
// a lane that drained to within v + AHEAD (it consumed more than K words a
// batch for a while) refills the whole ring and waits for it.  Either way
// words v .. v + AHEAD are in the ring: AHEAD covers a batch's consumption
// plus the four-word look-ahead (RW = 16: 8 codes of up to 15 bits, AHEAD =
// 8; RW = 32: 8 codes of up to 45 bits, AHEAD = 16).
template <uint32_t RW, uint32_t K, uint32_t AHEAD>
struct TrickleRing {
    uint32_t *r;          // slot 0 of this lane
    const uint32_t *src;  // the chunk's first word
    uint64_t avail;       // stream words from src to the end of the stream
    uint32_t qw;          // next word to request
    __device__ __forceinline__ uint32_t &at(uint32_t v) const { return r[(v & (RW - 1)) * 32]; }
    __device__ __forceinline__ void load(uint32_t v)
    {
        const bool in = v < avail;  // past the end: a zero word (src stays a valid address)
        cp_async4_fill(&at(v), in ? src + v : src, in ? 4u : 0u);
    }
    __device__ __forceinline__ void start(uint32_t *warp_ring, uint32_t lane, const uint32_t *chunk_src,
                                          uint64_t words_left)
    {
        r = warp_ring + lane;
        src = chunk_src;
        avail = words_left;
#pragma unroll
        for (uint32_t v = 0; v < RW; v++) load(v);
        cp_async_commit();
        cp_async_wait<0>();
        qw = RW;
    }
    // before a batch that starts at word v
    __device__ __forceinline__ void refill(uint32_t v)
    {
        const uint32_t q0 = qw;
#pragma unroll
        for (uint32_t k = 0; k < K; k++)
            if (qw < v + RW) load(qw++);  // a slot is free once its word is below v
        cp_async_commit();
        if (q0 <= v + AHEAD) {  // drained: fill every free slot and wait for all of them
            while (qw < v + RW) load(qw++);
            cp_async_commit();
            cp_async_wait<0>();
        } else {
            cp_async_wait<1>();
        }
    }
};
using FastRing = TrickleRing<kRingFast, 2, 8>;

// Bit window: hi, lo, q0, q1 = words v .. v+3.  The next 32 stream bits are
// funnelshift(lo, hi, bo).  Each step reads word v+4 from the ring before it
// looks at the table, so that read is not behind the lookup in the
// dependency chain, and shifts it in with selects if a word was consumed.
struct Window {
    uint32_t v, bo, hi, lo, q0, q1;
};

struct DecTables {
    const uint32_t *lut;
    const uint16_t *lut2;  // second level (kLut2Entries) and its first prefix
    uint32_t l2lo;
    const unsigned long long *first;
    const uint32_t *count, *start;
    const uint16_t *sorted;
    uint32_t maxlen;
    uint32_t nsorted;  // entries of sorted (bins)
    Control *ctl;
};

template <class RG>
__device__ __forceinline__ void advance_one(Window &w, const RG &rg)
{
    w.v++;
    w.hi = w.lo;
    w.lo = w.q0;
    w.q0 = rg.at(w.v + 2);
    w.q1 = rg.at(w.v + 3);
}

// Window step after consuming len (< 32) bits: at most one word boundary;
// nxt is word v+4, read at the start of the step.
__device__ __forceinline__ void step(Window &w, uint32_t nxt, uint32_t len)
{
    w.bo += len;
    const bool adv = w.bo >= 32;
    w.bo &= 31u;
    w.v += adv ? 1u : 0u;
    w.hi = adv ? w.lo : w.hi;
    w.lo = adv ? w.q0 : w.lo;
    w.q0 = adv ? w.q1 : w.q0;
    w.q1 = adv ? nxt : w.q1;
}

// one symbol; sets bad on a code that is not in the codebook
__device__ __forceinline__ uint32_t decode_one(Window &w, const Ring<kRing> &rg, const DecTables &t, bool &bad)
{
    const uint32_t nxt = rg.at(w.v + 4);
    const uint32_t cur = __funnelshift_l(w.lo, w.hi, w.bo);
    uint32_t e = t.lut[cur >> (32 - kLutBits)];
    if (e == 0) {  // longer than 12 bits: the second level resolves codes of up to 16
        const uint32_t j = (cur >> (32 - kLutBits)) - t.l2lo;
        const uint32_t e2 = j < kLut2Prefixes ? t.lut2[(j << kLut2Bits) | ((cur >> (32 - kLutBits - kLut2Bits)) &
                                                                            ((1u << kLut2Bits) - 1))]
                                              : 0u;
        e = ((e2 >> 5) << 8) | (e2 & 31u);
    }
    uint32_t sym = e >> 8, len = e & 0xFFu;
    if (e == 0) {
        // a code longer than the table: search the canonical tables, then
        // consume it here (it may cross two word boundaries)
        const unsigned long long v64 = ((unsigned long long)cur << 32) | __funnelshift_l(w.q0, w.lo, w.bo);
        len = 0;
        for (uint32_t l = kLutBits + 1; l <= t.maxlen; l++) {
            const unsigned long long off = (v64 >> (64 - l)) - t.first[l];
            if (off < t.count[l]) {
                len = l;
                sym = GBSZ_CHECK(t.start[l] + off < t.nsorted, t.ctl) ? t.sorted[t.start[l] + off] : 0u;
                break;
            }
        }
        bad |= len == 0;
        w.bo += len;
        while (w.bo >= 32) {
            w.bo -= 32;
            advance_one(w, rg);
        }
        return sym;
    }
    step(w, nxt, len);
    return sym;
}

__device__ __forceinline__ uint32_t zeros_in(uint32_t pair)  // code-0 halves of a packed pair
{
    return __popc(__vcmpeq2(pair, 0u)) >> 4;
}

// one chunk c of the general decoder (any code length)
template <bool MULTI_TILE>
__device__ __forceinline__ void decode_chunk_general(const DecodeArgs &a, const DecTables &t, uint32_t *s_dyn,
                                                     uint64_t c)
{
    const uint32_t *stream = reinterpret_cast<const uint32_t *>(a.archive + a.off_stream);
    const uint32_t nbits = reinterpret_cast<const uint32_t *>(a.archive + a.off_bits)[c];
    const uint64_t coff = a.chunk_off[c];
    const uint64_t s0 = c * a.chunk;
    const uint32_t cnt = (uint32_t)(a.n - s0 < a.chunk ? a.n - s0 : a.chunk);
    const uint32_t R = a.radius;
    Ring<kRing> rg;
    rg.start(s_dyn + (threadIdx.x >> 5) * kRing * 32, threadIdx.x & 31, stream + coff,
             coff < a.words ? a.words - coff : 0);
    Window w{0, 0, rg.at(0), rg.at(1), rg.at(2), rg.at(3)};
    uint32_t zeros = 0, ssum = 0, tz = 0, tstart = 0;  // tz, tstart: zeros and first index of the open tile
    bool bad = false;
    uint16_t *out = a.codes + s0;
    const uint32_t full = cnt & ~(kBatch - 1);
    for (uint32_t k = 0; k < full; k += kBatch) {
        rg.refill(w.v);
        uint32_t sy[kBatch];
#pragma unroll
        for (int j = 0; j < (int)kBatch; j++) {
            sy[j] = decode_one(w, rg, t, bad);
            ssum += sy[j];
        }
        const uint4 o = make_uint4(sy[0] | (sy[1] << 16), sy[2] | (sy[3] << 16), sy[4] | (sy[5] << 16),
                                   sy[6] | (sy[7] << 16));
        if (GBSZ_CHECK(s0 + k + kBatch <= a.n, a.ctl)) *reinterpret_cast<uint4 *>(out + k) = o;
        tz += zeros_in(o.x) + zeros_in(o.y) + zeros_in(o.z) + zeros_in(o.w);
        if (MULTI_TILE && a.tile_sums && ((s0 + k + kBatch) & (kRecon1DTile - 1)) == 0) {
            // residual sum of the tile's in-cap codes: sum(code) - R * (#nonzero), mod 2^32
            const uint32_t m = k + kBatch - tstart;
            if (GBSZ_CHECK((s0 + k) / kRecon1DTile < (a.n + kRecon1DTile - 1) / kRecon1DTile, a.ctl))
                atomicAdd(&a.tile_sums[(s0 + k) / kRecon1DTile], ssum - R * (m - tz));
            zeros += tz;
            ssum = tz = 0;
            tstart = k + kBatch;
        }
        if (bad) break;
    }
    if (!bad && full < cnt) {
        rg.refill(w.v);
        for (uint32_t k = full; k < cnt; k++) {
            const uint32_t sym = decode_one(w, rg, t, bad);
            ssum += sym;
            tz += sym == 0;
            if (GBSZ_CHECK(s0 + k < a.n, a.ctl)) out[k] = (uint16_t)sym;
        }
    }
    zeros += tz;
    if (a.tile_sums && cnt > tstart) {
        const uint32_t tsum = ssum - R * (cnt - tstart - tz);
        if (tsum && GBSZ_CHECK(s0 + cnt - 1 < a.n, a.ctl)) atomicAdd(&a.tile_sums[(s0 + cnt - 1) / kRecon1DTile], tsum);
    }
    cp_async_wait<0>();  // nothing may still be landing in the ring when the block exits
    // a valid chunk ends exactly at its recorded bit count
    if (bad || (uint64_t)w.v * 32 + w.bo != nbits) atomicOr(&a.ctl->error, DERR_CORRUPT);
    if (zeros) atomicAdd(&a.ctl->zeros, (unsigned long long)zeros);
}

// Persistent: warp task k is chunks 32k .. 32k+31, one per lane; block b's
// warp w takes tasks w * gridDim.x + b, w * gridDim.x + b + (warps in the
// grid), ...  Tasks are spread over the blocks first, so every block, and so
// every SM, gets the same number of tasks to within one.
template <bool MULTI_TILE>
__device__ __forceinline__ void decode_general_body(const DecodeArgs &a, uint32_t sorted_in_smem, VGrid vg)
{
    __shared__ uint32_t lut[1 << kLutBits];
    __shared__ uint16_t lut2[kLut2Entries];
    __shared__ unsigned long long first[kMaxLen + 2];
    __shared__ uint32_t count[kMaxLen + 2], start[kMaxLen + 2];
    extern __shared__ uint32_t s_dyn[];  // rings, then the sorted symbols
    uint16_t *s_sorted = reinterpret_cast<uint16_t *>(s_dyn + kDecThreads * kRing);
    for (uint32_t i = threadIdx.x; i < (1u << kLutBits); i += blockDim.x) lut[i] = a.lut[i];
    const uint16_t *g2 = reinterpret_cast<const uint16_t *>(a.lut + (1u << kLutBits) + 1);
    for (uint32_t i = threadIdx.x; i < kLut2Entries; i += blockDim.x) lut2[i] = g2[i];
    for (uint32_t i = threadIdx.x; i < kMaxLen + 2; i += blockDim.x) {
        first[i] = a.first[i];
        count[i] = a.count[i];
        start[i] = a.start[i];
    }
    for (uint32_t i = threadIdx.x; i < sorted_in_smem; i += blockDim.x) s_sorted[i] = a.sorted[i];
    __syncthreads();
    if (a.ctl->error & DERR_CORRUPT) return;
    const DecTables t{lut,    lut2,     a.lut[1u << kLutBits], first, count, start, sorted_in_smem ? s_sorted : a.sorted,
                      a.maxlen, 2 * a.radius, a.ctl};
    const uint64_t ntask = (a.nchunk + 31) / 32, tstride = (uint64_t)(blockDim.x >> 5) * vg.nb;
    for (uint64_t k = (uint64_t)(threadIdx.x >> 5) * vg.nb + vg.bid; k < ntask; k += tstride) {
        const uint64_t c = k * 32 + (threadIdx.x & 31);
        if (c < a.nchunk) decode_chunk_general<MULTI_TILE>(a, t, s_dyn, c);
    }
}

template <bool MULTI_TILE>
__global__ void __launch_bounds__(kDecThreads) k_decode(const __grid_constant__ DecodeArgs a, uint32_t sorted_in_smem)
{
    decode_general_body<MULTI_TILE>(a, sorted_in_smem, vgrid_self());
}

// Two-level decode for archives whose codes all fit the complete table
// (at most kFastLutMax bits).  Level 1 resolves every code of at most 8 bits
// from the window's top byte.  Its 8-byte entries are replicated 16 times
// (entry i of copy c at 8-byte slot 16 i + c, lane l reading copy l % 16):
// the 16 lanes of each half warp, which one 8-byte shared access serves
// together, read 16 different copies in 32 different banks, so the lookups
// never conflict.  Longer codes take the complete table (16-bit
// entries (sym << 4) | len over B = maxlen bits) under a warp-uniform branch.
// A pattern that matches no code has length 0; the smallest length seen is
// checked after the chunk.
constexpr uint32_t kL1Bits = 8;
constexpr uint32_t kL1Copies = 16;

// complete-table entry from global memory (read-only path; the rarely used
// part of the table stays in L1)
__device__ __forceinline__ uint32_t ld_ft_pred(bool p, const uint16_t *addr, uint32_t keep)
{
    uint32_t v = keep;
    asm volatile(
        "{\n\t.reg .pred q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "@q ld.global.nc.u16 %0, [%2];\n\t}"
        : "+r"(v)
        : "r"((uint32_t)p), "l"(addr));
    return v;
}

// the same from a copy of the complete table in shared memory
__device__ __forceinline__ uint32_t ld_ft_pred_smem(bool p, const uint16_t *addr, uint32_t keep)
{
    uint32_t v = keep;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(addr);
    asm volatile(
        "{\n\t.reg .pred q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "@q ld.shared.u16 %0, [%2];\n\t}"
        : "+r"(v)
        : "r"((uint32_t)p), "r"(a));
    return v;
}
template <bool FT_SMEM>
__device__ __forceinline__ uint32_t ld_ft(bool p, const uint16_t *addr, uint32_t keep)
{
    return FT_SMEM ? ld_ft_pred_smem(p, addr, keep) : ld_ft_pred(p, addr, keep);
}

// Two codes per step.  The level-1 entry of the window's top byte holds the
// first code and, when it fits in the same byte, the second, as 8 bytes:
// x = sym1 | sym2 << 16 (the two symbols as they are stored), y = len1 |
// len2 << 8 (len1 = 0: the first code is longer than 8 bits; len2 = 0: the
// second is not in the byte).  Missing
// codes come from a second level-1 lookup after the first code and, for codes
// longer than 8 bits, from the complete table in global memory; each of these
// runs only when some lane of the warp needs it.  act1 / act2 = false (lanes past the end
// of a short chunk, kept in step for the warp votes): that code consumes no
// bits and its length is not checked.
__device__ __forceinline__ uint2 ld_shared_pred64(bool p, const void *addr)
{
    uint2 v = make_uint2(0u, 0u);
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(addr);
    asm volatile(
        "{\n\t.reg .pred q;\n\t"
        "setp.ne.u32 q, %2, 0;\n\t"
        "@q ld.shared.v2.u32 {%0, %1}, [%3];\n\t}"
        : "+r"(v.x), "+r"(v.y)
        : "r"((uint32_t)p), "r"(a));
    return v;
}

// Returns the two symbols packed as stored (sym1 | sym2 << 16).  FT_SMEM: ft
// is a copy of the complete table in shared memory.
// ZF: the level-1 entries also flag code-0 symbols (bit 16: the first code,
// bit 17: the second), and zf returns those two flags.
template <bool FT_SMEM = false, bool ZF = false, class RG = Ring<kRingFast>>
__device__ __forceinline__ uint32_t decode_two(Window &w, const RG &rg, const uint2 *l1,
                                               const uint16_t *ft, uint32_t shift, uint32_t &minlen, bool act1,
                                               bool act2, uint32_t *zf = nullptr)
{
    const uint32_t nxt = rg.at(w.v + 4);
    const uint32_t c0 = __funnelshift_l(w.lo, w.hi, w.bo);
    const uint32_t c1 = __funnelshift_l(w.q0, w.lo, w.bo);
    const uint2 e = l1[(c0 >> (32 - kL1Bits)) * kL1Copies];
    uint32_t sw = e.x;
    uint32_t l1n = e.y & 0xFFu, l2n = ZF ? (e.y >> 8) & 0xFFu : e.y >> 8;
    if (ZF) *zf = e.y >> 16;
    // One vote for both rare paths: an entry without a second code (l2n = 0)
    // covers a first code over 8 bits too (its entry is all zero).  The
    // lengths of an entry with both codes are those of real codewords, so a
    // pattern missing from the codebook (length 0) can only come out of this
    // branch, and the smallest length is tracked here alone.
    if (__any_sync(0xffffffffu, l2n == 0)) {
        const bool long1 = l1n == 0;
        if (__any_sync(0xffffffffu, long1)) {
            const uint32_t f = ld_ft<FT_SMEM>(long1, ft + (c0 >> shift), 0u);
            if (long1) {
                l1n = f & 15u;
                sw = f >> 4;
                l2n = 0;
            }
        }
        const bool need2 = l2n == 0;
        const uint32_t cur2 = __funnelshift_l(c1, c0, l1n);  // the bits after the first code (l1n < 16)
        const uint2 e2 = ld_shared_pred64(need2, l1 + (cur2 >> (32 - kL1Bits)) * kL1Copies);
        uint32_t l2b = e2.y & 0xFFu, s2b = e2.x & 0xFFFFu;
        const bool long2 = need2 && l2b == 0;
        if (__any_sync(0xffffffffu, long2)) {
            const uint32_t f = ld_ft<FT_SMEM>(long2, ft + (cur2 >> shift), 0u);
            if (long2) {
                l2b = f & 15u;
                s2b = f >> 4;
            }
        }
        if (need2) {
            l2n = l2b;
            sw = (sw & 0xFFFFu) | (s2b << 16);
        }
        minlen = min(minlen, min(act1 ? l1n : 15u, act2 ? l2n : 15u));
        if (ZF) *zf = ((sw & 0xFFFFu) == 0 ? 1u : 0u) | ((sw >> 16) == 0 ? 2u : 0u);
    }
    l1n = act1 ? l1n : 0u;
    l2n = act2 ? l2n : 0u;
    step(w, nxt, l1n + l2n);
    return sw;
}

// single code (the odd last symbol of a chunk)
template <bool FT_SMEM = false, bool ZF = false, class RG = Ring<kRingFast>>
__device__ __forceinline__ uint32_t decode_two_level(Window &w, const RG &rg, const uint2 *l1,
                                                     const uint16_t *ft, uint32_t shift, uint32_t &minlen,
                                                     bool active)
{
    uint32_t zf;
    return decode_two<FT_SMEM, ZF, RG>(w, rg, l1, ft, shift, minlen, active, false, &zf) & 0xFFFFu;
}

// One chunk of cnt symbols; the warp runs kend >= cnt symbol steps (GUARD:
// some lane's chunk is shorter than the warp's longest).
template <bool MULTI_TILE, bool GUARD>
__device__ __forceinline__ void decode_chunk(const DecodeArgs &a, Ring<kRingFast> &rg, Window &w, const uint2 *l1,
                                             const uint16_t *ft, uint32_t shift, uint64_t s0, uint32_t cnt,
                                             uint32_t kend, unsigned long long &zeros, uint32_t &minlen)
{
    const uint32_t R = a.radius;
    uint32_t ssum = 0, tz = 0, tstart = 0;
    uint16_t *out = a.codes + s0;
    const uint32_t full = kend & ~(kBatch - 1);
    for (uint32_t k = 0; k < full; k += kBatch) {
        rg.refill(w.v);
        uint32_t pw[kBatch / 2];  // symbol pairs as stored
#pragma unroll
        for (int j = 0; j < (int)kBatch; j += 2)
            pw[j / 2] = decode_two(w, rg, l1, ft, shift, minlen, !GUARD || k + j < cnt, !GUARD || k + j + 1 < cnt);
        if (!GUARD || k + kBatch <= cnt) {
            const uint4 o = make_uint4(pw[0], pw[1], pw[2], pw[3]);
            // symbols are below 4096 here, so the halves of the word sum cannot carry
            const uint32_t t4 = o.x + o.y + o.z + o.w;
            ssum += (t4 & 0xFFFFu) + (t4 >> 16);
            if (GBSZ_CHECK(s0 + k + kBatch <= a.n, a.ctl)) *reinterpret_cast<uint4 *>(out + k) = o;
            tz += zeros_in(o.x) + zeros_in(o.y) + zeros_in(o.z) + zeros_in(o.w);
        } else {
#pragma unroll
            for (int j = 0; j < (int)kBatch; j++) {
                if (k + j < cnt) {
                    const uint32_t sy = (pw[j / 2] >> ((j & 1) * 16)) & 0xFFFFu;
                    ssum += sy;
                    tz += sy == 0;
                    if (GBSZ_CHECK(s0 + k + j < a.n, a.ctl)) out[k + j] = (uint16_t)sy;
                }
            }
        }
        if (MULTI_TILE && a.tile_sums && (!GUARD || k + kBatch <= cnt) &&
            ((s0 + k + kBatch) & (kRecon1DTile - 1)) == 0) {
            // residual sum of the tile's in-cap codes: sum(code) - R * (#nonzero), mod 2^32
            const uint32_t m = k + kBatch - tstart;
            if (GBSZ_CHECK((s0 + k) / kRecon1DTile < (a.n + kRecon1DTile - 1) / kRecon1DTile, a.ctl))
                atomicAdd(&a.tile_sums[(s0 + k) / kRecon1DTile], ssum - R * (m - tz));
            zeros += tz;
            ssum = tz = 0;
            tstart = k + kBatch;
        }
    }
    if (full < kend) {
        rg.refill(w.v);
        for (uint32_t k = full; k < kend; k++) {
            const uint32_t sym = decode_two_level(w, rg, l1, ft, shift, minlen, !GUARD || k < cnt);
            if (!GUARD || k < cnt) {
                ssum += sym;
                tz += sym == 0;
                if (GBSZ_CHECK(s0 + k < a.n, a.ctl)) out[k] = (uint16_t)sym;
            }
        }
    }
    zeros += tz;
    if (a.tile_sums && cnt > tstart) {
        const uint32_t tsum = ssum - R * (cnt - tstart - tz);
        if (tsum && GBSZ_CHECK(s0 + cnt - 1 < a.n, a.ctl)) atomicAdd(&a.tile_sums[(s0 + cnt - 1) / kRecon1DTile], tsum);
    }
}

// Level 1 from the complete table: the code at the start of each byte if it
// has at most 8 bits, and the code after it if that fits in the byte; built
// once per block in the (not yet used) ring area, then copied per lane.
template <bool ZF = false>
__device__ __forceinline__ void build_level1(const DecodeArgs &a, uint32_t *s_dyn, uint2 *l1tab)
{
    const uint32_t B = a.fast_bits;
    const uint16_t *gft = static_cast<const uint16_t *>(a.lutf);
    auto ft_at = [&](uint32_t byte) -> uint32_t {  // complete-table entry of an 8-bit prefix
        return B >= kL1Bits ? gft[byte << (B - kL1Bits)] : gft[byte >> (kL1Bits - B)];
    };
    // the 256 entries once (in the ring area, not in use yet), then one copy per lane
    uint2 *l1once = reinterpret_cast<uint2 *>(s_dyn);
    for (uint32_t i = threadIdx.x; i < (1u << kL1Bits); i += blockDim.x) {
        const uint32_t f = ft_at(i);
        const uint32_t la = f & 15u;
        uint2 e = make_uint2(0u, 0u);
        if (la >= 1 && la <= kL1Bits) {
            e = make_uint2(f >> 4, la | (ZF && (f >> 4) == 0 ? 1u << 16 : 0u));
            if (la < kL1Bits) {
                const uint32_t g2 = ft_at((i << la) & 0xFFu);
                const uint32_t lb = g2 & 15u;
                if (lb >= 1 && lb <= kL1Bits - la)
                    e = make_uint2((f >> 4) | ((g2 >> 4) << 16),
                                   la | (lb << 8) | (ZF && (f >> 4) == 0 ? 1u << 16 : 0u) |
                                       (ZF && (g2 >> 4) == 0 ? 1u << 17 : 0u));
            }
        }
        l1once[i] = e;
    }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < (kL1Copies << kL1Bits); k += blockDim.x) l1tab[k] = l1once[k / kL1Copies];
    __syncthreads();
}

template <bool MULTI_TILE>
__device__ __forceinline__ void decode_fast_body(const DecodeArgs &a, VGrid vg)
{
    extern __shared__ uint32_t s_dyn[];  // rings, level-1 table (lane-replicated)
    uint2 *l1tab = reinterpret_cast<uint2 *>(s_dyn + blockDim.x * kRingFast);
    const uint32_t B = a.fast_bits, shift = 32 - B;
    const uint16_t *ft = static_cast<const uint16_t *>(a.lutf);
    build_level1(a, s_dyn, l1tab);
    if (a.ctl->error & DERR_CORRUPT) return;
    const uint32_t *stream = reinterpret_cast<const uint32_t *>(a.archive + a.off_stream);
    const uint32_t *bits_tab = reinterpret_cast<const uint32_t *>(a.archive + a.off_bits);
    uint32_t *warp_ring = s_dyn + (threadIdx.x >> 5) * kRingFast * 32;
    const uint32_t lane = threadIdx.x & 31;
    const uint2 *l1 = l1tab + lane % kL1Copies;
    unsigned long long zeros = 0;
    bool bad = false;
    const uint64_t stride = (uint64_t)vg.nb * blockDim.x;
    // whole warps iterate together (the level-1 fallback votes across the
    // warp); lanes past the last chunk decode nothing.  Consecutive chunks go
    // to consecutive threads: spreading warp tasks evenly over the blocks
    // instead (as k_decode does) measured about 4% slower here (2^28 symbols
    // in 2048-symbol chunks), since it does not even out the warps per
    // scheduler, which bound this latency-bound loop.
    for (uint64_t cw = (uint64_t)vg.bid * blockDim.x + threadIdx.x - lane; cw < a.nchunk; cw += stride) {
        const uint64_t c = cw + lane;
        const bool live = c < a.nchunk;
        const uint32_t nbits = live ? bits_tab[c] : 0u;
        const uint64_t coff = live ? a.chunk_off[c] : 0u;
        const uint64_t s0 = live ? c * a.chunk : 0u;
        const uint32_t cnt = live ? (uint32_t)(a.n - s0 < a.chunk ? a.n - s0 : a.chunk) : 0u;
        Ring<kRingFast> rg;
        rg.start(warp_ring, lane, stream + coff, coff < a.words ? a.words - coff : 0);
        Window w{0, 0, rg.at(0), rg.at(1), rg.at(2), rg.at(3)};
        uint32_t minlen = 15;
        if (__all_sync(0xffffffffu, cnt == a.chunk)) {
            decode_chunk<MULTI_TILE, false>(a, rg, w, l1, ft, shift, s0, cnt, cnt, zeros, minlen);
        } else {
            const uint32_t cmax = __reduce_max_sync(0xffffffffu, cnt);
            decode_chunk<MULTI_TILE, true>(a, rg, w, l1, ft, shift, s0, cnt, cmax, zeros, minlen);
        }
        cp_async_wait<0>();  // the ring is reused by the next chunk
        if (live) bad |= minlen == 0 || (uint64_t)w.v * 32 + w.bo != nbits;
        __syncwarp();
    }
    if (bad) atomicOr(&a.ctl->error, DERR_CORRUPT);
    if (zeros) atomicAdd(&a.ctl->zeros, zeros);
}

template <bool MULTI_TILE>
__global__ void __launch_bounds__(kDecFastThreads, 2) k_decode_fast(const __grid_constant__ DecodeArgs a)
{
    decode_fast_body<MULTI_TILE>(a, vgrid_self());
}

// 32-byte store of eight values (out 32-byte aligned), else two 16-byte stores
__device__ __forceinline__ void store8(float *out, const float (&v)[8], bool al32)
{
    if (al32) {
        asm volatile("st.global.v8.f32 [%0], {%1, %2, %3, %4, %5, %6, %7, %8};" ::"l"(out), "f"(v[0]), "f"(v[1]),
                     "f"(v[2]), "f"(v[3]), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7])
                     : "memory");
    } else {
        reinterpret_cast<float4 *>(out)[0] = make_float4(v[0], v[1], v[2], v[3]);
        reinterpret_cast<float4 *>(out)[1] = make_float4(v[4], v[5], v[6], v[7]);
    }
}

// A lane's place in the index-ordered outlier list: its chunk's entries are
// op .. oend-1; the next two are loaded one batch ahead of their use.
struct OutlierCursor {
    uint32_t op, oend;
    uint2 o1, o2;
    __device__ __forceinline__ uint2 at(const DecodeArgs &a, uint32_t i) const
    {
        return i < oend ? a.outl[i] : make_uint2(0xFFFFFFFFu, 0u);
    }
    __device__ __forceinline__ void fetch(const DecodeArgs &a)
    {
        o1 = at(a, op);
        o2 = at(a, op + 1);
    }
};

// Residuals of `cnt8` (<= 8) decoded symbols starting at point p0: code - R,
// and for code 0 the residual of the lane's next outlier entry, whose index
// must be the point's.  The patch goes through the thread's two staging
// slots in shared memory (the code-0 positions are only known at run time);
// the branch around it is warp-uniform.
__device__ __forceinline__ void residuals8(const DecodeArgs &a, const uint32_t (&pw)[4], uint32_t cnt8, uint64_t p0,
                                           uint32_t zflags, uint32_t (&d)[8], OutlierCursor &oc, uint4 *stg0,
                                           uint4 *stg1, bool &bad, unsigned long long &zeros)
{
    const uint32_t R = a.radius;
    // zflags: bit j set for a code-0 symbol j (from the decode tables)
    const uint32_t zm = zflags & (cnt8 >= 8 ? 0xFFu : (1u << cnt8) - 1u);
#pragma unroll
    for (int j = 0; j < 8; j++) {
        const uint32_t sy = (pw[j >> 1] >> ((j & 1) * 16)) & 0xFFFFu;
        d[j] = (uint32_t)j < cnt8 ? sy - R : 0u;
    }
    if (__any_sync(0xffffffffu, zm != 0)) {
        *stg0 = make_uint4(d[0], d[1], d[2], d[3]);
        *stg1 = make_uint4(d[4], d[5], d[6], d[7]);
        // the first two code-0 points take the two prefetched records without
        // a loop; a third or more in one batch (rare) read theirs in a loop
        const uint32_t nz = __popc(zm);
        const uint32_t m1 = zm & (zm - 1u);
        if (nz >= 1) {
            const uint32_t j = __ffs(zm) - 1;
            bad |= oc.op >= oc.oend || oc.o1.x != (uint32_t)(p0 + j);
            reinterpret_cast<uint32_t *>(j < 4 ? stg0 : stg1)[j & 3] = oc.o1.y;
        }
        if (nz >= 2) {
            const uint32_t j = __ffs(m1) - 1;
            bad |= oc.op + 1 >= oc.oend || oc.o2.x != (uint32_t)(p0 + j);
            reinterpret_cast<uint32_t *>(j < 4 ? stg0 : stg1)[j & 3] = oc.o2.y;
        }
        if (nz > 2) {
            uint32_t mm = m1 & (m1 - 1u);
            for (uint32_t t = 2; mm; t++) {
                const uint32_t j = __ffs(mm) - 1;
                mm &= mm - 1;
                const uint2 e = oc.at(a, oc.op + t);
                bad |= oc.op + t >= oc.oend || e.x != (uint32_t)(p0 + j);
                reinterpret_cast<uint32_t *>(j < 4 ? stg0 : stg1)[j & 3] = e.y;
            }
        }
        if (nz) {
            oc.op += nz;
            zeros += nz;
            oc.fetch(a);
        }
        const uint4 u0 = *stg0, u1 = *stg1;
        d[0] = u0.x; d[1] = u0.y; d[2] = u0.z; d[3] = u0.w;
        d[4] = u1.x; d[5] = u1.y; d[6] = u1.z; d[7] = u1.w;
    }
}

// One chunk of an anchored 1D archive decoded straight to values: q is the
// running prequantized integer (from the chunk's anchor), each value is
// fl(2eb * fl(q)) as in the separate reconstruction, and the eight values of
// a batch leave in one 32-byte store.
template <bool GUARD, bool FT_SMEM>
__device__ __forceinline__ void decode_chunk_values(const DecodeArgs &a, FastRing &rg, Window &w,
                                                    const uint2 *l1, const uint16_t *ft, uint32_t shift, uint64_t s0,
                                                    uint32_t cnt, uint32_t kend, uint32_t &q, OutlierCursor &oc,
                                                    uint4 *stg0, uint4 *stg1, bool al32, bool &bad,
                                                    unsigned long long &zeros, uint32_t &minlen)
{
    const float ebx2 = a.ebx2;
    float *out = a.out + s0;
    for (uint32_t k = 0; k < kend; k += kBatch) {
        rg.refill(w.v);
        uint32_t pw[kBatch / 2], zfl = 0;
        if (k + kBatch <= kend) {
#pragma unroll
            for (int j = 0; j < (int)kBatch; j += 2) {
                uint32_t zf;
                pw[j / 2] = decode_two<FT_SMEM, true, FastRing>(w, rg, l1, ft, shift, minlen,
                                                                   !GUARD || k + j < cnt, !GUARD || k + j + 1 < cnt,
                                                                   &zf);
                zfl |= zf << j;
            }
        } else {  // the warp's last, partial batch: one code at a time
#pragma unroll
            for (int j = 0; j < (int)kBatch; j++) {
                const uint32_t sy =
                    k + j < kend ? decode_two_level<FT_SMEM, true, FastRing>(w, rg, l1, ft, shift, minlen, k + j < cnt)
                                 : 1u;
                pw[j / 2] = (j & 1) ? pw[j / 2] | (sy << 16) : sy;
                zfl |= (sy == 0 ? 1u : 0u) << j;
            }
        }
        const uint32_t cnt8 = !GUARD || k + kBatch <= cnt ? kBatch : (k < cnt ? cnt - k : 0u);
        uint32_t d[8];
        residuals8(a, pw, cnt8, s0 + k, zfl, d, oc, stg0, stg1, bad, zeros);
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            q += d[j];
            v[j] = recon_value((int32_t)q, ebx2);
        }
        if (cnt8 == kBatch) {
            if (GBSZ_CHECK(s0 + k + kBatch <= a.n, a.ctl)) store8(out + k, v, al32);
        } else {
#pragma unroll
            for (int j = 0; j < 8; j++)
                if ((uint32_t)j < cnt8 && GBSZ_CHECK(s0 + k + j < a.n, a.ctl)) out[k + j] = v[j];
        }
    }
}

// The complete-table decoder with the 1D reconstruction fused in (anchored
// archives): every lane starts its chunk at the chunk's anchor and its first
// outlier entry, and afterwards checks that it consumed exactly its bits and
// its outlier entries and reached the next chunk's anchor.
template <bool FT_SMEM>
__device__ __forceinline__ void decode_fast_values_body(const DecodeArgs &a, VGrid vg)
{
    // rings, level-1 table (lane-replicated), staging slots, and with FT_SMEM
    // the complete table (2^fast_bits 16-bit entries)
    extern __shared__ uint32_t s_dyn[];
    uint2 *l1tab = reinterpret_cast<uint2 *>(s_dyn + blockDim.x * kRingFast);
    uint4 *s_stage = reinterpret_cast<uint4 *>(l1tab + (kL1Copies << kL1Bits));
    const uint16_t *ft = static_cast<const uint16_t *>(a.lutf);
    if (FT_SMEM) {
        uint4 *s_ft = s_stage + 2 * blockDim.x;
        // 2^fast_bits entries of 2 bytes in 16-byte pieces (at least one: the
        // table's buffer holds 2^15 entries)
        const uint4 *g_ft = static_cast<const uint4 *>(a.lutf);
        const uint32_t pieces = ((1u << a.fast_bits) + 7) >> 3;
        for (uint32_t i = threadIdx.x; i < pieces; i += blockDim.x) s_ft[i] = g_ft[i];
        ft = reinterpret_cast<const uint16_t *>(s_ft);  // visible after build_level1's barriers
    }
    build_level1<true>(a, s_dyn, l1tab);
    if (a.ctl->error & DERR_CORRUPT) return;
    const uint32_t shift = 32 - a.fast_bits;
    const uint32_t *stream = reinterpret_cast<const uint32_t *>(a.archive + a.off_stream);
    const uint32_t *bits_tab = reinterpret_cast<const uint32_t *>(a.archive + a.off_bits);
    uint32_t *warp_ring = s_dyn + (threadIdx.x >> 5) * kRingFast * 32;
    uint4 *stg0 = s_stage + threadIdx.x, *stg1 = s_stage + blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31;
    const uint2 *l1 = l1tab + lane % kL1Copies;
    const bool al32 = (reinterpret_cast<uintptr_t>(a.out) & 31) == 0;
    unsigned long long zeros = 0;
    bool bad = false;
    const uint64_t stride = (uint64_t)vg.nb * blockDim.x;
    for (uint64_t cw = (uint64_t)vg.bid * blockDim.x + threadIdx.x - lane; cw < a.nchunk; cw += stride) {
        const uint64_t c = cw + lane;
        const bool live = c < a.nchunk;
        const uint32_t nbits = live ? bits_tab[c] : 0u;
        const uint64_t coff = live ? a.chunk_off[c] : 0u;
        const uint64_t s0 = live ? c * a.chunk : 0u;
        const uint32_t cnt = live ? (uint32_t)(a.n - s0 < a.chunk ? a.n - s0 : a.chunk) : 0u;
        uint32_t q = live ? a.anchors[c] : 0u;
        OutlierCursor oc;
        oc.op = live ? a.ostart[c] : 0u;
        oc.oend = live ? a.ostart[c + 1] : 0u;
        if (oc.oend > a.m || oc.op > oc.oend) {  // (the start kernel flags a bad list; never read past it)
            bad = true;
            oc.op = oc.oend = 0;
        }
        oc.fetch(a);
        FastRing rg;
        rg.start(warp_ring, lane, stream + coff, coff < a.words ? a.words - coff : 0);
        Window w{0, 0, rg.at(0), rg.at(1), rg.at(2), rg.at(3)};
        uint32_t minlen = 15;
        if (__all_sync(0xffffffffu, cnt == a.chunk)) {
            decode_chunk_values<false, FT_SMEM>(a, rg, w, l1, ft, shift, s0, cnt, cnt, q, oc, stg0, stg1, al32, bad,
                                                zeros, minlen);
        } else {
            const uint32_t cmax = __reduce_max_sync(0xffffffffu, cnt);
            decode_chunk_values<true, FT_SMEM>(a, rg, w, l1, ft, shift, s0, cnt, cmax, q, oc, stg0, stg1, al32, bad,
                                               zeros, minlen);
        }
        cp_async_wait<0>();  // the ring is reused by the next chunk
        if (live) {
            bad |= minlen == 0 || (uint64_t)w.v * 32 + w.bo != nbits || oc.op != oc.oend;
            if (c == 0) bad |= a.anchors[0] != 0u;
            if (c + 1 < a.nchunk) bad |= a.anchors[c + 1] != q;  // the next chunk starts where this one ends
        }
        __syncwarp();
    }
    if (bad) atomicOr(&a.ctl->error, DERR_CORRUPT);
    if (zeros) atomicAdd(&a.ctl->zeros, zeros);
}

// Launched either as one block per SM of 32 x ceil(warps / SMs) threads (at
// most 1024), so that every SM and every scheduler gets the same number of
// chunks to within one warp, or, for more chunks than that, as the persistent
// 512-thread blocks of k_decode_fast (see launch_decode).
template <bool FT_SMEM>
__global__ void __launch_bounds__(kFastValuesMaxThreads, 1) k_decode_fast_values(const __grid_constant__ DecodeArgs a)
{
    decode_fast_values_body<FT_SMEM>(a, vgrid_self());
}

// rings, level-1 copies and the two staging slots of every thread
constexpr size_t fast_values_smem(uint32_t threads, uint32_t ft_bits = 0)
{
    return (size_t)threads * kRingFast * 4 + 8u * kL1Copies * (1u << kL1Bits) + 2u * threads * 16u +
           (ft_bits ? ((2u << ft_bits) + 15u) / 16u * 16u : 0u);
}

// each chunk's first outlier (see launch_outlier_chunk_starts)
__global__ void k_outlier_chunk_starts(const uint2 *outl, uint64_t m, uint64_t n, uint32_t chunk, uint32_t nchunk,
                                       uint32_t *ostart, Control *ctl)
{
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < m; t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t idx = outl[t].x;
        bool ok = idx < n;
        int64_t gprev = -1;
        if (t > 0) {
            const uint32_t pidx = outl[t - 1].x;
            ok &= idx > pidx;
            gprev = (int64_t)(pidx / chunk);
        }
        if (!ok) {
            atomicOr(&ctl->error, DERR_CORRUPT);
            continue;
        }
        const int64_t g = (int64_t)(idx / chunk);
        for (int64_t u = gprev + 1; u <= g; u++)
            if (GBSZ_CHECK((uint64_t)u <= nchunk, ctl)) ostart[u] = (uint32_t)t;
        if (t + 1 == m)
            for (uint64_t u = (uint64_t)g + 1; u <= nchunk; u++) ostart[u] = (uint32_t)m;
    }
}

// grouped decoders: one launch per variant over every field of the variant
template <bool FAST, bool MULTI_TILE>
__global__ void __launch_bounds__(FAST ? kDecFastThreads : kDecThreads, FAST ? 2 : 1)
    k_decode_group(const DecodeItem *items, const uint32_t *first, uint32_t ni)
{
    VGrid vg;
    const DecodeItem &d = items[group_item(first, ni, vg)];
    if (FAST) decode_fast_body<MULTI_TILE>(d.a, vg);
    else decode_general_body<MULTI_TILE>(d.a, d.sorted_in_smem, vg);
}

}  // namespace

int launch_decode(const DecodeArgs &a, cudaStream_t st, int phase)
{
    const ChunkWords op = chunk_words_op(a);
    if (phase == 0) return launch_scan(op, a.nchunk, a.scan_partial, a.ctl, st);
    DecodeItem it;
    int variant;
    size_t dyn;
    const unsigned g = decode_plan(a, &it, &variant, &dyn);
    if (phase == 2) {
        // the values straight from the complete-table decoder.  When every
        // chunk fits one wave: one block per SM of 32 x ceil(warps / SMs)
        // threads, so that every SM and every scheduler gets the same number
        // of chunks to within one warp.  Measured on 2^28 points in 131 072
        // chunks: 0.557 ms as 256 blocks of 512 threads (which leave 48 of
        // 152 SMs with half the others' work), 0.532 ms as 152 blocks of 864.
        // (The decoder writing codes measured 0.504 against 0.510 ms the same
        // way and keeps its 512-thread blocks.)
        const uint64_t sms = (uint64_t)(a.num_sms ? a.num_sms : 1);
        const uint64_t per_sm = ((a.nchunk + 31) / 32 + sms - 1) / sms;  // warps of chunks per SM
        if (per_sm * 32 <= (uint64_t)kFastValuesMaxThreads) {
            // one block per SM leaves room for the complete table in shared
            // memory, so codes longer than 8 bits are looked up there
            const uint32_t t = (uint32_t)per_sm * 32;
            k_decode_fast_values<true>
                <<<(unsigned)((a.nchunk + t - 1) / t), t, fast_values_smem(t, a.fast_bits), st>>>(a);
        } else {
            k_decode_fast_values<false><<<g, kDecFastThreads, fast_values_smem(kDecFastThreads), st>>>(a);
        }
        return 1;
    }
    const bool multi = variant & 1;
    if (variant & 2) {
        if (multi) k_decode_fast<true><<<g, kDecFastThreads, dyn, st>>>(a);
        else k_decode_fast<false><<<g, kDecFastThreads, dyn, st>>>(a);
    } else {
        if (multi) k_decode<true><<<g, kDecThreads, dyn, st>>>(a, it.sorted_in_smem);
        else k_decode<false><<<g, kDecThreads, dyn, st>>>(a, it.sorted_in_smem);
    }
    return 1;
}

namespace {

// opt in to the dynamic shared memory of the decoders, once per device
// (host threads may race here: the bits are atomic, and setting an
// attribute twice is harmless)
void set_decode_smem(int dev)
{
    static std::atomic<unsigned long long> attr_done{0};  // one bit per device id < 64
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0;
    if (bit && (attr_done.load() & bit)) return;
    const int most = (int)(kDecThreads * kRing * 4 + kSortedSmemMax * sizeof(uint16_t));
    const int most_fast = (int)(kDecFastThreads * kRingFast * 4 + 8u * kL1Copies * (1u << kL1Bits));
    cudaFuncSetAttribute(k_decode<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    cudaFuncSetAttribute(k_decode<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    cudaFuncSetAttribute(k_decode_fast<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most_fast);
    cudaFuncSetAttribute(k_decode_fast<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, most_fast);
    cudaFuncSetAttribute(k_decode_fast_values<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fast_values_smem(kFastValuesMaxThreads, kFastLutMax));
    cudaFuncSetAttribute(k_decode_fast_values<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)fast_values_smem(kDecFastThreads));
    cudaFuncSetAttribute(k_decode_group<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    cudaFuncSetAttribute(k_decode_group<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    cudaFuncSetAttribute(k_decode_group<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most_fast);
    cudaFuncSetAttribute(k_decode_group<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, most_fast);
    attr_done.fetch_or(bit);
}

}  // namespace

unsigned decode_plan(const DecodeArgs &a, DecodeItem *it, int *variant, size_t *dyn_out)
{
    int dev = 0;
    cudaGetDevice(&dev);
    set_decode_smem(dev);
    it->a = a;
    const uint64_t ntask = (a.nchunk + 31) / 32;
    const uint32_t nb = 2 * a.radius;
    const uint32_t in_smem = nb <= kSortedSmemMax ? nb : 0u;
    it->sorted_in_smem = in_smem;
    const bool multi = a.chunk > kRecon1DTile;
    const uint64_t sms = (uint64_t)(a.num_sms ? a.num_sms : 1);
    if (a.fast_bits) {
        *variant = 2 + (multi ? 1 : 0);
        *dyn_out = (size_t)kDecFastThreads * kRingFast * 4 + 8u * kL1Copies * (1u << kL1Bits);
        const uint64_t want = (a.nchunk + kDecFastThreads - 1) / kDecFastThreads;
        return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, sms * 2));
    }
    *variant = multi ? 1 : 0;
    *dyn_out = (size_t)kDecThreads * kRing * 4 + in_smem * sizeof(uint16_t);
    // persistent: as many blocks as are resident at once.  k_decode blocks
    // resident per SM, by device, MULTI_TILE and the sorted table's size in
    // shared memory (steps of 512 symbols); 0: not queried yet
    static std::atomic<int> resident[64][2][kSortedSmemMax / 512 + 1];
    const uint32_t qb = (in_smem + 511) / 512;
    int per_sm = 1;
    if (dev >= 0 && dev < 64) {
        std::atomic<int> &r = resident[dev][multi ? 1 : 0][qb];
        if (r.load() == 0) {
            const size_t dq = (size_t)kDecThreads * kRing * 4 + (size_t)qb * 512 * sizeof(uint16_t);
            int blocks = 0;
            const cudaError_t e =
                multi ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_decode<true>, kDecThreads, dq)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_decode<false>, kDecThreads, dq);
            if (e != cudaSuccess) {
                cudaGetLastError();
                blocks = 0;
            }
            r.store(blocks > 0 ? blocks : 1);
        }
        per_sm = r.load();
    }
    return (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(ntask, sms * per_sm));
}

void launch_decode_group(int variant, const DecodeItem *items, const uint32_t *first, uint32_t ni, uint32_t blocks,
                         size_t dyn, cudaStream_t st)
{
    switch (variant) {
    case 0: k_decode_group<false, false><<<blocks, kDecThreads, dyn, st>>>(items, first, ni); break;
    case 1: k_decode_group<false, true><<<blocks, kDecThreads, dyn, st>>>(items, first, ni); break;
    case 2: k_decode_group<true, false><<<blocks, kDecFastThreads, dyn, st>>>(items, first, ni); break;
    case 3: k_decode_group<true, true><<<blocks, kDecFastThreads, dyn, st>>>(items, first, ni); break;
    default: break;
    }
}

int launch_offsets_scan_group(const ScanItem<ChunkWords> *items, const uint32_t *first, uint32_t ni, uint32_t blocks,
                              cudaStream_t st)
{
    return launch_scan_group(items, first, ni, blocks, st);
}

int launch_outlier_chunk_starts(const uint2 *outl, uint64_t m, uint64_t n, uint32_t chunk, uint32_t nchunk,
                                uint32_t *ostart, Control *ctl, cudaStream_t st)
{
    if (m == 0) {  // every chunk starts (and ends) at entry 0
        cudaMemsetAsync(ostart, 0, ((size_t)nchunk + 1) * 4, st);
        return 0;
    }
    const uint64_t want = (m + 255) / 256;
    // (a version reading each record once and taking the previous index from
    // the neighbouring lane, with one block per 256 records, measured slower:
    // 20.7 -> 24.5 us for 4.3e6 records)
    k_outlier_chunk_starts<<<(unsigned)std::min<uint64_t>(want, 4096), 256, 0, st>>>(outl, m, n, chunk, nchunk,
                                                                                      ostart, ctl);
    return 1;
}

namespace {
struct HeaderWords {
    uint32_t w[kHeaderBytes / 4];  // 32: one per lane
};

// one warp: the archive's header word by word against the copy the
// decompression was planned from
__global__ void k_header_check(const uint32_t *arc, const __grid_constant__ HeaderWords expect, Control *ctl)
{
    const uint32_t lane = threadIdx.x & 31;
    const bool differs = arc[lane] != expect.w[lane];
    if (__any_sync(0xffffffffu, differs) && lane == 0) atomicOr(&ctl->error, DERR_STALE);
}
}  // namespace

void launch_header_check(const void *arc, const uint8_t *expect, Control *ctl, cudaStream_t st)
{
    static_assert(kHeaderBytes == 128, "one header word per lane");
    HeaderWords h;
    memcpy(h.w, expect, kHeaderBytes);
    k_header_check<<<1, 32, 0, st>>>(static_cast<const uint32_t *>(arc), h, ctl);
}

}  // namespace gbsz
