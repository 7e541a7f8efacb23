// k_decode.cu -- S7: Huffman decode (inflate, Sec. 3.3).
//
// Chunk word offsets are the exclusive prefix sum of ceil(bits/32) over the
// archive's chunk table (three coalesced scan kernels).  Decoding is
// sequential inside a chunk, as in the paper; one thread decodes one chunk.
// Each thread keeps a 32-word ring of its chunk's stream in shared memory,
// filled eight words at a time by cp.async (issued about two quarters before
// the words are needed, so refills never stall the decode), and a bit window
// of three registers (current word, next word, one look-ahead) advanced with
// selects instead of branches.  A 4096-entry shared-memory table resolves
// every code of at most 12 bits in one lookup; longer codes fall back to the
// canonical per-length tables, also in shared memory.  Decoded codes leave in
// 16-byte stores.  Every chunk must consume exactly its recorded bit count and
// every code must exist in the codebook; anything else marks the archive
// corrupt.  For 1D fields the decoder also accumulates the residual sum of
// every 4096-point tile (in-cap codes only; outliers are added by the
// scatter), which the reconstruction scans instead of making another pass
// over the codes.
#include "common.cuh"
#include "scan.cuh"

#include <algorithm>

namespace gbsz {

namespace {

constexpr int kDecThreads = 256;
constexpr uint32_t kSortedSmemMax = 8192;  // symbols whose table is copied to shared memory

struct WordsOp {
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

constexpr uint32_t kRing = 32;       // stream words per thread in shared memory (any code length)
constexpr uint32_t kRingFast = 16;   // the same for codes of at most kFastLutMax bits
constexpr int kDecFastThreads = 512;
constexpr uint32_t kBatch = 8;       // symbols between refill checks

__device__ __forceinline__ void cp_async4(uint32_t *dst, const uint32_t *src)
{
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(src) : "memory");
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
            uint32_t *d = &at(v);
            if (v < avail) cp_async4(d, src + v);
            else *d = 0u;
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

// Bit window: hi, lo, q0, q1 = words v .. v+3.  The next 32 stream bits are
// funnelshift(lo, hi, bo).  Each step reads word v+4 from the ring before it
// looks at the table, so that read is not behind the lookup in the
// dependency chain, and shifts it in with selects if a word was consumed.
struct Window {
    uint32_t v, bo, hi, lo, q0, q1;
};

struct DecTables {
    const uint32_t *lut;
    const unsigned long long *first;
    const uint32_t *count, *start;
    const uint16_t *sorted;
    uint32_t maxlen;
};

template <uint32_t RW>
__device__ __forceinline__ void advance_one(Window &w, const Ring<RW> &rg)
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
    const uint32_t e = t.lut[cur >> (32 - kLutBits)];
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
                sym = t.sorted[t.start[l] + off];
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

template <bool MULTI_TILE>
__global__ void __launch_bounds__(kDecThreads) k_decode(DecodeArgs a, uint32_t sorted_in_smem)
{
    __shared__ uint32_t lut[1 << kLutBits];
    __shared__ unsigned long long first[kMaxLen + 2];
    __shared__ uint32_t count[kMaxLen + 2], start[kMaxLen + 2];
    extern __shared__ uint32_t s_dyn[];  // rings, then the sorted symbols
    uint16_t *s_sorted = reinterpret_cast<uint16_t *>(s_dyn + kDecThreads * kRing);
    for (uint32_t i = threadIdx.x; i < (1u << kLutBits); i += blockDim.x) lut[i] = a.lut[i];
    for (uint32_t i = threadIdx.x; i < kMaxLen + 2; i += blockDim.x) {
        first[i] = a.first[i];
        count[i] = a.count[i];
        start[i] = a.start[i];
    }
    for (uint32_t i = threadIdx.x; i < sorted_in_smem; i += blockDim.x) s_sorted[i] = a.sorted[i];
    __syncthreads();
    if (a.ctl->error & DERR_CORRUPT) return;
    const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.nchunk) return;
    DecTables t{lut, first, count, start, sorted_in_smem ? s_sorted : a.sorted, a.maxlen};
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
        *reinterpret_cast<uint4 *>(out + k) = o;
        tz += zeros_in(o.x) + zeros_in(o.y) + zeros_in(o.z) + zeros_in(o.w);
        if (MULTI_TILE && a.tile_sums && ((s0 + k + kBatch) & (kRecon1DTile - 1)) == 0) {
            // residual sum of the tile's in-cap codes: sum(code) - R * (#nonzero), mod 2^32
            const uint32_t m = k + kBatch - tstart;
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
            out[k] = (uint16_t)sym;
        }
    }
    zeros += tz;
    if (a.tile_sums && cnt > tstart) {
        const uint32_t tsum = ssum - R * (cnt - tstart - tz);
        if (tsum) atomicAdd(&a.tile_sums[(s0 + cnt - 1) / kRecon1DTile], tsum);
    }
    cp_async_wait<0>();  // nothing may still be landing in the ring when the block exits
    // a valid chunk ends exactly at its recorded bit count
    if (bad || (uint64_t)w.v * 32 + w.bo != nbits) atomicOr(&a.ctl->error, DERR_CORRUPT);
    if (zeros) atomicAdd(&a.ctl->zeros, (unsigned long long)zeros);
}

// One code from the 16-bit complete table: no long-code path, no branch.  A
// pattern that matches no code has entry 0 (length 0); the smallest length
// seen is checked after the chunk.
__device__ __forceinline__ uint32_t decode_single(Window &w, const Ring<kRingFast> &rg, const uint16_t *lut,
                                                  uint32_t shift, uint32_t &minlen)
{
    const uint32_t nxt = rg.at(w.v + 4);
    const uint32_t cur = __funnelshift_l(w.lo, w.hi, w.bo);
    const uint32_t e = lut[cur >> shift];
    const uint32_t len = e & 15u;
    minlen = min(minlen, len);
    step(w, nxt, len);
    return e >> 4;
}

// Two codes from the pair table: the entry of the first B bits gives the
// first code and, when it fits in those B bits, the second; otherwise the
// second comes from a lookup of the B bits after the first code (a
// predicated load, so lanes that need none leave the banks alone).
__device__ __forceinline__ void decode_pair(Window &w, const Ring<kRingFast> &rg, const uint32_t *lut,
                                            uint32_t shift, uint32_t &minlen, uint32_t &s1, uint32_t &s2)
{
    const uint32_t nxt = rg.at(w.v + 4);
    const uint32_t c0 = __funnelshift_l(w.lo, w.hi, w.bo);
    const uint32_t c1 = __funnelshift_l(w.q0, w.lo, w.bo);
    const uint32_t e = lut[c0 >> shift];
    const uint32_t l1 = e & 15u;
    const uint32_t cur2 = __funnelshift_l(c1, c0, l1);  // the 32 bits after the first code (l1 < 16)
    uint32_t e2 = e >> 4;                                // len2 | sym1 << 4 | sym2 << 16 as a fallback shape
    const uint32_t saddr = (uint32_t)__cvta_generic_to_shared(lut) + ((cur2 >> shift) << 2);
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.eq.u32 p, %1, 0;\n\t"
        "@p ld.shared.u32 %0, [%2];\n\t}"
        : "+r"(e2)
        : "r"((e >> 4) & 15u), "r"(saddr));
    // e2 is either the original entry shifted right by 4 (second code
    // present: its length in bits 0-3, symbol in bits 16-27) or a fresh
    // entry (first code of the later lookup: length bits 0-3, symbol 8-19)
    const bool second_inline = ((e >> 4) & 15u) != 0;
    const uint32_t l2 = e2 & 15u;
    s1 = (e >> 8) & 0xFFFu;
    s2 = second_inline ? (e2 >> 16) : ((e2 >> 8) & 0xFFFu);
    minlen = min(minlen, min(l1, l2));
    step(w, nxt, l1 + l2);
}

// Persistent decoder for archives whose codes all fit the complete table
// (at most kFastLutMax bits): each thread decodes chunks c, c + grid, ...
template <bool MULTI_TILE, bool PAIR>
__global__ void __launch_bounds__(kDecFastThreads, 2) k_decode_fast(DecodeArgs a)
{
    extern __shared__ uint32_t s_dyn[];  // rings, then the table
    uint32_t *tab = s_dyn + kDecFastThreads * kRingFast;
    const uint32_t B = a.fast_bits, shift = 32 - B;
    const uint32_t tab_words = PAIR ? (1u << B) : ((1u << B) + 1) / 2;
    for (uint32_t i = threadIdx.x; i < tab_words; i += blockDim.x) tab[i] = static_cast<const uint32_t *>(a.lutf)[i];
    __syncthreads();
    if (a.ctl->error & DERR_CORRUPT) return;
    const uint32_t *stream = reinterpret_cast<const uint32_t *>(a.archive + a.off_stream);
    const uint32_t *bits_tab = reinterpret_cast<const uint32_t *>(a.archive + a.off_bits);
    const uint32_t R = a.radius;
    uint32_t *warp_ring = s_dyn + (threadIdx.x >> 5) * kRingFast * 32;
    const uint32_t lane = threadIdx.x & 31;
    unsigned long long zeros = 0;
    bool bad = false;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint32_t nbits = 0;
    uint64_t coff = 0;
    if (c < a.nchunk) {
        nbits = bits_tab[c];
        coff = a.chunk_off[c];
    }
    for (; c < a.nchunk; c += stride) {
        // the next chunk's bit count and offset are fetched while this one decodes
        const uint64_t cn = c + stride;
        uint32_t nbits_n = 0;
        uint64_t coff_n = 0;
        if (cn < a.nchunk) {
            nbits_n = bits_tab[cn];
            coff_n = a.chunk_off[cn];
        }
        const uint64_t s0 = c * a.chunk;
        const uint32_t cnt = (uint32_t)(a.n - s0 < a.chunk ? a.n - s0 : a.chunk);
        Ring<kRingFast> rg;
        rg.start(warp_ring, lane, stream + coff, coff < a.words ? a.words - coff : 0);
        Window w{0, 0, rg.at(0), rg.at(1), rg.at(2), rg.at(3)};
        uint32_t ssum = 0, tz = 0, tstart = 0, minlen = 15;
        uint16_t *out = a.codes + s0;
        const uint32_t full = cnt & ~(kBatch - 1);
        for (uint32_t k = 0; k < full; k += kBatch) {
            rg.refill(w.v);
            uint32_t sy[kBatch];
            if (PAIR) {
#pragma unroll
                for (int j = 0; j < (int)kBatch; j += 2)
                    decode_pair(w, rg, tab, shift, minlen, sy[j], sy[j + 1]);
            } else {
#pragma unroll
                for (int j = 0; j < (int)kBatch; j++)
                    sy[j] = decode_single(w, rg, reinterpret_cast<const uint16_t *>(tab), shift, minlen);
            }
            const uint4 o = make_uint4(sy[0] | (sy[1] << 16), sy[2] | (sy[3] << 16), sy[4] | (sy[5] << 16),
                                       sy[6] | (sy[7] << 16));
            // symbols are below 4096 here, so the halves of the word sum cannot carry
            const uint32_t t4 = o.x + o.y + o.z + o.w;
            ssum += (t4 & 0xFFFFu) + (t4 >> 16);
            *reinterpret_cast<uint4 *>(out + k) = o;
            tz += zeros_in(o.x) + zeros_in(o.y) + zeros_in(o.z) + zeros_in(o.w);
            if (MULTI_TILE && a.tile_sums && ((s0 + k + kBatch) & (kRecon1DTile - 1)) == 0) {
                // residual sum of the tile's in-cap codes: sum(code) - R * (#nonzero), mod 2^32
                const uint32_t m = k + kBatch - tstart;
                atomicAdd(&a.tile_sums[(s0 + k) / kRecon1DTile], ssum - R * (m - tz));
                zeros += tz;
                ssum = tz = 0;
                tstart = k + kBatch;
            }
        }
        if (full < cnt) {
            rg.refill(w.v);
            for (uint32_t k = full; k < cnt; k++) {
                const uint32_t sym =
                    PAIR ? 0u : decode_single(w, rg, reinterpret_cast<const uint16_t *>(tab), shift, minlen);
                uint32_t s = sym;
                if (PAIR) {
                    // one code: the first half of a pair entry
                    const uint32_t nxt = rg.at(w.v + 4);
                    const uint32_t cur = __funnelshift_l(w.lo, w.hi, w.bo);
                    const uint32_t e = tab[cur >> shift];
                    const uint32_t l1 = e & 15u;
                    minlen = min(minlen, l1);
                    step(w, nxt, l1);
                    s = (e >> 8) & 0xFFFu;
                }
                ssum += s;
                tz += s == 0;
                out[k] = (uint16_t)s;
            }
        }
        zeros += tz;
        if (a.tile_sums && cnt > tstart) {
            const uint32_t tsum = ssum - R * (cnt - tstart - tz);
            if (tsum) atomicAdd(&a.tile_sums[(s0 + cnt - 1) / kRecon1DTile], tsum);
        }
        cp_async_wait<0>();  // the ring is reused by the next chunk
        bad |= minlen == 0 || (uint64_t)w.v * 32 + w.bo != nbits;
        nbits = nbits_n;
        coff = coff_n;
    }
    if (bad) atomicOr(&a.ctl->error, DERR_CORRUPT);
    if (zeros) atomicAdd(&a.ctl->zeros, zeros);
}

}  // namespace

int launch_decode(const DecodeArgs &a, cudaStream_t st, int phase)
{
    WordsOp op;
    op.bits = reinterpret_cast<const uint32_t *>(a.archive + a.off_bits);
    op.off = a.chunk_off;
    op.words = a.words;
    op.maxbits = (unsigned long long)a.chunk * kMaxLen;
    op.ctl = a.ctl;
    if (phase == 0) return launch_scan(op, a.nchunk, a.scan_partial, st);
    const uint64_t grid = (a.nchunk + kDecThreads - 1) / kDecThreads;
    const uint32_t nb = 2 * a.radius;
    const uint32_t in_smem = nb <= kSortedSmemMax ? nb : 0u;
    const size_t dyn = (size_t)kDecThreads * kRing * 4 + in_smem * sizeof(uint16_t);
    static unsigned long long attr_done = 0;  // one bit per device id < 64
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0;
    if (!bit || !(attr_done & bit)) {
        const int most = (int)(kDecThreads * kRing * 4 + kSortedSmemMax * sizeof(uint16_t));
        cudaFuncSetAttribute(k_decode<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        cudaFuncSetAttribute(k_decode<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
        const int most_fast = (int)(kDecFastThreads * kRingFast * 4 + kFastLutBytes);
        cudaFuncSetAttribute(k_decode_fast<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most_fast);
        cudaFuncSetAttribute(k_decode_fast<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, most_fast);
        cudaFuncSetAttribute(k_decode_fast<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, most_fast);
        cudaFuncSetAttribute(k_decode_fast<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, most_fast);
        attr_done |= bit;
    }
    const bool multi = a.chunk > kRecon1DTile;
    if (a.fast_bits) {
        const size_t tab = a.fast_pair ? (4u << a.fast_bits) : (((2u << a.fast_bits) + 3) & ~3u);
        const size_t dyn_fast = (size_t)kDecFastThreads * kRingFast * 4 + tab;
        const uint64_t want = (a.nchunk + kDecFastThreads - 1) / kDecFastThreads;
        const unsigned g = (unsigned)std::min<uint64_t>(want, (uint64_t)(a.num_sms ? a.num_sms : 1) * 2);
        if (a.fast_pair) {
            if (multi) k_decode_fast<true, true><<<g, kDecFastThreads, dyn_fast, st>>>(a);
            else k_decode_fast<false, true><<<g, kDecFastThreads, dyn_fast, st>>>(a);
        } else {
            if (multi) k_decode_fast<true, false><<<g, kDecFastThreads, dyn_fast, st>>>(a);
            else k_decode_fast<false, false><<<g, kDecFastThreads, dyn_fast, st>>>(a);
        }
    } else if (multi) {
        k_decode<true><<<(unsigned)grid, kDecThreads, dyn, st>>>(a, in_smem);
    } else {
        k_decode<false><<<(unsigned)grid, kDecThreads, dyn, st>>>(a, in_smem);
    }
    return 1;
}

}  // namespace gbsz
