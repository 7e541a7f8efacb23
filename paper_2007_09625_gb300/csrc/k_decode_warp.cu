// k_decode_warp.cu -- S7 (Sec. 3.3) with one warp per Huffman chunk, and for
// 1D order-1 fields S8 (Algorithm 2's decompression loop) in the same pass.
//
// The archive has one entry point per chunk (Sec. 3.2.4: every chunk is
// deflated on its own and starts on a word).  The thread-per-chunk decoders
// walk a chunk as one serial chain; here the 32 lanes of a warp split the
// chunk's bits into 32 equal ranges and decode them together.  A range
// generally starts inside a codeword, but a prefix code falls back into step
// with the true codeword boundaries after a few codewords (most codes are
// self-synchronising), so:
//   1. every lane decodes its range from the range's first bit, noting the
//      codeword starts it passes in its first 64 bits and where its last
//      codeword ends (the first start at or past the range's end);
//   2. lane i's true first codeword starts where lane i-1's true path ended.
//      From there lane i follows the true codewords until one starts where
//      its own path had a start: from that point on its path is the true one
//      (in practice after a few codewords; past the 64 noted bits it follows
//      the true codewords to the range's end).  Rounds repeat until no
//      lane's true start moves: lane 0 is exact (it starts at bit 0), so
//      after round k lanes 0..k are settled -- at most 32 rounds, in
//      practice two (the first finds the starts, the second sees no move);
//   3. an exclusive warp scan of the lanes' codeword counts places every
//      lane's symbols, and each lane decodes its codewords once more into
//      the warp's chunk buffer in shared memory.
// A chunk is valid when its codewords cover exactly its recorded bit count,
// number exactly its symbols and are all codes of the table: the conditions
// the thread-per-chunk decoders check.
//
// Fused S8 (1D, order 1, whole-field Lorenzo): the reconstruction is then an
// inclusive prefix sum of the residuals along the field.  Each chunk's
// in-cap residual sum and code-0 count are published for a decoupled
// look-back over chunks (warps take chunks in order from a ticket counter,
// so every chunk a warp waits for is held by a running warp; a wait longer
// than 1 s gives up and the call reports a timeout).  The residuals of the outliers before the
// chunk come from an exclusive scan of the outlier list's residuals at the
// code-0 count before the chunk; the chunk's own outliers are matched, in
// order, to its code-0 points.  Values leave as floats with coalesced 16-byte
// stores; codes never reach global memory.
#include <algorithm>
#include <atomic>

#include "common.cuh"
#include "scan.cuh"

namespace gbsz {
namespace {

constexpr uint32_t kWThreads = 256;  // 8 warps per block, one chunk each at a time
constexpr uint32_t kWWarps = kWThreads / 32;
// first-level table: the code at the start of each byte value when it has at
// most 8 bits, and the code after it when that also fits in the byte; 8-byte
// entries replicated 16 times (entry i of copy c at slot 16 i + c, lane l
// reading copy l % 16), so the 16 lanes that one 8-byte shared access serves
// read 16 different copies in 32 different banks and never conflict
constexpr uint32_t kWL1Bits = 8, kWL1Copies = 16;
constexpr size_t kWTableBytes = 8u * kWL1Copies * (1u << kWL1Bits);
constexpr uint32_t kWSortedSmem = 4096;  // canonical symbol table in shared memory up to this many bins
static_assert(4u * (1u << kLutBits) + 2u * kLut2Entries + 16u * (kMaxLen + 2) + 2u * kWSortedSmem <= kWTableBytes,
              "the general tables fit the table area");
// look-back word: flag << 62 | code-0 count (30 bits) << 32 | in-cap residual sum
constexpr unsigned long long kLbAgg = 1ull << 62, kLbInc = 2ull << 62;
constexpr unsigned long long kLbWaitNs = 1000000000ull;  // a look-back gives up after waiting 1 s
constexpr uint32_t kNone = 0xFFFFFFFFu;

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void st_relaxed(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// A lane's view of the chunk's bits: the next bits at the top of buf (at
// least 32 valid between steps), the following word loaded ahead.  Words past
// the stream's end read as 0.
struct Bits {
    const uint32_t *w;  // the chunk's first word
    uint32_t avail;     // words readable from w
    uint64_t buf;
    uint32_t nb, k, nxt, pos;  // valid bits, index of nxt, next word, position of the top bit
    __device__ __forceinline__ uint32_t ld(uint32_t i) const { return i < avail ? __ldg(w + i) : 0u; }
    __device__ __forceinline__ void seek(uint32_t p)
    {
        const uint32_t i = p >> 5, o = p & 31u;
        buf = (((uint64_t)ld(i) << 32) | ld(i + 1)) << o;
        nb = 64 - o;
        k = i + 2;
        nxt = ld(k);
        pos = p;
    }
    __device__ __forceinline__ uint32_t top() const { return (uint32_t)(buf >> 32); }
    // the next 64 bits (buf's valid bits, then the word after them)
    __device__ __forceinline__ uint64_t view64() const { return buf | ((uint64_t)nxt >> (nb - 32)); }
    // l <= 16
    __device__ __forceinline__ void skip(uint32_t l)
    {
        buf <<= l;
        nb -= l;
        pos += l;
        if (nb < 32) {
            buf |= (uint64_t)nxt << (32 - nb);
            nb += 32;
            k++;
            nxt = ld(k);
        }
    }
    // any l (codes of up to kMaxLen bits)
    __device__ __forceinline__ void skip_any(uint32_t l)
    {
        while (l > 16) {
            skip(16);
            l -= 16;
        }
        skip(l);
    }
};

// One or two codes at the top of the window.  l1 = 0 after the lookup: no
// code matches (an invalid pattern).  l2 = 0: no second code in the byte.
struct Codes {
    uint32_t s1, l1, s2, l2;
};

// Codes of at most 15 bits and symbols below 4096: the replicated first-level
// table, then the complete table in global memory for codes of 9..15 bits.
struct FastLK {
    static constexpr bool kLong = false;
    const uint2 *l1;  // this lane's copy
    const uint16_t *ft;
    uint32_t shift;
    __device__ __forceinline__ Codes operator()(const Bits &b) const
    {
        const uint32_t top = b.top();
        const uint2 e = l1[(top >> (32 - kWL1Bits)) * kWL1Copies];
        Codes c{e.x & 0xFFFFu, e.y & 0xFFu, e.x >> 16, e.y >> 8};
        if (c.l1 == 0) {  // longer than 8 bits: the complete table (entries (sym << 4) | len)
            const uint32_t f = __ldg(ft + (top >> shift));
            c.l1 = f & 15u;
            c.s1 = f >> 4;
            c.l2 = 0;
        }
        return c;
    }
};

// Any codebook: the 12-bit first level and the second level for codes of up
// to 16 bits (both in shared memory), then the canonical tables (codes of
// length l are the values first[l] .. first[l] + count[l] - 1 of their l
// bits, standing for sorted[start[l] ..], Sec. 3.2.3) for longer codes.
struct GeneralLK {
    static constexpr bool kLong = true;
    const uint32_t *lut;
    const uint16_t *lut2;
    uint32_t l2lo;
    const unsigned long long *first;
    const uint32_t *count, *start;
    const uint16_t *sorted;
    uint32_t maxlen;
    __device__ __forceinline__ Codes operator()(const Bits &b) const
    {
        const uint32_t cur = b.top();
        uint32_t e = lut[cur >> (32 - kLutBits)];
        if (e == 0) {
            const uint32_t j = (cur >> (32 - kLutBits)) - l2lo;
            const uint32_t e2 =
                j < kLut2Prefixes ? lut2[(j << kLut2Bits) | ((cur >> (32 - kLutBits - kLut2Bits)) & ((1u << kLut2Bits) - 1))]
                                  : 0u;
            e = ((e2 >> 5) << 8) | (e2 & 31u);
        }
        Codes c{e >> 8, e & 0xFFu, 0u, 0u};
        if (e == 0) {
            const uint64_t v = b.view64();
            for (uint32_t l = kLutBits + 1; l <= maxlen; l++) {
                const unsigned long long off = (v >> (64 - l)) - first[l];
                if (off < count[l]) {
                    c.l1 = l;
                    c.s1 = sorted[start[l] + off];
                    break;
                }
            }
        }
        return c;
    }
};

template <class LK>
__device__ __forceinline__ void consume(Bits &b, uint32_t l)
{
    if (LK::kLong) b.skip_any(l);
    else b.skip(l);
}

// A lane's decoded path: codewords starting in [start, stop).
struct Path {
    uint64_t mask;                  // codeword starts at offsets < 64 from start
    uint32_t start, cnt, end, bad;  // bad: first invalid start (kNone: none)
};

template <class LK>
__device__ __forceinline__ void run_path(Bits &b, uint32_t start, uint32_t stop, const LK &lk, Path &p)
{
    b.seek(start);
    p.start = start;
    p.cnt = 0;
    p.mask = 0;
    p.bad = kNone;
    // the first 64 bits noting the starts, then the rest without
    const uint32_t mstop = min(stop, start + 64);
    while (b.pos < mstop) {
        Codes c = lk(b);
        const uint32_t off = b.pos - start;
        p.mask |= 1ull << off;
        if (c.l1 == 0) {  // an invalid pattern: note it and move on by one bit
            p.bad = min(p.bad, b.pos);
            c.l1 = 1;
            c.l2 = 0;
        }
        uint32_t adv = c.l1;
        p.cnt++;
        if (c.l2 && b.pos + c.l1 < stop) {
            const uint32_t off2 = off + c.l1;
            if (off2 < 64) p.mask |= 1ull << off2;
            adv += c.l2;
            p.cnt++;
        }
        consume<LK>(b, adv);
    }
    while (b.pos < stop) {
        Codes c = lk(b);
        if (c.l1 == 0) {
            p.bad = min(p.bad, b.pos);
            c.l1 = 1;
            c.l2 = 0;
        }
        uint32_t adv = c.l1;
        p.cnt++;
        if (c.l2 && b.pos + c.l1 < stop) {
            adv += c.l2;
            p.cnt++;
        }
        consume<LK>(b, adv);
    }
    p.end = b.pos;
}

// the first-level table from the complete one (B = fast_bits index bits)
__device__ __forceinline__ void build_l1(uint2 *l1tab, const uint16_t *ft, uint32_t B)
{
    auto ft_at = [&](uint32_t byte) -> uint32_t {
        return B >= kWL1Bits ? ft[byte << (B - kWL1Bits)] : ft[byte >> (kWL1Bits - B)];
    };
    for (uint32_t k = threadIdx.x; k < (kWL1Copies << kWL1Bits); k += blockDim.x) {
        const uint32_t i = k / kWL1Copies;
        const uint32_t f = ft_at(i);
        const uint32_t la = f & 15u;
        uint2 e = make_uint2(0u, 0u);
        if (la >= 1 && la <= kWL1Bits) {
            e = make_uint2(f >> 4, la);
            if (la < kWL1Bits) {
                const uint32_t g2 = ft_at((i << la) & 0xFFu);
                const uint32_t lb = g2 & 15u;
                if (lb >= 1 && lb <= kWL1Bits - la) e = make_uint2((f >> 4) | ((g2 >> 4) << 16), la | (lb << 8));
            }
        }
        l1tab[k] = e;
    }
}

// the lookup's tables in the block's table area of shared memory (kWTableBytes)
__device__ __forceinline__ FastLK make_lk(const DecodeArgs &a, uint4 *area, FastLK *)
{
    uint2 *l1tab = reinterpret_cast<uint2 *>(area);
    const uint16_t *ft = static_cast<const uint16_t *>(a.lutf);
    build_l1(l1tab, ft, a.fast_bits);
    return FastLK{l1tab + (threadIdx.x & 31) % kWL1Copies, ft, 32 - a.fast_bits};
}

__device__ __forceinline__ GeneralLK make_lk(const DecodeArgs &a, uint4 *area, GeneralLK *)
{
    uint32_t *lut = reinterpret_cast<uint32_t *>(area);  // 16 KiB
    uint16_t *lut2 = reinterpret_cast<uint16_t *>(lut + (1u << kLutBits));  // 4 KiB
    unsigned long long *first = reinterpret_cast<unsigned long long *>(lut2 + kLut2Entries);
    uint32_t *count = reinterpret_cast<uint32_t *>(first + kMaxLen + 2);
    uint32_t *start = count + kMaxLen + 2;
    for (uint32_t i = threadIdx.x; i < (1u << kLutBits); i += blockDim.x) lut[i] = a.lut[i];
    const uint16_t *g2 = reinterpret_cast<const uint16_t *>(a.lut + (1u << kLutBits) + 1);
    for (uint32_t i = threadIdx.x; i < kLut2Entries; i += blockDim.x) lut2[i] = g2[i];
    for (uint32_t i = threadIdx.x; i < kMaxLen + 2; i += blockDim.x) {
        first[i] = a.first[i];
        count[i] = a.count[i];
        start[i] = a.start[i];
    }
    // the symbols of the canonical order, when they fit the rest of the area
    uint16_t *sorted = reinterpret_cast<uint16_t *>(start + kMaxLen + 2);
    const uint32_t nbins = 2 * a.radius;
    const bool in_smem = nbins <= kWSortedSmem;
    if (in_smem)
        for (uint32_t i = threadIdx.x; i < nbins; i += blockDim.x) sorted[i] = a.sorted[i];
    return GeneralLK{lut, lut2, a.lut[1u << kLutBits], first, count, start, in_smem ? sorted : a.sorted, a.maxlen};
}

template <bool FUSE, class LK>
__device__ __forceinline__ void decode_warp_body(const WarpDecodeArgs &wa)
{
    extern __shared__ uint4 s_w4[];
    const DecodeArgs &a = wa.d;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint16_t *cbuf = reinterpret_cast<uint16_t *>(reinterpret_cast<uint8_t *>(s_w4) + kWTableBytes) +
                     (size_t)warp * a.chunk;
    const LK lk = make_lk(a, s_w4, static_cast<LK *>(nullptr));
    __syncthreads();
    const uint32_t *stream = reinterpret_cast<const uint32_t *>(a.archive + a.off_stream);
    const uint32_t *bits_tab = reinterpret_cast<const uint32_t *>(a.archive + a.off_bits);
    const uint32_t R = a.radius;
    const bool al16 = (reinterpret_cast<uintptr_t>(FUSE ? (const void *)wa.out : (const void *)a.codes) & 15) == 0;
    volatile uint32_t *verr = &a.ctl->error;
    unsigned long long zeros = 0;
    bool bad = false, timeout = false;
    for (;;) {
        uint32_t c = kNone;
        if (lane == 0 && !(*verr & (DERR_CORRUPT | DERR_TIMEOUT))) c = atomicAdd(&a.ctl->ticket, 1u);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= a.nchunk) break;
        const uint32_t nbits = bits_tab[c];
        const uint64_t coff = a.chunk_off[c];
        const uint64_t s0 = (uint64_t)c * a.chunk;
        const uint32_t cnt = (uint32_t)(a.n - s0 < a.chunk ? a.n - s0 : a.chunk);
        Bits b;
        b.w = stream + coff;
        b.avail = coff < a.words ? (uint32_t)(a.words - coff < 0xFFFFFFFFull ? a.words - coff : 0xFFFFFFFFull) : 0u;
        const uint32_t lo = (uint32_t)(((uint64_t)lane * nbits) >> 5);
        const uint32_t stop = (uint32_t)(((uint64_t)(lane + 1) * nbits) >> 5);
        // 1. speculative paths
        Path p;
        run_path(b, lo, stop, lk, p);
        // 2. settle the lanes' true starts, lane 0 first
        uint32_t ts = lo, tc = p.cnt, tend = p.end;
        bool lane_bad = p.bad != kNone;
        bool settled = false;
        for (int round = 0; round < 34; round++) {
            const uint32_t e = __shfl_up_sync(0xffffffffu, tend, 1);
            const bool moved = lane > 0 && (round == 0 || e != ts);
            if (moved) {
                ts = e;
                if (e >= stop) {  // the previous lane's last codeword covers this range
                    tc = 0;
                    tend = e;
                    lane_bad = false;
                } else {
                    // follow the true codewords from e until one starts on this lane's path
                    b.seek(e);
                    uint32_t k = 0, wbad = kNone;
                    bool met = false;
                    while (b.pos < stop) {
                        const uint32_t off = b.pos - p.start;
                        if (b.pos >= p.start && off < 64 && ((p.mask >> off) & 1ull)) {
                            met = true;
                            break;
                        }
                        Codes cd = lk(b);
                        if (cd.l1 == 0) {
                            wbad = min(wbad, b.pos);
                            cd.l1 = 1;
                        }
                        k++;
                        consume<LK>(b, cd.l1);
                    }
                    if (met) {
                        const uint32_t off = b.pos - p.start;
                        tc = k + p.cnt - __popcll(p.mask & ((1ull << off) - 1ull));
                        tend = p.end;
                        lane_bad = wbad != kNone || (p.bad != kNone && p.bad >= b.pos);
                    } else {
                        tc = k;
                        tend = b.pos;
                        lane_bad = wbad != kNone;
                    }
                }
            }
            if (!__any_sync(0xffffffffu, moved)) {
                settled = true;
                break;
            }
        }
        const uint32_t total = __reduce_add_sync(0xffffffffu, tc);
        const uint32_t end31 = __shfl_sync(0xffffffffu, tend, 31);
        const bool ok = settled && !__any_sync(0xffffffffu, lane_bad) && total == cnt && end31 == nbits;
        // 3. every lane's codewords into the chunk buffer
        uint32_t isum = 0, zc = 0;
        if (ok) {
            const uint32_t o = warp_incl_scan(tc) - tc;
            b.seek(ts);
            for (uint32_t j = 0; j < tc;) {
                const Codes cd = lk(b);
                uint32_t adv = cd.l1;
                if (GBSZ_CHECK(o + j < a.chunk, a.ctl)) cbuf[o + j] = (uint16_t)cd.s1;
                j++;
                isum += cd.s1 ? cd.s1 - R : 0u;
                zc += cd.s1 == 0;
                if (cd.l2 && j < tc) {
                    if (GBSZ_CHECK(o + j < a.chunk, a.ctl)) cbuf[o + j] = (uint16_t)cd.s2;
                    j++;
                    isum += cd.s2 ? cd.s2 - R : 0u;
                    zc += cd.s2 == 0;
                    adv += cd.l2;
                }
                consume<LK>(b, adv);
            }
        }
        bad |= !ok;
        const uint32_t Z = __reduce_add_sync(0xffffffffu, zc);
        zeros += Z;
        __syncwarp();
        if (!FUSE) {
            if (ok) {  // the chunk's codes, 16 bytes per lane per step where aligned
                uint16_t *dst = a.codes + s0;
                const uint32_t n8 = al16 ? cnt / 8 : 0;
                for (uint32_t i = lane; i < n8; i += 32)
                    if (GBSZ_CHECK(s0 + 8 * i + 8 <= a.n, a.ctl))
                        reinterpret_cast<uint4 *>(dst)[i] = reinterpret_cast<const uint4 *>(cbuf)[i];
                for (uint32_t i = n8 * 8 + lane; i < cnt; i += 32)
                    if (GBSZ_CHECK(s0 + i < a.n, a.ctl)) dst[i] = cbuf[i];
            }
            __syncwarp();
            continue;
        }
        // fused S8: publish, look back, then the values
        const uint32_t S = __reduce_add_sync(0xffffffffu, isum);
        unsigned long long *look = wa.look;
        const bool publish = c != wa.hold_chunk;
        if (lane == 0 && publish)
            st_relaxed(&look[c], ((c == 0 || !ok) ? kLbInc : kLbAgg) | ((unsigned long long)Z << 32) | S);
        if (!ok) continue;  // published as final, so no later chunk waits on it
        uint32_t Sp = 0, Zp = 0;
        if (c > 0) {
            int64_t base = (int64_t)c - 1;
            const unsigned long long t0 = now_ns();
            for (;;) {
                const int64_t idx = base - (int64_t)lane;
                const unsigned long long v = idx >= 0 ? ld_relaxed(&look[idx]) : kLbInc;
                const uint32_t fl = (uint32_t)(v >> 62);
                const unsigned inc = __ballot_sync(0xffffffffu, fl == 2);
                const unsigned notyet = __ballot_sync(0xffffffffu, fl == 0);
                const uint32_t fi = inc ? __ffs(inc) - 1 : 31u;
                const unsigned need = fi == 31 ? 0xffffffffu : ((2u << fi) - 1u);
                if (notyet & need) {
                    // the same decision in every lane: the loop's votes need the whole warp
                    if (__any_sync(0xffffffffu, now_ns() - t0 > kLbWaitNs)) {
                        timeout = true;
                        break;
                    }
                    __nanosleep(64);
                    continue;
                }
                const bool take = lane <= fi;
                Sp += __reduce_add_sync(0xffffffffu, take ? (uint32_t)v : 0u);
                Zp += __reduce_add_sync(0xffffffffu, take ? (uint32_t)(v >> 32) & 0x3FFFFFFFu : 0u);
                if (inc) break;
                base -= 32;
            }
            if (lane == 0 && publish)
                st_relaxed(&look[c], kLbInc | ((unsigned long long)((Zp + Z) & 0x3FFFFFFFu) << 32) | (Sp + S));
            if (timeout) break;
        }
        if ((uint64_t)Zp + Z > wa.m) {  // more code-0 points than outliers
            bad = true;
            continue;
        }
        // values: rows of 128 points, 4 consecutive per lane
        uint32_t carry = Sp + wa.odp[Zp];
        uint32_t zb = Zp;
        const float ebx2 = wa.ebx2;
        float *out = wa.out + s0;
        for (uint32_t r0 = 0; r0 < cnt; r0 += 128) {
            const uint32_t q = r0 + 4 * lane;
            uint32_t cc[4];
            if (q + 4 <= cnt) {
                const uint2 v = *reinterpret_cast<const uint2 *>(cbuf + q);
                cc[0] = v.x & 0xFFFFu;
                cc[1] = v.x >> 16;
                cc[2] = v.y & 0xFFFFu;
                cc[3] = v.y >> 16;
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++) cc[j] = q + j < cnt ? cbuf[q + j] : R;  // past the end: residual 0
            }
            uint32_t zl = 0;
#pragma unroll
            for (int j = 0; j < 4; j++) zl += cc[j] == 0;
            const uint32_t zi = warp_incl_scan(zl);
            uint32_t ord = zb + zi - zl;
            uint32_t dv[4], sl = 0;
#pragma unroll
            for (int j = 0; j < 4; j++) {
                if (cc[j] == 0) {
                    const uint2 en = GBSZ_CHECK(ord < wa.m, a.ctl) ? wa.outl[ord] : make_uint2(kNone, 0u);
                    ord++;
                    bad |= en.x != (uint32_t)(s0 + q + j);
                    dv[j] = en.y;
                } else {
                    dv[j] = cc[j] - R;
                }
                sl += dv[j];
            }
            const uint32_t si = warp_incl_scan(sl);
            uint32_t run = carry + si - sl;
            float v[4];
#pragma unroll
            for (int j = 0; j < 4; j++) {
                run += dv[j];
                v[j] = recon_value((int32_t)run, ebx2);
            }
            const uint32_t nst = q + 4 <= cnt ? 4u : q < cnt ? cnt - q : 0u;  // points this lane stores
            if (!GBSZ_CHECK(nst == 0 || s0 + q + nst <= a.n, a.ctl)) {
                // (bounds-checking build) skip the row's stores
            } else if (al16 && q + 4 <= cnt) {
                *reinterpret_cast<float4 *>(out + q) = make_float4(v[0], v[1], v[2], v[3]);
            } else {
#pragma unroll
                for (int j = 0; j < 4; j++)
                    if (q + j < cnt) out[q + j] = v[j];
            }
            carry += __shfl_sync(0xffffffffu, si, 31);
            zb += __shfl_sync(0xffffffffu, zi, 31);
        }
        // anchored archive: the chunk's last integer is the next chunk's anchor
        if (wa.anchors && lane == 0) {
            if (c + 1 < a.nchunk && wa.anchors[c + 1] != carry) bad = true;
            if (c == 0 && wa.anchors[0] != 0u) bad = true;
        }
        __syncwarp();
    }
    if (lane == 0 && zeros) atomicAdd(&a.ctl->zeros, zeros);
    if (bad) atomicOr(&a.ctl->error, DERR_CORRUPT);
    if (timeout && lane == 0) atomicOr(&a.ctl->error, DERR_TIMEOUT);
}

template <bool FUSE, bool GENERAL>
__global__ void __launch_bounds__(kWThreads) k_decode_warp(const __grid_constant__ WarpDecodeArgs wa)
{
    if (GENERAL) decode_warp_body<FUSE, GeneralLK>(wa);
    else decode_warp_body<FUSE, FastLK>(wa);
}

struct OutlierResiduals {
    using T = uint32_t;
    const uint2 *outl;
    uint64_t m;
    uint32_t *odp;
    __device__ T load(uint64_t i) const { return i < m ? outl[i].y : 0u; }
    __device__ void store(uint64_t i, T v) const { odp[i] = v; }
    __device__ void total(T) const {}
};

size_t warp_smem(uint32_t chunk) { return kWTableBytes + (size_t)kWWarps * chunk * sizeof(uint16_t); }

// blocks of k_decode_warp resident per SM, by device, variant and chunk (64..4096)
int warp_blocks_per_sm(int variant, uint32_t chunk)
{
    static std::atomic<int> cache[64][4][7];
    int dev = 0;
    cudaGetDevice(&dev);
    uint32_t lc = 0;
    while ((64u << lc) < chunk && lc < 6) lc++;
    std::atomic<int> *slot = dev >= 0 && dev < 64 ? &cache[dev][variant][lc] : nullptr;
    if (slot && slot->load() > 0) return slot->load();
    const int most = (int)warp_smem(kWarpMaxChunk);
    const void *fns[4] = {(const void *)k_decode_warp<false, false>, (const void *)k_decode_warp<false, true>,
                          (const void *)k_decode_warp<true, false>, (const void *)k_decode_warp<true, true>};
    for (const void *f : fns) cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, most);
    int blocks = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, fns[variant], kWThreads, warp_smem(chunk)) !=
        cudaSuccess) {
        cudaGetLastError();
        blocks = 1;
    }
    blocks = blocks > 0 ? blocks : 1;
    if (slot) slot->store(blocks);
    return blocks;
}

}  // namespace

int launch_decode_warp(const WarpDecodeArgs &w, bool fuse, cudaStream_t st)
{
    const bool general = w.d.fast_bits == 0;
    const int variant = (fuse ? 2 : 0) + (general ? 1 : 0);
    const int per_sm = warp_blocks_per_sm(variant, w.d.chunk);
    const uint64_t want = (w.d.nchunk + kWWarps - 1) / kWWarps;
    const uint64_t sms = (uint64_t)(w.d.num_sms ? w.d.num_sms : 1);
    const unsigned grid = (unsigned)std::max<uint64_t>(1, std::min<uint64_t>(want, sms * per_sm));
    const size_t smem = warp_smem(w.d.chunk);
    switch (variant) {
    case 0: k_decode_warp<false, false><<<grid, kWThreads, smem, st>>>(w); break;
    case 1: k_decode_warp<false, true><<<grid, kWThreads, smem, st>>>(w); break;
    case 2: k_decode_warp<true, false><<<grid, kWThreads, smem, st>>>(w); break;
    default: k_decode_warp<true, true><<<grid, kWThreads, smem, st>>>(w); break;
    }
    return 1;
}

int launch_outlier_prefix(const uint2 *outl, uint64_t m, uint32_t *odp, uint32_t *partial, Control *ctl,
                          cudaStream_t st)
{
    return launch_scan(OutlierResiduals{outl, m, odp}, m + 1, partial, ctl, st);
}

}  // namespace gbsz
