// k_encode.cu -- S5: Huffman encode + deflate (Sec. 3.2.4) and S6 archive
// assembly.
//
// The paper deflates one chunk per thread.  Here one warp deflates one work
// unit with warp-level scans and shuffles only, in three fully parallel
// phases with no waiting between CTAs:
//   lanes     each lane owns S = min(128, C) consecutive symbols, so chunk
//             boundaries fall on lane boundaries; a unit is 32*S symbols
//             (4096/C chunks) or, for C > 4096, one whole chunk in rounds of
//             4096 symbols;
//   count     code lengths -> bits per lane -> chunk bits (segmented warp
//             sums, written to the archive's chunk table) -> the unit's
//             words and outliers (its exceptions were counted by the
//             dual-quant kernels);
//   scan      exclusive prefix sums of the unit totals give every unit's
//             global word / outlier / exception offsets;
//   pack      each lane packs its codewords MSB-first into 32-bit words and
//             stores the words it owns; the word it shares with the previous
//             lane of the same chunk is handed to that lane by a shuffle and
//             stored once, merged; outliers (idx, delta) and exceptions (idx,
//             raw bits) are written in index order at their global offsets;
//             the last unit writes the header.
// The dual-quant kernel parked {residual, is-exception} for every code-0
// point; it is read only where there are outliers (exception flags only when
// the field has exceptions at all), and the field only for exceptions.
#include "common.cuh"

#include <atomic>
#include "scan.cuh"

#include <algorithm>

namespace gbsz {

namespace {

constexpr int kEncThreads = 256;
constexpr int kWarps = kEncThreads / 32;
constexpr uint32_t kLaneMax = 128;  // symbols per lane
constexpr uint32_t kRound = 32 * kLaneMax;

template <bool CW32>
struct Table {
    const void *tab;
    __device__ __forceinline__ void get(uint32_t sym, uint32_t &len, unsigned long long &code) const
    {
        if (CW32) {
            const uint32_t v = static_cast<const uint32_t *>(tab)[sym];
            len = v >> 24;
            code = v & 0xFFFFFFu;
        } else {
            const unsigned long long v = static_cast<const unsigned long long *>(tab)[sym];
            len = (uint32_t)(v >> 56);
            code = v & ((1ull << 56) - 1);
        }
    }
    __device__ __forceinline__ uint32_t raw32(uint32_t sym) const { return static_cast<const uint32_t *>(tab)[sym]; }
    // PAIR layout in shared memory: {code, length} in two words, so a pair
    // of codewords is joined without masking or shifting the length out
    __device__ __forceinline__ uint2 split(uint32_t sym) const { return static_cast<const uint2 *>(tab)[sym]; }
    __device__ __forceinline__ uint32_t len_of(uint32_t sym) const
    {
        if (CW32) return static_cast<const uint32_t *>(tab)[sym] >> 24;
        return (uint32_t)(static_cast<const unsigned long long *>(tab)[sym] >> 56);
    }
};

__device__ __forceinline__ uint32_t warp_sum(uint32_t v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// sum over aligned groups of g lanes (g a power of two)
__device__ __forceinline__ uint32_t group_sum(uint32_t v, uint32_t g)
{
    for (uint32_t o = 1; o < g; o <<= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// exclusive scan inside aligned groups of g lanes
__device__ __forceinline__ uint32_t group_excl_scan(uint32_t v, uint32_t g)
{
    const uint32_t lane = threadIdx.x & 31, gl = lane & (g - 1);
    uint32_t inc = v;
    for (uint32_t o = 1; o < g; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (gl >= o) inc += t;
    }
    return inc - v;
}

// A lane's symbols, 8 at a time.  When the whole 32*S-symbol round lies in
// the field, the warp first copies it into its shared-memory slot with one
// burst of coalesced 16-byte loads (16 per lane, all independent), stored
// swizzled so that lanes reading "their" 16 bytes hit different banks; a
// partial last round is read from global memory directly.
struct Lane {
    const uint16_t *g;  // global codes of this lane (s0)
    const uint4 *sm;    // this warp's shared slot, or nullptr
    uint32_t lane, nv;  // nv = S / 8 vectors per lane
    uint32_t cnt;       // symbols of this lane (0..S)
    __device__ __forceinline__ uint4 vec(uint32_t j) const
    {
        return sm[lane * nv + ((j + lane) & (nv - 1))];
    }
};

__device__ __forceinline__ void stage_round(const uint16_t *codes, uint64_t r0, uint32_t S, uint4 *slot)
{
    const uint32_t lane = threadIdx.x & 31, nv = S / 8;
    const uint4 *src = reinterpret_cast<const uint4 *>(codes + r0);
    for (uint32_t k = 0; k < nv; k++) {
        const uint32_t gidx = k * 32 + lane, L = gidx / nv, j = gidx % nv;
        const uint32_t dst = (uint32_t)__cvta_generic_to_shared(slot + L * nv + ((j + L) & (nv - 1)));
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src + gidx) : "memory");
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    __syncwarp();
}

__device__ __forceinline__ void put_u32(uint8_t *p, uint32_t v) { *reinterpret_cast<uint32_t *>(p) = v; }
__host__ __device__ inline bool anchors_of(const EncodeArgs &a) { return anchored(a.ndim, a.order, a.lblock, a.chunk); }

// archive header and the zero bytes between sections (last unit's warp)
__device__ void write_header(const EncodeArgs &a, const Layout &L, uint64_t nchunk, uint64_t m, uint64_t e,
                             uint64_t w, uint32_t maxlen)
{
    uint32_t h[kHeaderBytes / 4];
    for (int i = 0; i < (int)(kHeaderBytes / 4); i++) h[i] = 0;
    auto set64 = [&](uint32_t off, unsigned long long v) {
        h[off / 4] = (uint32_t)v;
        h[off / 4 + 1] = (uint32_t)(v >> 32);
    };
    h[H_MAGIC / 4] = kMagic;
    h[H_VERSION / 4] = (uint32_t)kVersion | (kHeaderBytes << 16);
    h[H_NDIM / 4] = a.ndim;
    h[H_EBMODE / 4] = a.eb_mode;
    set64(H_DIMS, a.dims[0]);
    set64(H_DIMS + 8, a.dims[1]);
    set64(H_DIMS + 16, a.dims[2]);
    set64(H_N, a.n);
    set64(H_EB, (unsigned long long)__double_as_longlong(a.eb));
    h[H_EBF / 4] = __float_as_uint(a.ctl->eb);
    h[H_EBX2 / 4] = __float_as_uint(a.ctl->ebx2);
    h[H_INV2EB / 4] = __float_as_uint(a.ctl->inv2eb);
    h[H_RADIUS / 4] = a.radius;
    h[H_CHUNK / 4] = a.chunk;
    h[H_NCHUNK / 4] = (uint32_t)nchunk;
    set64(H_M, m);
    set64(H_E, e);
    set64(H_W, w);
    h[H_MAXLEN / 4] = maxlen;
    h[H_LBLOCK / 4] = a.lblock;
    set64(H_TOTAL, L.total);
    h[H_ORDER / 4] = a.order;
    h[H_DIM3 / 4] = (uint32_t)a.dims[3];  // below 2^32 as n is
    for (int i = 0; i < (int)(kHeaderBytes / 4); i++) put_u32(a.archive + 4 * i, h[i]);
    for (uint64_t b = L.len + a.nbins; b < L.bits; b++) a.archive[b] = 0;
    for (uint64_t b = L.bits + 4 * nchunk; b < L.anch; b++) a.archive[b] = 0;
    for (uint64_t b = L.anch + 4 * L.nanch; b < L.outl; b++) a.archive[b] = 0;  // anchors: written by dual-quant
    for (uint64_t b = L.exc + 8 * e; b < L.stream; b++) a.archive[b] = 0;
}

struct UnitGeom {
    uint32_t S;       // symbols per lane
    bool multi;       // a unit is one chunk of several 4096-symbol rounds
    uint32_t G;       // lanes per chunk inside a round
    uint64_t U;       // symbols per unit
    __device__ __forceinline__ explicit UnitGeom(uint32_t C)
    {
        S = C < kLaneMax ? C : kLaneMax;
        multi = C > kRound;
        G = multi ? 32u : C / S;
        U = multi ? C : 32ull * S;
    }
};

// Phase 1: per-unit totals, per-lane bit counts and the archive's chunk bit
// counts.  Codes are read with coalesced 16-byte loads, four in flight per
// lane (lane l holds symbols 256k + 8l .. +7 of step k).  A "count entry" per
// symbol packs its code length (bits 0-15) with a code-0 flag (bit 16), so one
// add per symbol accumulates both; a unit's exceptions were counted by the
// dual-quant kernels, so no residual is read here.  Each lane parks
// the packed sum of its 8 symbols in a padded per-warp shared array, and lane
// l then sums the S / 8 partials of its S-symbol segment (the segment lane l
// packs in phase 3).
struct CountSmem {
    const uint32_t *t;
    __device__ __forceinline__ uint32_t operator()(uint32_t c) const { return t[c]; }
};
template <bool CW32>
struct CountGlobal {
    Table<CW32> tab;
    __device__ __forceinline__ uint32_t operator()(uint32_t c) const
    {
        return tab.len_of(c) | (c == 0 ? 0x10000u : 0u);
    }
};

constexpr uint32_t kPartStride = 33;  // padded row of per-lane partials

// one 128-bit read-only load (codes do not change while the encoder runs)
__device__ __forceinline__ uint4 ldg_nc16(const void *p)
{
    uint4 v;
    asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

__device__ __forceinline__ uint32_t count8(const CountSmem &ct, uint4 w)
{
    return ct(w.x & 0xFFFFu) + ct(w.x >> 16) + ct(w.y & 0xFFFFu) + ct(w.y >> 16) + ct(w.z & 0xFFFFu) +
           ct(w.z >> 16) + ct(w.w & 0xFFFFu) + ct(w.w >> 16);
}
template <typename CT>
__device__ __forceinline__ uint32_t count8(const CT &ct, uint4 w)
{
    const uint32_t v[4] = {w.x, w.y, w.z, w.w};
    uint32_t s = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) s += ct(v[q] & 0xFFFFu) + ct(v[q] >> 16);
    return s;
}

template <typename CT>
__device__ __forceinline__ uint32_t count_tail(const EncodeArgs &a, const CT &ct, uint64_t p, uint64_t n, uint32_t &z)
{
    uint32_t s = 0, m = 0;
    for (uint32_t q = 0; q < 8 && p + q < n; q++) {
        const uint32_t e = ct(a.codes[p + q]);
        s += e;
        m += e << q;
    }
    z = m >> 16;
    return s;
}

// The code-0 positions of eight symbols (bit q: symbol q, x's low half
// first) from their count entries: sum_q entry_q << q keeps the length parts
// below bit 16 (255 * 45 < 2^16), so bits 16..23 are the code-0 flags.
template <typename CT>
__device__ __forceinline__ uint32_t count8z(const CT &ct, uint4 w, uint32_t &z)
{
    const uint32_t v[4] = {w.x, w.y, w.z, w.w};
    uint32_t s = 0, m = 0;
#pragma unroll
    for (int q = 0; q < 4; q++) {
        const uint32_t e0 = ct(v[q] & 0xFFFFu), e1 = ct(v[q] >> 16);
        s += e0 + e1;
        m += (e0 << (2 * q)) + (e1 << (2 * q + 1));
    }
    z = m >> 16;
    return s;
}

// ZB: the kernel may write the code-0 bitmap (when a.zbits is set)
template <bool ZB, typename CT>
__device__ __forceinline__ void count_units(const EncodeArgs &a, uint64_t nunits, const CT &ct, uint32_t *part,
                                            VGrid vg)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t n = a.n;
    const uint32_t C = a.chunk;
    const UnitGeom ug(C);
    const uint32_t S = ug.S, per = S / 8;  // partials per segment
    const uint32_t segs = 32 / per;        // segments per 256-symbol step
    const uint32_t steps = S / 8;          // 256-symbol steps per round: 8 or 16
    const uint64_t nchunk = (n + C - 1) / C;
    const Layout L0 = make_layout(a.radius, nchunk, a.ctl->n_out, a.ctl->n_exc, 0, anchors_of(a));
    const bool first_of_chunk = (lane & (ug.G - 1)) == 0;
    const uint32_t *myseg = part + (lane / segs) * kPartStride + (lane % segs) * per;
    uint8_t *zb8 = ZB ? reinterpret_cast<uint8_t *>(a.zbits) : nullptr;  // a byte per 8 points (coalesced stores)
    const uint64_t gw = ((uint64_t)vg.bid * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)vg.nb * blockDim.x) >> 5;
    for (uint64_t u = gw; u < nunits; u += nw) {
        const uint64_t ubase = u * ug.U;
        const uint64_t ulen = n - ubase < ug.U ? n - ubase : ug.U;
        const uint32_t rounds = ug.multi ? (uint32_t)((ulen + kRound - 1) / kRound) : 1u;
        uint32_t unit_words = 0, unit_out = 0;
        unsigned long long chunk_bits = 0;
        for (uint32_t r = 0; r < rounds; r++) {
            const uint64_t r0 = ubase + (uint64_t)r * 32 * S;
            const bool full = r0 + 32ull * S <= n;
            const uint4 *src = reinterpret_cast<const uint4 *>(a.codes + r0) + lane;
            __syncwarp();  // the previous round's partials have been read
            // eight 16-byte loads in flight per lane (steps is 8 or 16)
            for (uint32_t k = 0; k < steps; k += 8) {
                uint32_t s8[8];
                if (full) {
                    uint4 w[8];
#pragma unroll
                    for (int i = 0; i < 8; i++) w[i] = ldg_nc16(src + 32 * (k + i));
                    if (zb8) {
                        const uint64_t b0 = r0 / 8 + 32ull * k + lane;
#pragma unroll
                        for (int i = 0; i < 8; i++) {
                            uint32_t z;
                            s8[i] = count8z(ct, w[i], z);
                            if (GBSZ_CHECK(b0 + 32 * i < (n + 7) / 8, a.ctl)) zb8[b0 + 32 * i] = (uint8_t)z;
                        }
                    } else {
#pragma unroll
                        for (int i = 0; i < 8; i++) s8[i] = count8(ct, w[i]);
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < 8; i++) {
                        const uint64_t p = r0 + 256ull * (k + i) + 8ull * lane;
                        uint32_t z = 0;
                        s8[i] = p + 8 <= n ? count8z(ct, src[32 * (k + i)], z) : count_tail(a, ct, p, n, z);
                        if (zb8 && p < n && GBSZ_CHECK(p / 8 < (n + 7) / 8, a.ctl)) zb8[p / 8] = (uint8_t)z;
                    }
                }
#pragma unroll
                for (int i = 0; i < 8; i++) part[(k + i) * kPartStride + lane] = s8[i];
            }
            __syncwarp();
            uint32_t seg = 0;
            for (uint32_t t = 0; t < per; t++) seg += myseg[t];
            const uint32_t sb = seg & 0xFFFFu, so = seg >> 16;
            const uint64_t s0 = r0 + (uint64_t)lane * S;
            const uint32_t cnt = s0 < n ? (uint32_t)(n - s0 < S ? n - s0 : S) : 0u;
            if (cnt) a.lane_bits[r0 / S + lane] = sb;
            if (ug.multi) {
                chunk_bits += warp_sum(sb);
            } else {
                const uint32_t cb = group_sum(sb, ug.G);
                uint32_t cw = 0;
                if (first_of_chunk && cnt) {
                    cw = (cb + 31) / 32;
                    if (GBSZ_CHECK(s0 / C < (n + C - 1) / C, a.ctl)) put_u32(a.archive + L0.bits + 4 * (s0 / C), cb);
                }
                unit_words += warp_sum(cw);
            }
            unit_out += so;
        }
        unit_out = warp_sum(unit_out);
        const uint32_t unit_exc = a.unit_exc[u];
        if (ug.multi) {
            unit_words = (uint32_t)((chunk_bits + 31) / 32);
            if (lane == 0 && GBSZ_CHECK(u < (n + C - 1) / C, a.ctl))
                put_u32(a.archive + L0.bits + 4 * u, (uint32_t)chunk_bits);
        }
        if (lane == 0)
            a.unit_tot[u] = make_ulonglong2(unit_words, (unsigned long long)unit_out | ((unsigned long long)unit_exc << 32));
    }
}

// appends one codeword to the bit accumulator; returns true when a full word
// (acc >> nacc, low 32 bits) is ready.  Codes of at most 24 bits (CW32) need
// no masking: bits above the 32 still pending just shift out of the 64-bit
// accumulator.
template <bool CW32>
__device__ __forceinline__ void append(unsigned long long &acc, uint32_t &nacc, unsigned long long code, uint32_t len,
                                       uint32_t *w, uint32_t &nw)
{
    nw = 0;
    if (!CW32 && len > 32) {
        const uint32_t hl = len - 32;
        acc = (acc << hl) | (code >> 32);
        nacc += hl;
        if (nacc >= 32) {
            nacc -= 32;
            w[nw++] = (uint32_t)(acc >> nacc);
        }
        code &= 0xFFFFFFFFull;
        len = 32;
    }
    acc = (acc << len) | code;
    nacc += len;
    if (nacc >= 32) {
        nacc -= 32;
        w[nw++] = (uint32_t)(acc >> nacc);
    }
}

// The outlier records (index, residual) and exception records (index, raw
// value bits) of one round, in index order.  zlo / zhi mark the code-0 points
// among the lane's S points from s0 (bit j: point s0 + j); orun / erun are
// the warp's running record offsets, advanced by the round's totals.  A
// lane's residuals are loaded four at a time, then written.
__device__ __forceinline__ void emit_outliers(const EncodeArgs &a, const Layout &L0, uint64_t s0,
                                              unsigned long long zlo, unsigned long long zhi, bool unit_exc,
                                              uint64_t &orun, uint64_t &erun, bool &cap_err)
{
    const uint64_t n = a.n;
    const uint32_t nz = __popcll(zlo) + __popcll(zhi);
    uint32_t ne = 0;
    if (unit_exc) {
        for (unsigned long long m = zlo; m; m &= m - 1)
            if (GBSZ_CHECK(s0 + __ffsll(m) - 1 < n, a.ctl)) ne += a.dscr[s0 + __ffsll(m) - 1].y != 0;
        for (unsigned long long m = zhi; m; m &= m - 1)
            if (GBSZ_CHECK(s0 + 63 + __ffsll(m) < n, a.ctl)) ne += a.dscr[s0 + 63 + __ffsll(m)].y != 0;
    }
    const uint32_t oinc = warp_incl_scan(nz), einc = warp_incl_scan(ne);
    uint64_t oi = orun + (oinc - nz), ei = erun + (einc - ne);
    auto emit_outlier = [&](uint64_t idx, int2 dv) {
        const uint64_t o8 = L0.outl + 8 * oi++;
        if (o8 + 8 <= a.capacity) {
            put_u32(a.archive + o8, (uint32_t)idx);
            put_u32(a.archive + o8 + 4, (uint32_t)dv.x);
        } else {
            cap_err = true;
        }
        if (dv.y) {
            const uint64_t e8 = L0.exc + 8 * ei++;
            if (e8 + 8 <= a.capacity) {
                put_u32(a.archive + e8, (uint32_t)idx);
                put_u32(a.archive + e8 + 4, __float_as_uint(a.x[idx]));
            } else {
                cap_err = true;
            }
        }
    };
    unsigned long long mlo = zlo, mhi = zhi;
    while (mlo | mhi) {
        uint64_t idx[4];
        bool has[4];
#pragma unroll
        for (int k = 0; k < 4; k++) {
            has[k] = (mlo | mhi) != 0;
            uint32_t j = 0;
            if (mlo) {
                j = __ffsll(mlo) - 1;
                mlo &= mlo - 1;
            } else if (mhi) {
                j = 63 + __ffsll(mhi);
                mhi &= mhi - 1;
            }
            idx[k] = s0 + j;
        }
        int2 dv[4];
#pragma unroll
        for (int k = 0; k < 4; k++)
            dv[k] = has[k] && GBSZ_CHECK(idx[k] < n, a.ctl) ? a.dscr[idx[k]] : make_int2(0, 0);
#pragma unroll
        for (int k = 0; k < 4; k++)
            if (has[k]) emit_outlier(idx[k], dv[k]);
    }
    orun += __shfl_sync(0xffffffffu, oinc, 31);
    erun += __shfl_sync(0xffffffffu, einc, 31);
}

// Phase 3: pack every unit at its offsets; the last unit writes the header.
// With a code-0 bitmap (1D order 1) the records are k_encode_outliers' work
// and the lanes only pack.  (Zero masks and residual loads in the packing
// warps cost 0.146 of 0.338 ms at 2^28 points with 1.6% outliers: pack runs
// three blocks per SM for its shared-memory staging, too few warps to cover
// the residuals' random loads.)
// PAIR (longest code at most 16 bits, or with LONG at most 24): two
// codewords are joined into one of at most 32 bits before they enter the
// accumulator, so each pair needs one shift-in and one full-word test; with
// LONG a pair longer than 32 bits together takes two shift-ins instead.
// (Longest code 18 bits, 512^3 lognormal field at rel eb 1e-4: pack 0.244 ms
// with one codeword per shift-in, 0.240 ms in pairs.)
template <bool CW32, bool PAIR, bool LONG = false>
__device__ void pack_units(const EncodeArgs &a, uint64_t nunits, const Table<CW32> &tab, uint4 *slot, VGrid vg)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t n = a.n;
    const uint32_t C = a.chunk;
    const UnitGeom ug(C);
    const uint32_t S = ug.S, G = ug.G, nv = S / 8;
    const bool multi = ug.multi;
    const uint64_t nchunk = (n + C - 1) / C;
    const uint64_t M = a.ctl->n_out, E = a.ctl->n_exc;
    const bool any_exc = E != 0;
    const Layout L0 = make_layout(a.radius, nchunk, M, E, 0, anchors_of(a));
    uint32_t *stream = reinterpret_cast<uint32_t *>(a.archive + L0.stream);
    const uint64_t stream_cap = a.capacity > L0.stream ? (a.capacity - L0.stream) / 4 : 0;
    const bool first_of_chunk = (lane & (G - 1)) == 0;
    const bool zb = a.zbits != nullptr;  // records written by k_encode_outliers
    const uint64_t gw = ((uint64_t)vg.bid * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)vg.nb * blockDim.x) >> 5;
    bool cap_err = false;
    for (uint64_t u = gw; u < nunits; u += nwarps) {
        const uint64_t ubase = u * ug.U;
        const uint64_t ulen = n - ubase < ug.U ? n - ubase : ug.U;
        const uint32_t rounds = multi ? (uint32_t)((ulen + kRound - 1) / kRound) : 1u;
        const ulonglong2 off = a.unit_off[u];
        const unsigned long long W0 = off.x, O0 = off.y & 0xFFFFFFFFull, E0 = off.y >> 32;
        // exceptions of the unit, counted by dual-quant
        const bool unit_exc = !zb && any_exc && a.unit_exc[u] != 0;
        if (u == nunits - 1 && lane == 0) {
            const ulonglong2 tot = a.unit_tot[u];
            const unsigned long long W = W0 + tot.x;
            const Layout L = make_layout(a.radius, nchunk, M, E, W, anchors_of(a));
            if (O0 + (tot.y & 0xFFFFFFFFull) != M || E0 + (tot.y >> 32) != E) atomicOr(&a.ctl->error, DERR_INTERNAL);
            a.ctl->words = W;
            a.ctl->total = L.total;
            if (L.total > a.capacity) atomicOr(&a.ctl->error, DERR_CAPACITY);
            if (L.stream <= a.capacity) write_header(a, L, nchunk, M, E, W, a.ctl->maxlen);
        }
        unsigned long long round_bits = 0;  // multi: bits of earlier rounds of the chunk
        uint64_t orun = O0, erun = E0;      // record offsets of this round
        uint32_t carry = 0;                 // multi: partial last word of the previous round
        for (uint32_t r = 0; r < rounds; r++) {
            const uint64_t r0 = ubase + (uint64_t)r * 32 * S, s0 = r0 + (uint64_t)lane * S;
            const uint32_t cnt = s0 < n ? (uint32_t)(n - s0 < S ? n - s0 : S) : 0u;
            const bool full = r0 + 32ull * S <= n;
            const uint32_t bits = cnt ? a.lane_bits[r0 / S + lane] : 0u;
            __syncwarp();
            if (full) stage_round(a.codes, r0, S, slot);
            const Lane ln{a.codes + s0, full ? slot : nullptr, lane, nv, cnt};
            unsigned long long gbit;  // global bit position of this lane's first bit
            uint32_t rtot = 0;
            if (multi) {
                const uint32_t inc = warp_incl_scan(bits);
                rtot = __shfl_sync(0xffffffffu, inc, 31);
                gbit = W0 * 32 + round_bits + (inc - bits);
            } else {
                const uint32_t cb = group_sum(bits, G);
                const uint32_t cw = first_of_chunk && cnt ? (cb + 31) / 32 : 0u;
                const uint32_t bin = group_excl_scan(bits, G);
                const uint32_t winc = warp_incl_scan(cw);
                const uint32_t woff = __shfl_sync(0xffffffffu, winc - cw, lane & ~(G - 1));
                gbit = (W0 + woff) * 32 + bin;
            }
            // pack: every completed word is stored as soon as it is full,
            // with no branch (the store is predicated).  The accumulator
            // starts with (gbit & 31) zero bits, so a lane that starts inside
            // a word (the "head", shared with the previous lane of its chunk)
            // stores that word with only its own bits; after the loop the
            // head is read back and handed to the previous lane, which stores
            // its last partial word (the "tail") merged with it.  Every full
            // lane holds at least S >= 64 bits, so it always completes its
            // head word inside the loop; only a short last lane can end inside
            // it, and then its bits are handed over without being stored.
            const bool starts_mid = (gbit & 31u) != 0 && cnt > 0;
            if ((gbit + bits + 31) / 32 > stream_cap) cap_err = true;
            const bool ok = !cap_err;
            uint32_t *lout = stream + (gbit >> 5);
            unsigned long long acc = 0;
            uint32_t nacc = (uint32_t)(gbit & 31u);
            uint32_t nw32 = 0;  // words completed by this lane
            unsigned long long zlo = 0, zhi = 0;  // code-0 positions of this lane
            if (ln.sm) {
                for (uint32_t j = 0; j < ln.nv; j++) {
                    const uint4 q4 = ln.vec(j);
                    const uint32_t v[4] = {q4.x, q4.y, q4.z, q4.w};
                    if (!zb) {
                        // zero symbols of these 8, as bits 8j.. of the lane's mask
                        const uint32_t z = ((__vcmpeq2(v[0], 0) & 0x00010001u) * 1u) |
                                           ((__vcmpeq2(v[1], 0) & 0x00010001u) << 2) |
                                           ((__vcmpeq2(v[2], 0) & 0x00010001u) << 4) |
                                           ((__vcmpeq2(v[3], 0) & 0x00010001u) << 6);
                        const uint32_t z8 = (z | (z >> 15)) & 0xFFu;
                        if (z8) {
                            if (j < 8) zlo |= (unsigned long long)z8 << (8 * j);
                            else zhi |= (unsigned long long)z8 << (8 * (j - 8));
                        }
                    }
                    if (CW32 && PAIR) {
#pragma unroll
                        for (int k = 0; k < 4; k++) {
                            const uint2 e0 = tab.split(v[k] & 0xFFFFu), e1 = tab.split(v[k] >> 16);
                            const uint32_t len = e0.y + e1.y;
                            if (LONG && len > 32) {
                                // two codes of up to 24 bits that do not fit one word together
                                // (rare): one shift-in each
                                acc = (acc << e0.y) | e0.x;
                                nacc += e0.y;
                                bool full_w = nacc >= 32;
                                nacc -= full_w ? 32u : 0u;
                                if (full_w && ok) lout[nw32] = (uint32_t)(acc >> nacc);
                                nw32 += full_w ? 1u : 0u;
                                acc = (acc << e1.y) | e1.x;
                                nacc += e1.y;
                                full_w = nacc >= 32;
                                nacc -= full_w ? 32u : 0u;
                                if (full_w && ok) lout[nw32] = (uint32_t)(acc >> nacc);
                                nw32 += full_w ? 1u : 0u;
                                continue;
                            }
                            acc = (acc << len) | ((e0.x << e1.y) | e1.x);
                            nacc += len;
                            const bool full_w = nacc >= 32;
                            nacc -= full_w ? 32u : 0u;
                            if (full_w && ok) lout[nw32] = (uint32_t)(acc >> nacc);
                            nw32 += full_w ? 1u : 0u;
                        }
                    } else {
#pragma unroll
                        for (int k = 0; k < 8; k++) {
                            const uint32_t c = (v[k >> 1] >> ((k & 1) * 16)) & 0xFFFFu;
                            if (CW32) {
                                const uint32_t e = tab.raw32(c);
                                const uint32_t len = e >> 24;
                                acc = (acc << len) | (e & 0xFFFFFFu);
                                nacc += len;
                                const bool full_w = nacc >= 32;
                                nacc -= full_w ? 32u : 0u;
                                if (full_w && ok) lout[nw32] = (uint32_t)(acc >> nacc);
                                nw32 += full_w ? 1u : 0u;
                            } else {
                                uint32_t len;
                                unsigned long long code;
                                tab.get(c, len, code);
                                uint32_t w[2], nw;
                                append<CW32>(acc, nacc, code, len, w, nw);
                                for (uint32_t q = 0; q < nw; q++) {
                                    if (ok) lout[nw32] = w[q];
                                    nw32++;
                                }
                            }
                        }
                    }
                }
            } else {
                for (uint32_t j = 0; j < cnt; j++) {
                    const uint32_t c = ln.g[j];
                    uint32_t len;
                    unsigned long long code;
                    if (PAIR) {  // the {code, length} layout
                        const uint2 e = tab.split(c);
                        len = e.y;
                        code = e.x;
                    } else {
                        tab.get(c, len, code);
                    }
                    uint32_t w[2], nw;
                    append<CW32>(acc, nacc, code, len, w, nw);
                    for (uint32_t q = 0; q < nw; q++) {
                        if (ok) lout[nw32] = w[q];
                        nw32++;
                    }
                    if (c == 0 && !zb) {
                        if (j < 64) zlo |= 1ull << j;
                        else zhi |= 1ull << (j - 64);
                    }
                }
            }
            __syncwarp();  // in-loop head stores land before the previous lane's merged store
            const uint32_t last = nacc > 0 ? (uint32_t)(acc << (32 - nacc)) : 0u;
            const bool inside_head = starts_mid && nw32 == 0;  // short last lane
            uint32_t head = 0;
            if (starts_mid && ok) head = inside_head ? last : lout[0];
            const bool has_tail = nacc > 0 && cnt > 0 && !inside_head;
            // hand heads to the previous lane of the same chunk
            const uint32_t next_head = __shfl_down_sync(0xffffffffu, head, 1);
            const bool next_starts_mid = __shfl_down_sync(0xffffffffu, starts_mid ? 1u : 0u, 1) != 0;
            const bool next_same_chunk = lane < 31 && ((lane + 1) & (G - 1)) != 0;
            const uint32_t prev_carry = __shfl_sync(0xffffffffu, carry, 31);
            if (has_tail) {
                uint32_t v = last;
                if (next_same_chunk && next_starts_mid) v |= next_head;
                if (multi && lane == 31 && r + 1 < rounds) {
                    carry = v;  // the next round's lane 0 finishes this word
                } else if (ok) {
                    lout[nw32] = v;
                }
            }
            if (multi && lane == 0 && r > 0 && starts_mid && ok) lout[0] = head | prev_carry;
            if (multi && !(lane == 31 && has_tail)) carry = 0;
            if (!zb) emit_outliers(a, L0, s0, zlo, zhi, unit_exc, orun, erun, cap_err);
            round_bits += rtot;
        }
    }
    if (cap_err) atomicOr(&a.ctl->error, DERR_CAPACITY);
}

// Outlier and exception records from the dual-quant kernel's code-0 bitmap:
// one warp per unit, its rounds in order as in pack, lane l reading the
// bitmap words of the same S points as there (S / 32 = 2 or 4 words, one 8-
// or 16-byte load).  The ranks are the bitmap's popcounts scanned across the
// warp on top of the unit's offsets from the count/scan phases, so the
// records land exactly where pack would have put them.  The warp lists the
// round's code-0 points in rank order in shared memory; lane l then takes
// records l, l + 32, ..., so its residual loads are issued together and the
// records are stored coalesced; exceptions are ranked by ballot.  A round of
// more than kOutWin outliers takes the per-lane path instead.  Bits of points
// at or past n are cleared (their entries were never written).
constexpr uint32_t kOutWin = 512;  // listed positions per warp (16-bit offsets in the round)

__device__ void outlier_units(const EncodeArgs &a, uint64_t nunits, uint16_t *pos, VGrid vg)
{
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t n = a.n;
    const uint32_t C = a.chunk;
    const UnitGeom ug(C);
    const uint32_t S = ug.S;
    const uint64_t nchunk = (n + C - 1) / C;
    const uint64_t M = a.ctl->n_out, E = a.ctl->n_exc;
    const Layout L0 = make_layout(a.radius, nchunk, M, E, 0, anchors_of(a));
    const uint64_t gw = ((uint64_t)vg.bid * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)vg.nb * blockDim.x) >> 5;
    bool cap_err = false;
    for (uint64_t u = gw; u < nunits; u += nwarps) {
        const uint64_t ubase = u * ug.U;
        const uint64_t ulen = n - ubase < ug.U ? n - ubase : ug.U;
        const uint32_t rounds = ug.multi ? (uint32_t)((ulen + kRound - 1) / kRound) : 1u;
        const ulonglong2 off = a.unit_off[u];
        uint64_t orun = off.y & 0xFFFFFFFFull, erun = off.y >> 32;
        const bool unit_exc = E != 0 && a.unit_exc[u] != 0;
        for (uint32_t r = 0; r < rounds; r++) {
            const uint64_t r0 = ubase + (uint64_t)r * 32 * S, s0 = r0 + (uint64_t)lane * S;
            unsigned long long zlo = 0, zhi = 0;
            if (s0 < n && GBSZ_CHECK(s0 + S <= (n + 127) / 128 * 128, a.ctl)) {
                const uint32_t *zw = a.zbits + s0 / 32;
                if (S == 128) {
                    const uint4 q = *reinterpret_cast<const uint4 *>(zw);
                    zlo = q.x | ((unsigned long long)q.y << 32);
                    zhi = q.z | ((unsigned long long)q.w << 32);
                } else {  // S = 64
                    const uint2 q = *reinterpret_cast<const uint2 *>(zw);
                    zlo = q.x | ((unsigned long long)q.y << 32);
                }
                if (s0 + S > n) {  // the field's last lane
                    const uint64_t k = n - s0;  // points of the lane, 1..S-1
                    if (k < 64) {
                        zlo &= (1ull << k) - 1;
                        zhi = 0;
                    } else {
                        zhi &= (1ull << (k - 64)) - 1;
                    }
                }
            }
            const uint32_t nz = __popcll(zlo) + __popcll(zhi);
            const uint32_t oinc = warp_incl_scan(nz), T = __shfl_sync(0xffffffffu, oinc, 31);
            if (T > kOutWin) {
                emit_outliers(a, L0, s0, zlo, zhi, unit_exc, orun, erun, cap_err);
                continue;
            }
            uint32_t k = oinc - nz;
            for (unsigned long long m = zlo; m; m &= m - 1) pos[k++] = (uint16_t)(lane * S + __ffsll(m) - 1);
            for (unsigned long long m = zhi; m; m &= m - 1) pos[k++] = (uint16_t)(lane * S + 63 + __ffsll(m));
            __syncwarp();
            for (uint32_t k0 = 0; k0 < T; k0 += 128) {
                uint64_t idx[4];
                int2 dv[4];
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t kk = k0 + 32 * q + lane;
                    idx[q] = kk < T ? r0 + pos[kk] : 0;
                    dv[q] = kk < T && GBSZ_CHECK(idx[q] < n, a.ctl) ? a.dscr[idx[q]] : make_int2(0, 0);
                }
#pragma unroll
                for (int q = 0; q < 4; q++) {
                    const uint32_t kk = k0 + 32 * q + lane;
                    const bool valid = kk < T;
                    if (valid) {
                        const uint64_t o8 = L0.outl + 8 * (orun + kk);
                        if (o8 + 8 <= a.capacity) {
                            put_u32(a.archive + o8, (uint32_t)idx[q]);
                            put_u32(a.archive + o8 + 4, (uint32_t)dv[q].x);
                        } else {
                            cap_err = true;
                        }
                    }
                    if (unit_exc) {  // warp-uniform
                        const bool ex = valid && dv[q].y != 0;
                        const uint32_t b = __ballot_sync(0xffffffffu, ex);
                        if (ex) {
                            const uint64_t e8 = L0.exc + 8 * (erun + __popc(b & ((1u << lane) - 1)));
                            if (e8 + 8 <= a.capacity) {
                                put_u32(a.archive + e8, (uint32_t)idx[q]);
                                put_u32(a.archive + e8 + 4, __float_as_uint(a.x[idx[q]]));
                            } else {
                                cap_err = true;
                            }
                        }
                        erun += __popc(b);
                    }
                }
            }
            orun += T;
            __syncwarp();  // the list is rewritten next round
        }
    }
    if (cap_err) atomicOr(&a.ctl->error, DERR_CAPACITY);
}

// The codeword width is chosen on the device from the longest code length
// the codebook kernel found: 32-bit entries when it is at most 24 bits.
__device__ __forceinline__ const void *load_table(const EncodeArgs &a, uint32_t use_smem, unsigned long long *s_tab,
                                                  bool w32, bool pair = false)
{
    if (!use_smem) return w32 ? (const void *)a.cw32 : (const void *)a.cw64;
    if (pair) {
        uint2 *st = reinterpret_cast<uint2 *>(s_tab);
        for (uint32_t i = threadIdx.x; i < a.nbins; i += blockDim.x) {
            const uint32_t e = a.cw32[i];
            st[i] = make_uint2(e & 0xFFFFFFu, e >> 24);
        }
    } else if (w32) {
        uint32_t *st = reinterpret_cast<uint32_t *>(s_tab);
        for (uint32_t i = threadIdx.x; i < a.nbins; i += blockDim.x) st[i] = a.cw32[i];
    } else {
        for (uint32_t i = threadIdx.x; i < a.nbins; i += blockDim.x) s_tab[i] = a.cw64[i];
    }
    __syncthreads();
    return s_tab;
}

constexpr uint32_t kCountSmemBins = 8192;
constexpr uint32_t kPartWords = 16 * kPartStride;  // per warp, S <= 128

template <bool ZB>
__device__ __forceinline__ void count_dispatch(const EncodeArgs &a, uint64_t nunits, uint32_t *part, uint32_t *tab,
                                               bool w32, VGrid vg)
{
    if (a.nbins <= kCountSmemBins) count_units<ZB>(a, nunits, CountSmem{tab}, part, vg);
    else if (w32) count_units<ZB>(a, nunits, CountGlobal<true>{Table<true>{a.cw32}}, part, vg);
    else count_units<ZB>(a, nunits, CountGlobal<false>{Table<false>{a.cw64}}, part, vg);
}

template <bool ZB>
__device__ __forceinline__ void count_body(const EncodeArgs &a, uint64_t nunits, VGrid vg)
{
    extern __shared__ uint32_t s_cnt[];
    uint32_t *part = s_cnt + (threadIdx.x >> 5) * kPartWords;
    uint32_t *tab = s_cnt + kWarps * kPartWords;
    if (a.ctl->error & (DERR_EB | DERR_INTERNAL)) return;
    const bool w32 = !a.cw64_only && a.ctl->maxlen <= 24;
    if (a.nbins <= kCountSmemBins) {
        for (uint32_t i = threadIdx.x; i < a.nbins; i += blockDim.x) {
            const uint32_t len = w32 ? a.cw32[i] >> 24 : (uint32_t)(a.cw64[i] >> 56);
            tab[i] = len | (i == 0 ? 0x10000u : 0u);
        }
        __syncthreads();
    }
    count_dispatch<ZB>(a, nunits, part, tab, w32, vg);
}

__global__ void __launch_bounds__(kEncThreads, 4) k_encode_count(const __grid_constant__ EncodeArgs a, uint64_t nunits)
{
    count_body<true>(a, nunits, vgrid_self());
}

__device__ __forceinline__ void pack_body(const EncodeArgs &a, uint64_t nunits, uint32_t use_smem, VGrid vg)
{
    extern __shared__ uint4 s_dyn[];
    uint4 *slot = s_dyn + (threadIdx.x >> 5) * (kRound / 8);  // 8 KB per warp
    unsigned long long *s_tab = reinterpret_cast<unsigned long long *>(s_dyn + kWarps * (kRound / 8));
    if (a.ctl->error & (DERR_EB | DERR_INTERNAL)) return;
    const bool w32 = !a.cw64_only && a.ctl->maxlen <= 24;
    // each call sees where its table lives, so shared-memory tables are read
    // with shared loads
    const bool pair = w32;
    if (use_smem) {
        load_table(a, 1, s_tab, w32, pair);
        if (pair && a.ctl->maxlen <= 16) pack_units<true, true>(a, nunits, Table<true>{s_tab}, slot, vg);
        else if (pair) pack_units<true, true, true>(a, nunits, Table<true>{s_tab}, slot, vg);
        else pack_units<false, false>(a, nunits, Table<false>{s_tab}, slot, vg);
    } else {
        if (w32) pack_units<true, false>(a, nunits, Table<true>{a.cw32}, slot, vg);
        else pack_units<false, false>(a, nunits, Table<false>{a.cw64}, slot, vg);
    }
}

__global__ void __launch_bounds__(kEncThreads, 3) k_encode_pack(const __grid_constant__ EncodeArgs a, uint64_t nunits,
                                                                uint32_t use_smem)
{
    pack_body(a, nunits, use_smem, vgrid_self());
}

// few registers and no shared memory: five blocks per SM keep many
// residual loads in flight
__global__ void __launch_bounds__(kEncThreads, 5) k_encode_outliers(const __grid_constant__ EncodeArgs a,
                                                                    uint64_t nunits)
{
    __shared__ uint16_t s_pos[kWarps * kOutWin];
    if (a.ctl->error & (DERR_EB | DERR_INTERNAL)) return;
    outlier_units(a, nunits, s_pos + (threadIdx.x >> 5) * kOutWin, vgrid_self());
}

// grouped: the count / pack of every field of a batch in one launch
__global__ void __launch_bounds__(kEncThreads, 4) k_encode_count_group(const EncodeItem *items, const uint32_t *first,
                                                                       uint32_t ni)
{
    VGrid vg;
    const EncodeItem &e = items[group_item(first, ni, vg)];
    count_body<false>(e.a, e.nunits, vg);  // batches write no bitmap
}

__global__ void __launch_bounds__(kEncThreads, 3) k_encode_pack_group(const EncodeItem *items, const uint32_t *first,
                                                                      uint32_t ni)
{
    VGrid vg;
    const EncodeItem &e = items[group_item(first, ni, vg)];
    pack_body(e.a, e.nunits, e.use_smem, vg);
}

// opt in to the dynamic shared memory the kernels need, once per device
// (host threads may race here: the bits are atomic, and setting an attribute
// twice is harmless)
void set_encode_smem()
{
    static std::atomic<unsigned long long> done{0};  // one bit per device id < 64
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0;
    if (bit && (done.load() & bit)) return;
    const size_t most = (size_t)kWarps * kRound * 2 + 4096 * 8;
    cudaFuncSetAttribute(k_encode_pack, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
    cudaFuncSetAttribute(k_encode_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)((kWarps * kPartWords + kCountSmemBins) * 4));
    cudaFuncSetAttribute(k_encode_pack_group, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
    cudaFuncSetAttribute(k_encode_count_group, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)((kWarps * kPartWords + kCountSmemBins) * 4));
    done.fetch_or(bit);
}

}  // namespace

uint32_t encode_unit_shift(uint32_t chunk)
{
    const uint32_t S = chunk < kLaneMax ? chunk : kLaneMax;
    const uint64_t U = chunk > kRound ? chunk : 32ull * S;
    uint32_t sh = 0;
    while ((1ull << sh) < U) sh++;
    return sh;
}

uint64_t encode_units(uint64_t n, uint32_t chunk)
{
    const uint32_t S = chunk < kLaneMax ? chunk : kLaneMax;
    const uint64_t U = chunk > kRound ? chunk : 32ull * S;
    return (n + U - 1) / U;
}

int launch_encode(const EncodeArgs &a, cudaStream_t st, int phase)
{
    const uint64_t nunits = encode_units(a.n, a.chunk);
    const uint32_t use_smem = a.nbins <= 4096 ? 1u : 0u;
    const size_t tab = use_smem ? (size_t)a.nbins * 8 : 0;
    set_encode_smem();
    const uint64_t want = (nunits + kWarps - 1) / kWarps;
    if (phase == 0) {
        const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)a.num_sms * 4));
        const size_t smem = (kWarps * kPartWords + (a.nbins <= kCountSmemBins ? a.nbins : 0)) * 4;
        k_encode_count<<<grid, kEncThreads, smem, st>>>(a, nunits);
        return 1;
    }
    if (phase == 1) return launch_scan(UnitScan{a.unit_tot, a.unit_off}, nunits, a.scan_part, a.ctl, st);
    const int grid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)a.num_sms * 3));
    k_encode_pack<<<grid, kEncThreads, (size_t)kWarps * kRound * 2 + tab, st>>>(a, nunits, use_smem);
    if (!a.zbits) return 1;
    const int ogrid = (int)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)a.num_sms * 5));
    k_encode_outliers<<<ogrid, kEncThreads, 0, st>>>(a, nunits);
    return 2;
}

void encode_plan(const EncodeArgs &a, EncodeItem *it, uint32_t blocks[2], size_t smem[2], uint64_t *scan_items)
{
    const uint64_t nunits = encode_units(a.n, a.chunk);
    it->a = a;
    it->nunits = nunits;
    it->use_smem = a.nbins <= 4096 ? 1u : 0u;
    const uint64_t want = (nunits + kWarps - 1) / kWarps;
    blocks[0] = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)a.num_sms * 4));
    blocks[1] = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)a.num_sms * 3));
    smem[0] = (kWarps * kPartWords + (a.nbins <= kCountSmemBins ? a.nbins : 0)) * 4;
    smem[1] = (size_t)kWarps * kRound * 2 + (it->use_smem ? (size_t)a.nbins * 8 : 0);
    *scan_items = nunits;
}

void launch_encode_group(int phase, const EncodeItem *items, const uint32_t *first, uint32_t ni, uint32_t blocks,
                         size_t smem, cudaStream_t st)
{
    set_encode_smem();
    if (phase == 0) k_encode_count_group<<<blocks, kEncThreads, smem, st>>>(items, first, ni);
    else k_encode_pack_group<<<blocks, kEncThreads, smem, st>>>(items, first, ni);
}

int launch_unit_scan_group(const ScanItem<UnitScan> *items, const uint32_t *first, uint32_t ni, uint32_t blocks,
                           cudaStream_t st)
{
    return launch_scan_group(items, first, ni, blocks, st);
}

}  // namespace gbsz
