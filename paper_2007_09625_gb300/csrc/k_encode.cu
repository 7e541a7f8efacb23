// k_encode.cu -- S5: Huffman encode + deflate (Sec. 3.2.4) and S6 archive
// assembly.
//
// The paper deflates one chunk per thread.  Here a CTA of 128 threads works
// on a unit of 4096 symbols (32 per thread; a unit holds 4096/C chunks when
// C <= 4096, or is one C-symbol chunk of C/4096 tiles otherwise):
//   pass 1  code lengths -> per-thread bit counts, block scans give each
//           chunk's bits and the unit's words, outliers and exceptions;
//   look-back  a decoupled look-back over units (bounded waits) turns unit
//           totals into global word / outlier / exception offsets;
//   pass 2  each thread packs its codewords MSB-first into a shared-memory
//           copy of the unit's words, which is written out with 16-byte
//           stores; outliers (idx, delta) and exceptions (idx, raw bits) are
//           emitted in index order at their global offsets.
// Outlier residuals were parked per point by the dual-quant kernel; whether a
// code-0 point is a verbatim exception is recomputed from the input value
// with the same prequantization function.
#include "common.cuh"

#include <algorithm>

namespace gbsz {

namespace {

constexpr int kEncThreads = 128;
constexpr int kSPT = 32;
constexpr int kTile = kEncThreads * kSPT;
constexpr int kMaxTileWords = kTile * kMaxLen / 32 + 4;

struct Entry {
    uint32_t len;
    unsigned long long code;
};

template <bool CW32>
struct Table {
    const void *tab;
    __device__ __forceinline__ Entry get(uint32_t sym) const
    {
        Entry e;
        if (CW32) {
            const uint32_t v = static_cast<const uint32_t *>(tab)[sym];
            e.len = v >> 24;
            e.code = v & 0xFFFFFFu;
        } else {
            const unsigned long long v = static_cast<const unsigned long long *>(tab)[sym];
            e.len = (uint32_t)(v >> 56);
            e.code = v & ((1ull << 56) - 1);
        }
        return e;
    }
};

// bit writer into shared-memory words; the first word starts `skip` bits in
__device__ __forceinline__ void put_bits(unsigned long long &acc, uint32_t &nacc, uint32_t &widx,
                                         uint32_t *sw, unsigned long long code, uint32_t len)
{
    if (len > 32) {
        const uint32_t hl = len - 32;
        acc = (acc << hl) | (code >> 32);
        nacc += hl;
        if (nacc >= 32) {
            atomicOr(&sw[widx++], (uint32_t)(acc >> (nacc - 32)));
            nacc -= 32;
            acc &= (1ull << nacc) - 1;
        }
        code &= 0xFFFFFFFFull;
        len = 32;
    }
    acc = (acc << len) | code;
    nacc += len;
    if (nacc >= 32) {
        atomicOr(&sw[widx++], (uint32_t)(acc >> (nacc - 32)));
        nacc -= 32;
        acc &= (1ull << nacc) - 1;
    }
}

__device__ __forceinline__ void flush_bits(unsigned long long acc, uint32_t nacc, uint32_t widx, uint32_t *sw)
{
    if (nacc) atomicOr(&sw[widx], (uint32_t)(acc << (32 - nacc)));
}

struct Smem {
    uint32_t words[kMaxTileWords];
    uint32_t e[kEncThreads + 1];
    uint32_t wo[kEncThreads + 1];
    uint32_t scan[33];
    unsigned long long scan64[33];
    uint32_t unit;
    unsigned long long excl_w, excl_oe;
    uint32_t carry;
};

__device__ __forceinline__ void load_codes(const uint16_t *codes, uint64_t n, uint64_t s0, uint32_t *cr)
{
    if (s0 + kSPT <= n) {
        const uint4 *p = reinterpret_cast<const uint4 *>(codes + s0);
#pragma unroll
        for (int v = 0; v < 4; v++) {
            const uint4 w = p[v];
            cr[4 * v + 0] = w.x;
            cr[4 * v + 1] = w.y;
            cr[4 * v + 2] = w.z;
            cr[4 * v + 3] = w.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < kSPT / 2; j++) {
            const uint32_t a = s0 + 2 * j < n ? codes[s0 + 2 * j] : 0u;
            const uint32_t b = s0 + 2 * j + 1 < n ? codes[s0 + 2 * j + 1] : 0u;
            cr[j] = a | (b << 16);
        }
    }
}

__device__ __forceinline__ uint32_t sym_of(const uint32_t *cr, int j) { return (cr[j >> 1] >> ((j & 1) * 16)) & 0xFFFFu; }

// Decoupled look-back (warp 0).  Publishes the unit's aggregate, gathers the
// exclusive prefix of (words, outliers | exceptions << 32) and publishes the
// inclusive value.
__device__ void look_back(const EncodeArgs &a, uint32_t u, unsigned long long agg_w,
                          unsigned long long agg_oe, unsigned long long &ex_w, unsigned long long &ex_oe)
{
    const int lane = threadIdx.x & 31;
    const uint32_t tag = a.epoch << 2;
    if (u == 0) {
        ex_w = 0;
        ex_oe = 0;
        if (lane == 0) {
            __stcg(&a.lb_inc[0], make_ulonglong2(agg_w, agg_oe));
            __threadfence();
            atomicExch(&a.lb_flag[0], tag | 2u);
        }
        return;
    }
    if (lane == 0) {
        __stcg(&a.lb_agg[u], make_ulonglong2(agg_w, agg_oe));
        __threadfence();
        atomicExch(&a.lb_flag[u], tag | 1u);
    }
    unsigned long long sw = 0, soe = 0;
    int64_t j = (int64_t)u - 1;
    for (;;) {
        const int64_t jj = j - lane;
        unsigned long long vw = 0, voe = 0;
        bool inc = true;
        if (jj >= 0) {
            const uint32_t f = spin_until_nonzero_epoch(&a.lb_flag[jj], a.epoch, kSpinLimit);
            if (f == 0) {
                atomicOr(&a.ctl->error, DERR_TIMEOUT);
            } else {
                __threadfence();
                inc = (f & 3u) == 2u;
                const ulonglong2 v = inc ? __ldcg(&a.lb_inc[jj]) : __ldcg(&a.lb_agg[jj]);
                vw = v.x;
                voe = v.y;
            }
        }
        const uint32_t m = __ballot_sync(0xffffffffu, inc);
        const int first = m ? __ffs(m) - 1 : 32;
        if (lane > first) {
            vw = 0;
            voe = 0;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            vw += __shfl_xor_sync(0xffffffffu, vw, o);
            voe += __shfl_xor_sync(0xffffffffu, voe, o);
        }
        sw += vw;
        soe += voe;
        if (m) break;
        j -= 32;
    }
    ex_w = sw;
    ex_oe = soe;
    if (lane == 0) {
        __stcg(&a.lb_inc[u], make_ulonglong2(sw + agg_w, soe + agg_oe));
        __threadfence();
        atomicExch(&a.lb_flag[u], tag | 2u);
    }
}

__device__ __forceinline__ void put_u32(uint8_t *p, uint32_t v) { *reinterpret_cast<uint32_t *>(p) = v; }

// archive header and the zero bytes between sections (last unit's CTA)
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
    h[H_LBLOCK / 4] = 0;
    set64(H_TOTAL, L.total);
    for (int i = 0; i < (int)(kHeaderBytes / 4); i++) put_u32(a.archive + 4 * i, h[i]);
    for (uint64_t b = L.len + a.nbins; b < L.bits; b++) a.archive[b] = 0;
    for (uint64_t b = L.bits + 4 * nchunk; b < L.outl; b++) a.archive[b] = 0;
    for (uint64_t b = L.exc + 8 * e; b < L.stream; b++) a.archive[b] = 0;
}

template <bool MULTI, bool CW32>
__device__ __forceinline__ void encode_body(const EncodeArgs &a, uint64_t nunits, uint32_t use_smem_table,
                                            Smem &s, unsigned long long *s_tab)
{
    const uint32_t t = threadIdx.x;
    const uint32_t nbins = a.nbins;
    Table<CW32> tab;
    if (use_smem_table) {
        if (CW32) {
            uint32_t *st = reinterpret_cast<uint32_t *>(s_tab);
            for (uint32_t i = t; i < nbins; i += kEncThreads) st[i] = a.cw32[i];
        } else {
            for (uint32_t i = t; i < nbins; i += kEncThreads) s_tab[i] = a.cw64[i];
        }
        tab.tab = s_tab;
    } else {
        tab.tab = CW32 ? (const void *)a.cw32 : (const void *)a.cw64;
    }
    const uint64_t n = a.n;
    const uint32_t C = a.chunk;
    const uint64_t nchunk = (n + C - 1) / C;
    const uint64_t M = a.ctl->n_out, E = a.ctl->n_exc;
    const Layout L0 = make_layout(a.radius, nchunk, M, E, 0);
    const EbScalars sc = load_scalars(a.ctl);
    const uint64_t U = MULTI ? C : kTile;

    for (;;) {
        if (t == 0) s.unit = atomicAdd(&a.ctl->ticket, 1u);
        __syncthreads();
        const uint32_t u = s.unit;
        __syncthreads();
        if (u >= nunits) break;
        const uint64_t ubase = (uint64_t)u * U;
        const uint64_t ulen = n - ubase < U ? n - ubase : U;
        const uint32_t ntile = MULTI ? (uint32_t)((ulen + kTile - 1) / kTile) : 1;

        // ---- pass 1
        uint32_t cr[kSPT / 2];
        uint32_t excmask = 0;
        uint32_t my_bits = 0, my_out = 0, my_exc = 0;
        unsigned long long unit_words = 0, unit_out = 0, unit_exc = 0;
        unsigned long long chunk_bits = 0;
        uint32_t seg_bit = 0, seg_word = 0;  // single-tile: bit offset in chunk, chunk word offset in unit
        for (uint32_t tj = 0; tj < ntile; tj++) {
            const uint64_t s0 = ubase + (uint64_t)tj * kTile + (uint64_t)t * kSPT;
            load_codes(a.codes, n, s0, cr);
            uint32_t b = 0, o = 0, ex = 0;
            excmask = 0;
#pragma unroll
            for (int j = 0; j < kSPT; j++) {
                const uint64_t i = s0 + j;
                if (i < n) {
                    const uint32_t c = sym_of(cr, j);
                    b += tab.get(c).len;
                    if (c == 0) {
                        o++;
                        bool e;
                        prequant(a.x[i], sc, e);
                        if (e) {
                            ex++;
                            excmask |= 1u << j;
                        }
                    }
                }
            }
            my_bits = b;
            my_out = o;
            my_exc = ex;
            uint32_t tot;
            const uint32_t eb_ = block_excl_scan(b, s.scan, &tot);
            if (MULTI) {
                chunk_bits += tot;
                uint32_t to, te;
                block_excl_scan(o, s.scan, &to);
                block_excl_scan(ex, s.scan, &te);
                unit_out += to;
                unit_exc += te;
            } else {
                // chunks of C/32 threads inside the 4096-symbol unit
                const uint32_t tpc = C / kSPT;
                const uint32_t cs = t - t % tpc;
                s.e[t] = eb_;
                if (t == 0) s.e[kEncThreads] = tot;
                __syncthreads();
                seg_bit = eb_ - s.e[cs];
                const bool first = t == cs;
                const uint64_t cstart = ubase + (uint64_t)cs * kSPT;
                uint32_t wc = 0;
                if (first && cstart < n) {
                    const uint32_t cb = s.e[min(cs + tpc, (uint32_t)kEncThreads)] - s.e[cs];
                    wc = (cb + 31) / 32;
                    const uint64_t c = cstart / C;
                    put_u32(a.archive + L0.bits + 4 * c, cb);
                }
                uint32_t tw;
                const uint32_t wo = block_excl_scan(wc, s.scan, &tw);
                if (first) s.wo[cs] = wo;
                unit_words = tw;
                uint32_t to, te;
                block_excl_scan(o, s.scan, &to);
                block_excl_scan(ex, s.scan, &te);
                unit_out = to;
                unit_exc = te;
                __syncthreads();
                seg_word = s.wo[cs];
            }
        }
        if (MULTI) {
            unit_words = (chunk_bits + 31) / 32;
            if (t == 0) put_u32(a.archive + L0.bits + 4 * (uint64_t)u, (uint32_t)chunk_bits);
        }

        // ---- look-back
        if (t < 32) {
            unsigned long long xw, xoe;
            look_back(a, u, unit_words, unit_out | (unit_exc << 32), xw, xoe);
            if (t == 0) {
                s.excl_w = xw;
                s.excl_oe = xoe;
                if (u == nunits - 1) {
                    const unsigned long long W = xw + unit_words;
                    const unsigned long long Mt = (xoe & 0xFFFFFFFFull) + unit_out;
                    const unsigned long long Et = (xoe >> 32) + unit_exc;
                    if (Mt != M || Et != E) atomicOr(&a.ctl->error, DERR_INTERNAL);
                    const Layout L = make_layout(a.radius, nchunk, M, E, W);
                    a.ctl->words = W;
                    a.ctl->total = L.total;
                    if (L.stream > a.capacity) atomicOr(&a.ctl->error, DERR_CAPACITY);
                    else write_header(a, L, nchunk, M, E, W, a.ctl->maxlen);
                }
            }
        }
        __syncthreads();
        const unsigned long long W0 = s.excl_w;
        const unsigned long long O0 = s.excl_oe & 0xFFFFFFFFull, E0 = s.excl_oe >> 32;

        // ---- pass 2
        unsigned long long run_bits = 0, run_out = 0, run_exc = 0;
        if (MULTI && t == 0) s.carry = 0;
        for (uint32_t tj = 0; tj < ntile; tj++) {
            const uint64_t s0 = ubase + (uint64_t)tj * kTile + (uint64_t)t * kSPT;
            uint32_t pbit, o_off, e_off, nw, wbase_rel;
            bool keep_last = false;
            if (MULTI) {
                load_codes(a.codes, n, s0, cr);
                uint32_t b = 0, o = 0, ex = 0;
                excmask = 0;
#pragma unroll
                for (int j = 0; j < kSPT; j++) {
                    const uint64_t i = s0 + j;
                    if (i < n) {
                        const uint32_t c = sym_of(cr, j);
                        b += tab.get(c).len;
                        if (c == 0) {
                            o++;
                            bool e;
                            prequant(a.x[i], sc, e);
                            if (e) {
                                ex++;
                                excmask |= 1u << j;
                            }
                        }
                    }
                }
                uint32_t tb, to, te;
                const uint32_t be = block_excl_scan(b, s.scan, &tb);
                o_off = block_excl_scan(o, s.scan, &to);
                e_off = block_excl_scan(ex, s.scan, &te);
                o_off += (uint32_t)run_out;
                e_off += (uint32_t)run_exc;
                const unsigned long long tstart = run_bits, tend = run_bits + tb;
                wbase_rel = (uint32_t)(tstart / 32);
                pbit = (uint32_t)(tstart - 32ull * wbase_rel) + be;
                nw = (uint32_t)((tend + 31) / 32 - wbase_rel);
                keep_last = (tj + 1 < ntile) && (tend % 32 != 0);
                run_bits = tend;
                run_out += to;
                run_exc += te;
                for (uint32_t i = t; i < nw; i += kEncThreads) s.words[i] = 0;
                __syncthreads();
                if (t == 0 && (tstart % 32)) s.words[0] = s.carry;
                __syncthreads();
            } else {
                uint32_t to, te;
                o_off = block_excl_scan(my_out, s.scan, &to);
                e_off = block_excl_scan(my_exc, s.scan, &te);
                wbase_rel = 0;
                pbit = seg_word * 32 + seg_bit;
                nw = (uint32_t)unit_words;
                for (uint32_t i = t; i < nw; i += kEncThreads) s.words[i] = 0;
                __syncthreads();
            }
            // pack codewords
            {
                unsigned long long acc = 0;
                uint32_t nacc = pbit % 32, widx = pbit / 32;
#pragma unroll
                for (int j = 0; j < kSPT; j++) {
                    if (s0 + j < n) {
                        const Entry en = tab.get(sym_of(cr, j));
                        put_bits(acc, nacc, widx, s.words, en.code, en.len);
                    }
                }
                flush_bits(acc, nacc, widx, s.words);
            }
            // outliers and exceptions in index order
            {
                uint32_t ko = 0, ke = 0;
                const uint64_t oe_base = L0.outl + 8 * (O0 + o_off);
                for (int j = 0; j < kSPT; j++) {
                    const uint64_t i = s0 + j;
                    if (i < n && sym_of(cr, j) == 0) {
                        const uint64_t off = oe_base + 8ull * ko++;
                        if (off + 8 <= a.capacity) {
                            put_u32(a.archive + off, (uint32_t)i);
                            put_u32(a.archive + off + 4, (uint32_t)a.dscr[i]);
                        } else {
                            atomicOr(&a.ctl->error, DERR_CAPACITY);
                        }
                        if (excmask & (1u << j)) {
                            const uint64_t eo = L0.outl + 8 * M + 8 * (E0 + e_off + ke++);
                            if (eo + 8 <= a.capacity) {
                                put_u32(a.archive + eo, (uint32_t)i);
                                put_u32(a.archive + eo + 4, __float_as_uint(a.x[i]));
                            } else {
                                atomicOr(&a.ctl->error, DERR_CAPACITY);
                            }
                        }
                    }
                }
            }
            __syncthreads();
            // write the staged words: global word index W0 + wbase_rel + i
            {
                const uint32_t nflush = keep_last ? nw - 1 : nw;
                const unsigned long long gw0 = W0 + wbase_rel;
                const Layout L = make_layout(a.radius, nchunk, M, E, 0);
                if (L.stream + 4 * (gw0 + nflush) > a.capacity) {
                    if (t == 0 && nflush) atomicOr(&a.ctl->error, DERR_CAPACITY);
                } else {
                    uint32_t *dst = reinterpret_cast<uint32_t *>(a.archive + L.stream) + gw0;
                    const uint32_t head = min((uint32_t)((4 - (gw0 & 3)) & 3), nflush);
                    if (t < head) dst[t] = s.words[t];
                    const uint32_t nvec = (nflush - head) / 4;
                    uint4 *dv = reinterpret_cast<uint4 *>(dst + head);
                    for (uint32_t v = t; v < nvec; v += kEncThreads) {
                        const uint32_t b = head + 4 * v;
                        dv[v] = make_uint4(s.words[b], s.words[b + 1], s.words[b + 2], s.words[b + 3]);
                    }
                    for (uint32_t i = head + 4 * nvec + t; i < nflush; i += kEncThreads) dst[i] = s.words[i];
                }
                if (MULTI && t == 0) s.carry = keep_last ? s.words[nw - 1] : 0u;
            }
            __syncthreads();
        }
    }
}

// The codeword width is chosen on the device from the longest code length
// the codebook kernel found: 32-bit entries when it is at most 24 bits.
template <bool MULTI>
__global__ void __launch_bounds__(kEncThreads) k_encode(EncodeArgs a, uint64_t nunits, uint32_t use_smem_table)
{
    __shared__ Smem s;
    extern __shared__ unsigned long long s_tab[];
    if (a.ctl->error & (DERR_EB | DERR_INTERNAL)) return;
    if (a.ctl->maxlen <= 24) encode_body<MULTI, true>(a, nunits, use_smem_table, s, s_tab);
    else encode_body<MULTI, false>(a, nunits, use_smem_table, s, s_tab);
}

}  // namespace

void launch_encode(const EncodeArgs &a, cudaStream_t st)
{
    const bool multi = a.chunk > (uint32_t)kTile;
    const uint64_t U = multi ? a.chunk : kTile;
    const uint64_t nunits = (a.n + U - 1) / U;
    const uint32_t use_smem = a.nbins <= 4096 ? 1u : 0u;
    const size_t tab_bytes = use_smem ? (size_t)a.nbins * 8 : 0;
    const int grid = (int)std::min<uint64_t>(nunits, (uint64_t)a.num_sms * 12);
    if (multi) k_encode<true><<<grid, kEncThreads, tab_bytes, st>>>(a, nunits, use_smem);
    else k_encode<false><<<grid, kEncThreads, tab_bytes, st>>>(a, nunits, use_smem);
}

}  // namespace gbsz
