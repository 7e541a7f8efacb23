// k_codebook.cu -- S4: Huffman code lengths, canonical codebook and the
// decoder's reverse codebook, each built by one CTA on the device so no
// frequency table or codebook crosses PCIe (Sec. 3.2.2, 3.2.3).
//
// Tree: leaves sorted by (frequency, symbol); the two-queue merge takes the
// leaf on equal frequency.  The paper builds the tree with one GPU thread;
// here the merge runs in phases: with a, b the two smallest available nodes,
// every available node of frequency <= a + b is consumed before any node not
// yet created (those are all >= a + b and lose ties), so that whole prefix is
// paired at once, pair j creating internal node j of the phase.  This yields
// exactly the serial merge's tree.  Depths by pointer jumping (depth <= 45).
//
// Canonization (Sec. 3.2.3): symbols in (length, symbol) order, first code 0,
// next = (prev + 1) << (len - prevlen); the order is found by counting, not
// sorting.  Codeword tables hold (len, code) as
// len << 24 | code in 32 bits when the longest code fits 24 bits, and
// len << 56 | code in 64 bits always (the paper's adaptive representation).
#include "common.cuh"

#include <atomic>

namespace gbsz {

namespace {

// one CTA of 1024 threads (measured against 256 and 512: the codebook kernel
// is within 10% for every bin count, the decoder tables are fastest here)
constexpr int kCbThreads = 1024;
constexpr uint32_t kBitonicMax = 8192;    // 8192 keys = 64 KB of shared memory
// merge state (4k words) in shared memory up to this many used symbols, and
// the pointer-jumping buffers too (12k words in all) up to kDepthSmemMax
// (the dynamic shared memory is 32K words)
constexpr uint32_t kMergeSmemMax = 8192;
constexpr uint32_t kDepthSmemMax = 2048;

// Stable sort of n unique 64-bit keys by bits [bit_lo, bit_hi); the keys are
// already ordered by the bits below bit_lo.  Returns the buffer holding the
// result (a or b).  s_cnt: 16 * blockDim.x words of shared memory.
__device__ unsigned long long *cta_sort(unsigned long long *a, unsigned long long *b, uint32_t n,
                                        int bit_lo, int bit_hi, uint32_t *s_cnt)
{
    const uint32_t T = blockDim.x, t = threadIdx.x;
    if (n <= 1 || bit_lo >= bit_hi) return a;
    if (n <= kBitonicMax) {
        // bitonic sort in shared memory of the full (unique) keys, padded to a
        // power of two with all-ones keys; the order of unique keys is the
        // order by the selected bits with ties in their original order,
        // because every caller's low bits (the symbol) ascend in input order
        unsigned long long *sk = reinterpret_cast<unsigned long long *>(s_cnt);
        uint32_t m = 1;
        while (m < n) m <<= 1;
        const unsigned long long hmask = bit_hi >= 64 ? ~0ull : ((1ull << bit_hi) - 1);
        for (uint32_t i = t; i < m; i += T) sk[i] = i < n ? (a[i] & hmask) : ~0ull;
        __syncthreads();
        for (uint32_t size = 2; size <= m; size <<= 1) {
            for (uint32_t stride = size >> 1; stride > 0; stride >>= 1) {
                for (uint32_t p = t; p < m / 2; p += T) {
                    const uint32_t i = 2 * p - (p & (stride - 1));  // lower index of the pair
                    const uint32_t j = i + stride;
                    const bool up = (i & size) == 0;
                    const unsigned long long x = sk[i], y = sk[j];
                    if ((x > y) == up) {
                        sk[i] = y;
                        sk[j] = x;
                    }
                }
                __syncthreads();
            }
        }
        for (uint32_t i = t; i < n; i += T) b[i] = sk[i];
        __syncthreads();
        return b;
    }
    const uint32_t per = (n + T - 1) / T;
    const uint32_t lo = min(n, t * per), hi = min(n, lo + per);
    __shared__ uint32_t s_scan[33];
    for (int bit = bit_lo; bit < bit_hi; bit += 4) {
        for (int d = 0; d < 16; d++) s_cnt[d * T + t] = 0;
        for (uint32_t i = lo; i < hi; i++) s_cnt[((a[i] >> bit) & 15u) * T + t]++;
        __syncthreads();
        // exclusive scan of the digit-major count matrix
        uint32_t loc = 0;
        for (int j = 0; j < 16; j++) loc += s_cnt[16 * t + j];
        uint32_t tot;
        uint32_t run = block_excl_scan(loc, s_scan, &tot);
        for (int j = 0; j < 16; j++) {
            const uint32_t c = s_cnt[16 * t + j];
            s_cnt[16 * t + j] = run;
            run += c;
        }
        __syncthreads();
        for (uint32_t i = lo; i < hi; i++) {
            const unsigned long long k = a[i];
            const uint32_t d = (uint32_t)((k >> bit) & 15u);
            b[s_cnt[d * T + t]++] = k;
        }
        __syncthreads();
        unsigned long long *tmp = a;
        a = b;
        b = tmp;
    }
    return a;
}

struct Canon {
    unsigned long long first[kMaxLen + 2];
    uint32_t count[kMaxLen + 2];
    uint32_t start[kMaxLen + 2];
};

// Canonical codes from lengths (all threads), without sorting: a symbol's
// place in (length, symbol) order is the start of its length plus the number
// of symbols before it with the same length.  Symbols go T at a time; in each
// pass a warp ranks its lanes among equal lengths (match_any), the per-warp
// counts of every length are scanned across the warps, and the running
// offset of every length then advances by the pass's count.  Fills sh
// (tables), writes sorted symbols (if non-NULL) and per-symbol codewords (if
// non-NULL).  s_cnt: at least 34 * (kMaxLen + 2) words.
__device__ void canonicalize(const uint8_t *len, uint32_t nbins, uint32_t *s_cnt, Canon &sh, uint16_t *sorted,
                             uint64_t *cw64, uint32_t *cw32, uint64_t *codes_only, uint32_t maxlen)
{
    constexpr uint32_t L = kMaxLen + 2;
    const uint32_t T = blockDim.x, t = threadIdx.x, lane = t & 31, w = t >> 5, W = (T + 31) >> 5;
    uint32_t *wcnt = s_cnt;           // [W][L]: per-warp counts, then their exclusive scan over warps
    uint32_t *base = s_cnt + 32 * L;  // [L]: first place of each length in the current pass
    uint32_t *ptot = base + L;        // [L]: the pass's count of each length
    for (uint32_t l = t; l < L; l += T) sh.count[l] = 0;
    __syncthreads();
    for (uint32_t s = t; s < nbins; s += T) {
        const uint32_t l = len[s];
        if (l) atomicAdd(&sh.count[l], 1u);
    }
    __syncthreads();
    if (t == 0) {
        uint32_t st = 0;
        unsigned long long f = 0;
        for (uint32_t l = 0; l < L; l++) {
            sh.start[l] = st;
            sh.first[l] = f;
            if (l >= 1) {
                st += sh.count[l];
                f = (f + sh.count[l]) << 1;
            }
        }
        sh.start[0] = 0;
        sh.first[0] = 0;
    }
    __syncthreads();
    for (uint32_t l = t; l < L; l += T) base[l] = sh.start[l];
    for (uint32_t c0 = 0; c0 < nbins; c0 += T) {
        const uint32_t s = c0 + t;
        const uint32_t l = s < nbins ? len[s] : 0u;
        if (!__syncthreads_or(l != 0)) continue;  // no used symbol in these bins
        const uint32_t peers = __match_any_sync(0xffffffffu, l);
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        for (uint32_t i = t; i < W * L; i += T) wcnt[i] = 0;
        __syncthreads();
        if (rank == 0 && l) wcnt[w * L + l] = __popc(peers);
        __syncthreads();
        for (uint32_t li = t; li < L; li += T) {
            uint32_t run = 0;
            for (uint32_t ww = 0; ww < W; ww++) {
                const uint32_t c = wcnt[ww * L + li];
                wcnt[ww * L + li] = run;
                run += c;
            }
            ptot[li] = run;
        }
        __syncthreads();
        if (l) {
            const uint32_t p = base[l] + wcnt[w * L + l] + rank;
            const unsigned long long code = sh.first[l] + (p - sh.start[l]);
            if (sorted) sorted[p] = (uint16_t)s;
            if (cw64) cw64[s] = ((unsigned long long)l << 56) | code;
            if (cw32) cw32[s] = maxlen <= 24 ? ((l << 24) | (uint32_t)code) : 0u;
            if (codes_only) codes_only[s] = code;
        }
        __syncthreads();
        for (uint32_t li = t; li < L; li += T) base[li] += ptot[li];
    }
    __syncthreads();
}

// The two-queue merge pair by pair on one thread, from the state (x leaves,
// y internal nodes consumed, ni internal nodes made) to the end: leaf first
// on equal frequency, internal nodes numbered in creation order.  The queue
// heads and the nodes after them are kept in registers, so only the loads of
// the next-but-one nodes are issued per pair, off the critical path.
__device__ void serial_merge_from(const uint32_t *LF, uint32_t *F, uint32_t *P, uint32_t k, uint32_t x, uint32_t y,
                                  uint32_t ni)
{
    uint32_t lx = x < k ? LF[x] : 0u, lxn = x + 1 < k ? LF[x + 1] : 0u;
    uint32_t fy = y < ni ? F[y] : 0u, fyn = y + 1 < ni ? F[y + 1] : 0u;
    for (; ni + 1 < k; ni++) {
        uint32_t f = 0;
        for (int r = 0; r < 2; r++) {
            if (x < k && (y >= ni || lx <= fy)) {
                f += lx;
                P[x] = k + ni;
                x++;
                lx = lxn;
                lxn = x + 1 < k ? LF[x + 1] : 0u;
            } else {
                f += fy;
                P[k + y] = k + ni;
                y++;
                fy = fyn;
                fyn = y + 1 < ni ? F[y + 1] : 0u;
            }
        }
        F[ni] = f;
        if (y == ni) fy = f;  // the node just made heads the internal queue
        else if (y + 1 == ni) fyn = f;
    }
}

// Entries of the ascending A[lo..hi) that are <= v, as lo + their count; the
// whole warp (32-ary search: each round a probe per lane and a ballot).
__device__ __forceinline__ uint32_t warp_upper(const uint32_t *A, uint32_t lo, uint32_t hi, unsigned long long v)
{
    const uint32_t lane = threadIdx.x & 31;
    while (hi - lo > 32) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t i = lo + lane * step;
        const uint32_t c = __popc(__ballot_sync(0xffffffffu, i < hi && (unsigned long long)A[i] <= v));
        if (c == 0) return lo;
        // the first entry above v lies after probe c - 1, at or before probe c
        const uint32_t nhi = c < 32 ? min(hi, lo + c * step) : hi;
        lo = lo + (c - 1) * step + 1;
        hi = nhi;
    }
    const uint32_t i = lo + lane;
    return lo + __popc(__ballot_sync(0xffffffffu, i < hi && (unsigned long long)A[i] <= v));
}

// The phases of the merge on one warp, from the state (lh leaves, ih internal
// nodes consumed, ni made): searches by ballot, the pairs of a phase spread
// over the lanes, warp barriers only; the last two pairs or fewer go
// serially.  Returns the internal nodes made (k - 1 when complete).
__device__ uint32_t warp_merge_from(const uint32_t *LF, uint32_t *F, uint32_t *P, uint32_t k, uint32_t lh,
                                    uint32_t ih, uint32_t ni)
{
    const uint32_t lane = threadIdx.x & 31;
    while ((k - lh) + (ni - ih) > 1) {
        uint32_t x = lh, y = ih;
        unsigned long long f2 = 0;
        for (int r = 0; r < 2; r++) {
            if (x < k && (y >= ni || LF[x] <= F[y])) f2 += LF[x++];
            else f2 += F[y++];
        }
        const uint32_t cl = warp_upper(LF, lh, k, f2) - lh, ci = warp_upper(F, ih, ni, f2) - ih;
        const uint32_t np = (cl + ci) >> 1;
        if (np <= 2) {
            if (lane == 0) serial_merge_from(LF, F, P, k, lh, ih, ni);
            __syncwarp();
            return k - 1;
        }
        uint32_t xend = 0;  // leaves consumed through this lane's last pair
        for (uint32_t p = lane; p < np; p += 32) {
            const uint32_t d = 2 * p;
            uint32_t l0 = d > ci ? d - ci : 0, l1 = min(d, cl);
            while (l0 < l1) {  // merge-path split: leaves among the first d merged nodes
                const uint32_t m = (l0 + l1) >> 1, b = d - m;
                if (b == 0 || m == cl || F[ih + b - 1] < LF[lh + m]) l1 = m;
                else l0 = m + 1;
            }
            uint32_t xx = l0, yy = d - l0, f = 0;
            for (int r = 0; r < 2; r++) {
                if (xx < cl && (yy >= ci || LF[lh + xx] <= F[ih + yy])) {
                    f += LF[lh + xx];
                    P[lh + xx] = k + ni + p;
                    xx++;
                } else {
                    f += F[ih + yy];
                    P[k + ih + yy] = k + ni + p;
                    yy++;
                }
            }
            F[ni + p] = f;
            xend = xx;
        }
        __syncwarp();
        const uint32_t xn = __shfl_sync(0xffffffffu, xend, (np - 1) & 31);
        lh += xn;
        ih += 2 * np - xn;
        ni += np;
    }
    return ni;
}

// a phase pairing fewer nodes than this (one per lane) continues on one warp
constexpr uint32_t kWarpPhaseMin = 32;

// Two-queue Huffman merge in phases (all threads).  LF: leaf frequencies in
// (frequency, symbol) order; F: internal frequencies in creation order; P:
// parent of every node (leaves 0..k-1, internal node i has id k+i).  With a,
// b the two smallest available nodes, every available node of frequency
// <= a + b is consumed, in merge order (leaf first on equal frequency),
// before any node not yet created, so the phase pairs that whole prefix.
// Once a phase would pair fewer than kWarpPhaseMin nodes, warp 0 finishes
// (when the arrays are in shared memory: in global memory the warp's
// dependent searches wait on L2 and the block's phases are faster).
__device__ void phase_merge(const uint32_t *LF, uint32_t *F, uint32_t *P, uint32_t k, bool in_smem, Control *ctl)
{
    __shared__ uint32_t s_lh, s_ih, s_ni, s_cl, s_ci, s_np, s_warp;
    const uint32_t t = threadIdx.x, T = blockDim.x;
    if (t == 0) {
        s_lh = 0;
        s_ih = 0;
        s_ni = 0;
        s_warp = 0;
    }
    __syncthreads();
    for (;;) {
        if (t == 0) {
            const uint32_t lh = s_lh, ih = s_ih, ni = s_ni;
            if ((k - lh) + (ni - ih) <= 1) {
                s_np = 0;
            } else {
                uint32_t x = lh, y = ih;
                unsigned long long f2 = 0;
                for (int r = 0; r < 2; r++) {
                    if (x < k && (y >= ni || LF[x] <= F[y])) f2 += LF[x++];
                    else f2 += F[y++];
                }
                // counts of available nodes with frequency <= f2
                uint32_t l0 = lh, l1 = k;
                while (l0 < l1) {
                    const uint32_t m = (l0 + l1) >> 1;
                    if ((unsigned long long)LF[m] <= f2) l0 = m + 1;
                    else l1 = m;
                }
                uint32_t i0 = ih, i1 = ni;
                while (i0 < i1) {
                    const uint32_t m = (i0 + i1) >> 1;
                    if ((unsigned long long)F[m] <= f2) i0 = m + 1;
                    else i1 = m;
                }
                s_cl = l0 - lh;
                s_ci = i0 - ih;
                s_np = (s_cl + s_ci) >> 1;
                // a small phase: its searches and block barriers cost more
                // than its pairs (a skewed distribution makes many of them)
                if (in_smem && s_np < kWarpPhaseMin) {
                    s_warp = 1;
                    s_np = 0;
                }
            }
        }
        __syncthreads();
        const uint32_t np = s_np;
        if (np == 0) break;
        const uint32_t lh = s_lh, ih = s_ih, ni = s_ni, cl = s_cl, ci = s_ci;
        // merge-path split: number of leaves among the first d merged nodes
        auto split = [&](uint32_t d) -> uint32_t {
            uint32_t l0 = d > ci ? d - ci : 0, l1 = min(d, cl);
            while (l0 < l1) {
                const uint32_t m = (l0 + l1) >> 1, b = d - m;
                if (b == 0 || m == cl || F[ih + b - 1] < LF[lh + m]) l1 = m;
                else l0 = m + 1;
            }
            return l0;
        };
        for (uint32_t p = t; p < np; p += T) {
            uint32_t x = split(2 * p), y = 2 * p - x;
            uint32_t f = 0;
            for (int r = 0; r < 2; r++) {
                if (x < cl && (y >= ci || LF[lh + x] <= F[ih + y])) {
                    f += LF[lh + x];
                    P[lh + x] = k + ni + p;
                    x++;
                } else {
                    f += F[ih + y];
                    P[k + ih + y] = k + ni + p;
                    y++;
                }
            }
            F[ni + p] = f;
        }
        __syncthreads();
        if (t == 0) {
            const uint32_t x = split(2 * np);
            s_lh = lh + x;
            s_ih = ih + (2 * np - x);
            s_ni = ni + np;
        }
        __syncthreads();
    }
    if (s_warp && t < 32) {
        const uint32_t made = warp_merge_from(LF, F, P, k, s_lh, s_ih, s_ni);
        if (t == 0) s_ni = made;
    }
    __syncthreads();
    if (t == 0 && s_ni != k - 1) atomicOr(&ctl->error, DERR_INTERNAL);
    __syncthreads();
}

__device__ __forceinline__ void codebook_body(const CodebookArgs &a)
{
    extern __shared__ uint32_t s_cnt[];  // kCbSmem bytes
    __shared__ Canon canon;
    __shared__ uint32_t s_scan[33];
    __shared__ unsigned long long s_scan64[33];
    const uint32_t T = blockDim.x, t = threadIdx.x, nbins = a.nbins;

    // symbols with nonzero frequency, keys (freq << 16 | sym) in symbol order:
    // warp w takes a contiguous run of bins in rounds of 32 consecutive bins
    // (coalesced loads; ballot ranks keep the symbol order)
    const uint32_t lane = t & 31, w = t >> 5, W = T >> 5;
    const uint32_t seg = ((nbins + 32 * W - 1) / (32 * W)) * 32;
    const uint32_t wlo = min(nbins, w * seg), whi = min(nbins, wlo + seg);
    uint32_t c = 0, fmax = 0;
    unsigned long long ftot = 0;
    for (uint32_t s0 = wlo; s0 < whi; s0 += 32) {
        const uint32_t s = s0 + lane;
        const uint32_t f = s < whi ? a.hist[s] : 0u;
        c += f > 0;
        fmax = max(fmax, f);
        ftot += f;
    }
    const uint32_t wc = __reduce_add_sync(0xffffffffu, c);
    uint32_t k;
    uint32_t wbase = block_excl_scan(lane == 0 ? wc : 0u, s_scan, &k);
    wbase = __shfl_sync(0xffffffffu, wbase, 0);
    fmax = block_max(fmax, s_scan);
    // the merge adds frequencies in 32 bits: a histogram whose total reaches
    // 2^32 is refused (the compressor's fields have fewer than 2^32 points)
    unsigned long long total;
    block_excl_scan64(ftot, s_scan64, &total);
    if (total >= (1ull << 32)) {
        if (t == 0) atomicOr(&a.ctl->error, DERR_RANGE);
        return;
    }
    for (uint32_t s0 = wlo; s0 < whi; s0 += 32) {
        const uint32_t s = s0 + lane;
        const uint32_t f = s < whi ? a.hist[s] : 0u;
        const unsigned used = __ballot_sync(0xffffffffu, f > 0);
        if (f) a.keyA[wbase + __popc(used & ((1u << lane) - 1u))] = ((unsigned long long)f << 16) | s;
        wbase += __popc(used);
    }
    for (uint32_t s = t; s < nbins; s += T) {
        a.len_out[s] = 0;
        a.cw64[s] = 0;
        a.cw32[s] = 0;
        a.codes_only[s] = 0;
    }
    __syncthreads();
    if (k == 0) {
        if (t == 0) atomicOr(&a.ctl->error, DERR_INTERNAL);
        return;
    }
    const int fbits = 32 - __clz(fmax);
    unsigned long long *K = cta_sort(a.keyA, a.keyB, k, 16, 16 + ((fbits + 3) & ~3), s_cnt);
    uint32_t maxlen = 1;
    if (k == 1) {
        if (t == 0) a.len_out[K[0] & 0xFFFFu] = 1;
    } else {
        // leaf frequencies, internal frequencies and parents: in shared memory
        // (the sort's buffer, free now) up to kMergeSmemMax used symbols
        const bool sm_merge = k <= kMergeSmemMax;
        uint32_t *LF = sm_merge ? s_cnt : a.distB;
        uint32_t *F = sm_merge ? LF + k : a.nodef;
        uint32_t *P = sm_merge ? F + k : a.parent;
        for (uint32_t i = t; i < k; i += T) LF[i] = (uint32_t)(K[i] >> 16);
        __syncthreads();
        phase_merge(LF, F, P, k, sm_merge, a.ctl);
        // depths by pointer jumping over 2k-1 nodes; root = 2k-2; depth <= 45
        const bool sm_depth = k <= kDepthSmemMax;
        const uint32_t N = 2 * k - 1, root = N - 1;
        uint32_t *pa = sm_depth ? P + 2 * k : a.parA, *da = sm_depth ? pa + 2 * k : a.distA;
        uint32_t *pb = sm_depth ? da + 2 * k : a.parB, *db = sm_depth ? pb + 2 * k : a.distB;
        for (uint32_t i = t; i < N; i += T) {
            pa[i] = i == root ? root : P[i];
            da[i] = i == root ? 0u : 1u;
        }
        __syncthreads();
        for (int r = 0; r < 6; r++) {
            for (uint32_t i = t; i < N; i += T) {
                const uint32_t p = pa[i];
                db[i] = da[i] + da[p];
                pb[i] = pa[p];
            }
            __syncthreads();
            uint32_t *tp = pa; pa = pb; pb = tp;
            tp = da; da = db; db = tp;
        }
        uint32_t ml = 0;
        for (uint32_t i = t; i < k; i += T) {
            const uint32_t d = da[i];
            ml = max(ml, d);
            if (GBSZ_CHECK((K[i] & 0xFFFFu) < a.nbins, a.ctl)) a.len_out[K[i] & 0xFFFFu] = (uint8_t)min(d, 255u);
        }
        maxlen = block_max(ml, s_scan);
        if (t == 0 && maxlen > kMaxLen) atomicOr(&a.ctl->error, DERR_INTERNAL);
    }
    __syncthreads();
    if (t == 0) {
        a.ctl->maxlen = maxlen;
        a.ctl->nsym = k;
    }
    if (maxlen > kMaxLen) return;
    canonicalize(a.len_out, nbins, s_cnt, canon, nullptr, a.cw64, a.cw32, a.codes_only, maxlen);
}

__global__ void __launch_bounds__(kCbThreads, 1) k_codebook(const __grid_constant__ CodebookArgs a)
{
    codebook_body(a);
}

// grouped: block i builds field i's codebook
__global__ void __launch_bounds__(kCbThreads, 1) k_codebook_group(const CodebookArgs *items)
{
    codebook_body(items[blockIdx.x]);
}

// Reverse codebook for decoding: validates the length table (every length
// <= 45, the header's maximum matches, Kraft sum <= 1), then builds the
// canonical tables and a 2^12-entry lookup of (symbol, length) for codes of
// at most 12 bits.
__device__ __forceinline__ void decode_tables_body(const CodebookArgs &a)
{
    extern __shared__ uint32_t s_cnt[];
    __shared__ Canon canon;
    __shared__ uint32_t s_scan[33];
    __shared__ unsigned long long s_scan64[33];
    __shared__ uint32_t s_bad;
    const uint32_t T = blockDim.x, t = threadIdx.x, nbins = a.nbins;
    if (t == 0) s_bad = 0;
    __syncthreads();
    uint32_t ml = 0;
    unsigned long long kr = 0;
    for (uint32_t s = t; s < nbins; s += T) {
        const uint32_t l = a.len_in[s];
        if (l > kMaxLen) atomicOr(&s_bad, 1u);
        ml = max(ml, l);
    }
    ml = block_max(ml, s_scan);
    if (ml == 0 || ml != a.expect_maxlen) atomicOr(&s_bad, 1u);
    __syncthreads();
    if (s_bad) {
        if (t == 0) atomicOr(&a.ctl->error, DERR_CORRUPT);
        return;
    }
    for (uint32_t s = t; s < nbins; s += T) {
        const uint32_t l = a.len_in[s];
        if (l) kr += 1ull << (ml - l);
    }
    unsigned long long ktot;
    block_excl_scan64(kr, s_scan64, &ktot);
    if (ktot > (1ull << ml)) {
        if (t == 0) atomicOr(&a.ctl->error, DERR_CORRUPT);
        return;
    }
    canonicalize(a.len_in, nbins, s_cnt, canon, a.sorted, nullptr, nullptr, nullptr, ml);
    for (uint32_t l = t; l < kMaxLen + 2; l += T) {
        a.first[l] = canon.first[l];
        a.count[l] = canon.count[l];
        a.start[l] = canon.start[l];
    }
    // lookup table: canonical decode of every 12-bit prefix
    uint32_t lo = 1u << kLutBits;  // smallest prefix that starts a longer code
    for (uint32_t v = t; v < (1u << kLutBits); v += T) {
        uint32_t e = 0;
        for (uint32_t l = 1; l <= (uint32_t)kLutBits && l <= ml; l++) {
            const unsigned long long code = v >> (kLutBits - l);
            const unsigned long long off = code - canon.first[l];
            if (off < canon.count[l]) {
                e = GBSZ_CHECK(canon.start[l] + off < a.nbins, a.ctl)
                        ? ((uint32_t)a.sorted[canon.start[l] + off] << 8) | l
                        : 0u;
                break;
            }
        }
        a.lut[v] = e;
        if (e == 0) lo = min(lo, v);
    }
    lo = (1u << kLutBits) - 1 - block_max((1u << kLutBits) - 1 - min(lo, (1u << kLutBits) - 1), s_scan);
    // second level under the prefixes lo .. lo + kLut2Prefixes - 1
    uint32_t *l2w = a.lut + (1u << kLutBits);
    uint16_t *l2 = reinterpret_cast<uint16_t *>(l2w + 1);
    if (t == 0) l2w[0] = lo;
    for (uint32_t k = t; k < kLut2Entries; k += T) {
        const uint32_t v = lo + (k >> kLut2Bits);
        const uint32_t pat = (v << kLut2Bits) | (k & ((1u << kLut2Bits) - 1));  // 16-bit string
        uint32_t e = 0;
        for (uint32_t l = kLutBits + 1; v < (1u << kLutBits) && l <= kLutBits + kLut2Bits && l <= ml; l++) {
            const unsigned long long off = (unsigned long long)(pat >> (kLutBits + kLut2Bits - l)) - canon.first[l];
            if (off < canon.count[l]) {
                const uint32_t sym = GBSZ_CHECK(canon.start[l] + off < a.nbins, a.ctl) ? a.sorted[canon.start[l] + off] : 0xFFFFu;
                if (sym < 2048u) e = (sym << 5) | l;
                break;
            }
        }
        l2[k] = (uint16_t)e;
    }
    // complete table over fast_bits-bit prefixes (every code fits)
    const uint32_t B = a.fast_bits;
    auto code_at = [&](uint32_t bits, uint32_t nb, uint32_t &len) -> uint32_t {
        // the code that starts the nb-bit string `bits` (MSB first), if any
        for (uint32_t l = 1; l <= nb; l++) {
            const unsigned long long off = (unsigned long long)(bits >> (nb - l)) - canon.first[l];
            if (off < canon.count[l]) {
                len = l;
                return GBSZ_CHECK(canon.start[l] + off < a.nbins, a.ctl) ? a.sorted[canon.start[l] + off] : 0u;
            }
        }
        len = 0;
        return 0;
    };
    for (uint32_t v = t; B && v < (1u << B); v += T) {
        uint32_t l1, l2 = 0, s2 = 0;
        const uint32_t s1 = code_at(v, B, l1);
        if (!a.fast_pair) {
            static_cast<uint16_t *>(a.lutf)[v] = (uint16_t)(l1 ? (s1 << 4) | l1 : 0u);
            continue;
        }
        if (l1 && l1 < B) {
            s2 = code_at(v & ((1u << (B - l1)) - 1), B - l1, l2);
            if (!l2) s2 = 0;
        }
        static_cast<uint32_t *>(a.lutf)[v] = l1 ? (l1 | (l2 << 4) | (s1 << 8) | (s2 << 20)) : 0u;
    }
}

__global__ void __launch_bounds__(kCbThreads, 1) k_decode_tables(const __grid_constant__ CodebookArgs a)
{
    decode_tables_body(a);
}

// grouped: block i builds field i's decode tables
__global__ void __launch_bounds__(kCbThreads, 1) k_decode_tables_group(const CodebookArgs *items)
{
    decode_tables_body(items[blockIdx.x]);
}

// 32K words: 8192 sort keys (or 16 digit counters per thread), and the merge
// of up to kMergeSmemMax used symbols
constexpr size_t kCbSmem = 32 * 1024 * sizeof(uint32_t);

// opt in to more than 48 KB of dynamic shared memory, once per device
// (host threads may race here: the bits are atomic, and setting an attribute
// twice is harmless)
void set_smem_attributes()
{
    static std::atomic<unsigned long long> done{0};  // one bit per device id < 64
    int dev = 0;
    cudaGetDevice(&dev);
    const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0;
    if (bit && (done.load() & bit)) return;
    cudaFuncSetAttribute(k_codebook, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCbSmem);
    cudaFuncSetAttribute(k_decode_tables, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCbSmem);
    cudaFuncSetAttribute(k_codebook_group, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCbSmem);
    cudaFuncSetAttribute(k_decode_tables_group, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kCbSmem);
    done.fetch_or(bit);
}

}  // namespace

void launch_codebook(const CodebookArgs &a, cudaStream_t st)
{
    set_smem_attributes();
    k_codebook<<<1, kCbThreads, kCbSmem, st>>>(a);
}

void launch_codebook_group(const CodebookArgs *items, uint32_t count, cudaStream_t st)
{
    set_smem_attributes();
    k_codebook_group<<<count, kCbThreads, kCbSmem, st>>>(items);
}

void launch_decode_tables(const CodebookArgs &a, cudaStream_t st)
{
    set_smem_attributes();
    k_decode_tables<<<1, kCbThreads, kCbSmem, st>>>(a);
}

void launch_decode_tables_group(const CodebookArgs *items, uint32_t count, cudaStream_t st)
{
    set_smem_attributes();
    k_decode_tables_group<<<count, kCbThreads, kCbSmem, st>>>(items);
}

}  // namespace gbsz
