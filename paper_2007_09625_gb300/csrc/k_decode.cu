// k_decode.cu -- S7: Huffman decode (inflate, Sec. 3.3).
//
// Chunk word offsets are the exclusive prefix sum of ceil(bits/32) over the
// archive's chunk table (three coalesced scan kernels).  Decoding is
// sequential inside a chunk, as in the paper; one thread decodes one chunk
// through a two-word bit window fed by a four-word look-ahead queue (each word
// is requested four refills before it is needed, so refills do not stall the
// warp) and a 4096-entry shared-memory table that resolves every code of at
// most 12 bits in one lookup; longer codes fall back to the canonical
// per-length tables, also in shared memory.  Decoded codes leave in 16-byte stores.  Every chunk
// must consume exactly its recorded bit count and every code must exist in
// the codebook; anything else marks the archive corrupt.  For 1D fields the
// decoder also accumulates the residual sum of every 4096-point tile (in-cap
// codes only; outliers are added by the scatter), which the reconstruction
// scans instead of making another pass over the codes.
#include "common.cuh"
#include "scan.cuh"

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

// Bit window: `hi` holds the current word, `lo` the next one, q0..q3 the four
// after it (each requested four refills before use).  The next 32 bits of the
// stream are funnelshift(lo, hi, bo).  Decodes `cnt` symbols; returns false on
// an unknown code.
struct BitReader {
    const uint32_t *p;
    uint32_t nwords, wi, bo, hi, lo, q0, q1, q2, q3;
    __device__ __forceinline__ uint32_t word(uint32_t i) const { return i < nwords ? __ldg(p + i) : 0u; }
    __device__ __forceinline__ void init(const uint32_t *base, uint32_t nw)
    {
        p = base;
        nwords = nw;
        wi = 0;
        bo = 0;
        hi = word(0);
        lo = word(1);
        q0 = word(2);
        q1 = word(3);
        q2 = word(4);
        q3 = word(5);
    }
    __device__ __forceinline__ uint32_t peek32() const { return __funnelshift_l(lo, hi, bo); }
    // 64 bits from the current position (for codes longer than the table)
    __device__ __forceinline__ unsigned long long peek64() const
    {
        return ((unsigned long long)peek32() << 32) | __funnelshift_l(q0, lo, bo);
    }
    __device__ __forceinline__ void skip(uint32_t len)
    {
        bo += len;
        if (bo >= 32) {
            bo -= 32;
            wi++;
            hi = lo;
            lo = q0;
            q0 = q1;
            q1 = q2;
            q2 = q3;
            q3 = word(wi + 5);
        }
    }
};

struct DecTables {
    const uint32_t *lut;
    const unsigned long long *first;
    const uint32_t *count, *start;
    const uint16_t *sorted;
    uint32_t maxlen;
};

// one symbol; len 0 = unknown code
__device__ __forceinline__ uint32_t decode_one(BitReader &br, const DecTables &t, uint32_t &len)
{
    const uint32_t cur = br.peek32();
    const uint32_t e = t.lut[cur >> (32 - kLutBits)];
    uint32_t sym = e >> 8;
    len = e & 0xFFu;
    if (e == 0) {
        const unsigned long long v = br.peek64();
        for (uint32_t l = kLutBits + 1; l <= t.maxlen; l++) {
            const unsigned long long off = (v >> (64 - l)) - t.first[l];
            if (off < t.count[l]) {
                len = l;
                sym = t.sorted[t.start[l] + off];
                break;
            }
        }
    }
    br.skip(len);
    return sym;
}

template <bool MULTI_TILE>
__global__ void __launch_bounds__(kDecThreads) k_decode(DecodeArgs a, uint32_t sorted_in_smem)
{
    __shared__ uint32_t lut[1 << kLutBits];
    __shared__ unsigned long long first[kMaxLen + 2];
    __shared__ uint32_t count[kMaxLen + 2], start[kMaxLen + 2];
    extern __shared__ uint16_t s_sorted[];
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
    const uint64_t s0 = c * a.chunk;
    const uint32_t cnt = (uint32_t)(a.n - s0 < a.chunk ? a.n - s0 : a.chunk);
    const uint32_t R = a.radius;
    BitReader br;
    br.init(stream + a.chunk_off[c], (nbits + 31) / 32);
    uint32_t zeros = 0, tsum = 0;
    bool bad = false;
    uint16_t *out = a.codes + s0;
    const uint32_t full = cnt & ~7u;
    for (uint32_t k = 0; k < full; k += 8) {
        uint32_t sy[8];
#pragma unroll
        for (int j = 0; j < 8; j++) {
            uint32_t len;
            sy[j] = decode_one(br, t, len);
            bad |= len == 0;
            zeros += sy[j] == 0;
            tsum += sy[j] ? sy[j] - R : 0u;
        }
        *reinterpret_cast<uint4 *>(out + k) = make_uint4(sy[0] | (sy[1] << 16), sy[2] | (sy[3] << 16),
                                                         sy[4] | (sy[5] << 16), sy[6] | (sy[7] << 16));
        if (MULTI_TILE && a.tile_sums && ((s0 + k + 8) & (kRecon1DTile - 1)) == 0) {
            atomicAdd(&a.tile_sums[(s0 + k) / kRecon1DTile], tsum);
            tsum = 0;
        }
        if (bad) break;
    }
    if (!bad) {
        for (uint32_t k = full; k < cnt; k++) {
            uint32_t len;
            const uint32_t sym = decode_one(br, t, len);
            bad |= len == 0;
            zeros += sym == 0;
            tsum += sym ? sym - R : 0u;
            out[k] = (uint16_t)sym;
        }
    }
    if (a.tile_sums && tsum) atomicAdd(&a.tile_sums[(s0 + cnt - 1) / kRecon1DTile], tsum);
    // a valid chunk ends exactly at its recorded bit count
    if (bad || br.wi * 32 + br.bo != nbits) atomicOr(&a.ctl->error, DERR_CORRUPT);
    if (zeros) atomicAdd(&a.ctl->zeros, (unsigned long long)zeros);
}

}  // namespace

int launch_decode(const DecodeArgs &a, cudaStream_t st)
{
    WordsOp op;
    op.bits = reinterpret_cast<const uint32_t *>(a.archive + a.off_bits);
    op.off = a.chunk_off;
    op.words = a.words;
    op.maxbits = (unsigned long long)a.chunk * kMaxLen;
    op.ctl = a.ctl;
    int nl = launch_scan(op, a.nchunk, a.scan_partial, st);
    const uint64_t grid = (a.nchunk + kDecThreads - 1) / kDecThreads;
    const uint32_t nb = 2 * a.radius;
    const uint32_t in_smem = nb <= kSortedSmemMax ? nb : 0u;
    if (a.chunk > kRecon1DTile)
        k_decode<true><<<(unsigned)grid, kDecThreads, in_smem * sizeof(uint16_t), st>>>(a, in_smem);
    else
        k_decode<false><<<(unsigned)grid, kDecThreads, in_smem * sizeof(uint16_t), st>>>(a, in_smem);
    return nl + 1;
}

}  // namespace gbsz
