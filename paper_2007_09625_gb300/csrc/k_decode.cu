// k_decode.cu -- S7: Huffman decode (inflate, Sec. 3.3).
//
// Chunk word offsets are the exclusive prefix sum of ceil(bits/32) over the
// archive's chunk table (one CTA).  Decoding is sequential inside a chunk, as
// in the paper; one thread decodes one chunk through a 64-bit bit window and
// a 4096-entry shared-memory table that resolves every code of at most 12
// bits in one lookup; longer codes fall back to the canonical per-length
// tables.  Decoded codes leave in 16-byte stores.  Every chunk must consume
// exactly its recorded bit count, and every code must exist in the codebook;
// anything else marks the archive corrupt.
#include "common.cuh"

namespace gbsz {

namespace {

constexpr int kOffThreads = 1024;
constexpr int kDecThreads = 64;

__global__ void __launch_bounds__(kOffThreads) k_chunk_offsets(DecodeArgs a)
{
    __shared__ unsigned long long s_scan[33];
    const uint32_t *bits = reinterpret_cast<const uint32_t *>(a.archive + a.off_bits);
    const uint32_t T = blockDim.x, t = threadIdx.x, nc = a.nchunk;
    const uint32_t per = (nc + T - 1) / T;
    const uint32_t lo = min(nc, t * per), hi = min(nc, lo + per);
    const unsigned long long maxbits = (unsigned long long)a.chunk * kMaxLen;
    unsigned long long s = 0;
    bool bad = false;
    for (uint32_t c = lo; c < hi; c++) {
        const uint32_t b = bits[c];
        bad |= b > maxbits;
        s += (b + 31ull) / 32;
    }
    if (bad) atomicOr(&a.ctl->error, DERR_CORRUPT);
    unsigned long long tot;
    unsigned long long run = block_excl_scan64(s, s_scan, &tot);
    for (uint32_t c = lo; c < hi; c++) {
        a.chunk_off[c] = run;
        run += (bits[c] + 31ull) / 32;
    }
    if (t == 0 && tot != a.words) atomicOr(&a.ctl->error, DERR_CORRUPT);
}

__global__ void __launch_bounds__(kDecThreads) k_decode(DecodeArgs a)
{
    __shared__ uint32_t lut[1 << kLutBits];
    __shared__ unsigned long long first[kMaxLen + 2];
    __shared__ uint32_t count[kMaxLen + 2], start[kMaxLen + 2];
    for (uint32_t i = threadIdx.x; i < (1u << kLutBits); i += blockDim.x) lut[i] = a.lut[i];
    for (uint32_t i = threadIdx.x; i < kMaxLen + 2; i += blockDim.x) {
        first[i] = a.first[i];
        count[i] = a.count[i];
        start[i] = a.start[i];
    }
    __syncthreads();
    if (a.ctl->error & DERR_CORRUPT) return;
    const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= a.nchunk) return;
    const uint32_t *stream = reinterpret_cast<const uint32_t *>(a.archive + a.off_stream);
    const uint32_t nbits = reinterpret_cast<const uint32_t *>(a.archive + a.off_bits)[c];
    const uint64_t w0 = a.chunk_off[c];
    const uint64_t nwords = (nbits + 31ull) / 32;
    const uint64_t s0 = c * a.chunk;
    const uint32_t cnt = (uint32_t)(a.n - s0 < a.chunk ? a.n - s0 : a.chunk);
    const uint32_t maxlen = a.maxlen;
    auto word = [&](uint64_t i) -> uint32_t { return i < nwords ? stream[w0 + i] : 0u; };
    uint64_t wi = 0;
    unsigned long long win = ((unsigned long long)word(0) << 32) | word(1);
    uint32_t bo = 0;
    uint32_t buf[4];
    uint32_t zeros = 0;
    bool bad = false;
    uint32_t k = 0;
    for (; k < cnt; k++) {
        const unsigned long long cur = win << bo;
        const uint32_t e = lut[(uint32_t)(cur >> (64 - kLutBits))];
        uint32_t len, sym;
        if (e) {
            len = e & 0xFFu;
            sym = e >> 8;
        } else {
            const unsigned long long v = cur | (bo ? (((unsigned long long)word(wi + 2) << bo) >> 32) : 0ull);
            len = 0;
            sym = 0;
            for (uint32_t l = kLutBits + 1; l <= maxlen; l++) {
                const unsigned long long off = (v >> (64 - l)) - first[l];
                if (off < count[l]) {
                    len = l;
                    sym = a.sorted[start[l] + off];
                    break;
                }
            }
            if (len == 0) {
                bad = true;
                break;
            }
        }
        if (wi * 32 + bo + len > nbits) {
            bad = true;
            break;
        }
        bo += len;
        if (bo >= 32) {
            bo -= 32;
            wi++;
            win = (win << 32) | word(wi + 1);
        }
        zeros += sym == 0;
        const uint32_t slot = k & 7u;
        if (slot & 1u) buf[slot >> 1] |= sym << 16;
        else buf[slot >> 1] = sym;
        if (slot == 7u) *reinterpret_cast<uint4 *>(a.codes + s0 + k - 7) = make_uint4(buf[0], buf[1], buf[2], buf[3]);
    }
    if (!bad) {
        for (uint32_t r = k & ~7u; r < k; r++) {
            const uint32_t slot = r & 7u;
            a.codes[s0 + r] = (uint16_t)((buf[slot >> 1] >> ((slot & 1u) * 16)) & 0xFFFFu);
        }
        if (wi * 32 + bo != nbits) bad = true;
    }
    if (bad) atomicOr(&a.ctl->error, DERR_CORRUPT);
    if (zeros) atomicAdd(&a.ctl->zeros, (unsigned long long)zeros);
}

}  // namespace

void launch_decode(const DecodeArgs &a, cudaStream_t st)
{
    k_chunk_offsets<<<1, kOffThreads, 0, st>>>(a);
    const uint64_t grid = (a.nchunk + kDecThreads - 1) / kDecThreads;
    k_decode<<<(unsigned)grid, kDecThreads, 0, st>>>(a);
}

}  // namespace gbsz
