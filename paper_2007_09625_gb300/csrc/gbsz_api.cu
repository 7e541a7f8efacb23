// gbsz_api.cu -- host side of the C ABI declared in include/gbsz.h:
// contexts with resident device scratch, argument validation, archive header
// parsing, stage orchestration, batches, stage timing.
//
// A context owns "slots": each slot is one complete set of per-call device
// scratch (control block, quant codes, outlier residuals, encoder unit totals,
// codebook and decode tables, carry arrays) plus a stream of its own.  A
// single-field call runs on slot 0 in the caller's stream.  A batch call
// forks the caller's stream into up to kMaxSlots slot streams, gives field i
// to slot i mod K, lets every field run without host synchronisation (the
// fields' kernels overlap on the GPU), joins back into the caller's stream
// and synchronises once.  Results never depend on the slot a field ran on.
#include "../../include/gbsz.h"
#include "common.cuh"
#include "scan.cuh"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

using namespace gbsz;

namespace {

constexpr int kMaxSlots = 8;

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DevGuard()
    {
        int cur;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

// Bumped whenever any scratch buffer of any context is allocated or freed:
// a captured batch graph is replayed only if nothing it points into moved.
std::atomic<uint64_t> g_alloc_gen{1};

struct Buf {
    void *p = nullptr;
    size_t cap = 0;
    bool ensure(size_t bytes)
    {
        if (bytes <= cap && p) return true;
        g_alloc_gen.fetch_add(1);
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
        size_t want = std::max<size_t>(bytes, 256);
        if (cudaMalloc(&p, want) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return false;
        }
        cap = want;
        return true;
    }
    void release()
    {
        if (p) {
            g_alloc_gen.fetch_add(1);
            cudaFree(p);
        }
        p = nullptr;
        cap = 0;
    }
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

// pinned host array, grown on demand
template <typename T> struct HostBuf {
    T *p = nullptr;
    size_t cap = 0;
    bool ensure(size_t count)
    {
        if (count <= cap && p) return true;
        g_alloc_gen.fetch_add(1);
        if (p) cudaFreeHost(p);
        p = nullptr;
        cap = 0;
        if (cudaMallocHost(&p, std::max<size_t>(count, 1) * sizeof(T)) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return false;
        }
        cap = std::max<size_t>(count, 1);
        return true;
    }
    void release()
    {
        if (p) {
            g_alloc_gen.fetch_add(1);
            cudaFreeHost(p);
        }
        p = nullptr;
        cap = 0;
    }
};

// A batch call recorded as a CUDA graph.  The key is every input of the
// call that shapes its launches (pointers, parameters, parsed headers) plus
// the allocation generation; the first call with a key runs eagerly, the
// second is captured, later ones replay the graph (one launch instead of
// about a dozen kernels, copies and memsets per field).
struct StageRec {
    int stage;
    cudaEvent_t a, b;
};

struct BatchGraph {
    std::vector<uint64_t> key;   // key of the captured graph
    std::vector<uint64_t> seen;  // key of the last eager call
    cudaGraphExec_t exec = nullptr;
    uint64_t launches = 0;       // kernels in one replay
    uint64_t captures = 0, replays = 0;
    // stage timing events recorded by the graph's own nodes (captured while
    // profiling); every replay records them again
    std::vector<StageRec> recs;
    void drop()
    {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        key.clear();
    }
};

struct Slot {
    Control *ctl = nullptr;
    // per-field scratch (grown on demand)
    Buf codes, dscr, unit_tot, unit_off, unit_part, unit_exc, lane_bits, chunk_off, faces, scan_part;
    Buf qint, excm;  // Lorenzo order > 1: prequantized integers, exception bits
    Buf zbits;       // 1D order 1 (large fields): code-0 bitmap of the dual-quant kernel
    // fixed-size scratch
    Buf hist, cw64, cw32, codes_only, keyA, keyB, nodef, parent, distA, distB, parA, parB;
    Buf lut, lutf, first, count, start, sorted;
    cudaStream_t stream = nullptr;  // used by batch calls
    cudaEvent_t done = nullptr;
    // the decoder tables are built on a second stream while the chunk offsets are scanned
    cudaStream_t aux = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;

    bool init()
    {
        const size_t B = kMaxBins;
        if (cudaMalloc(&ctl, sizeof(Control)) != cudaSuccess) {
            cudaGetLastError();
            ctl = nullptr;
            return false;
        }
        if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&done, cudaEventDisableTiming) != cudaSuccess ||
            cudaStreamCreateWithFlags(&aux, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return false;
        }
        return hist.ensure(B * 4) && cw64.ensure(B * 8) && cw32.ensure(B * 4) && codes_only.ensure(B * 8) &&
               keyA.ensure(B * 8) && keyB.ensure(B * 8) && nodef.ensure(B * 4) && parent.ensure(2 * B * 4) &&
               distA.ensure(2 * B * 4) && distB.ensure(2 * B * 4) && parA.ensure(2 * B * 4) &&
               parB.ensure(2 * B * 4) && lut.ensure(((1u << kLutBits) + kLut2Words) * 4) && lutf.ensure(kFastLutBytes) && first.ensure((kMaxLen + 2) * 8) &&
               count.ensure((kMaxLen + 2) * 4) && start.ensure((kMaxLen + 2) * 4) && sorted.ensure(B * 2);
    }
    // device bytes held (buffers and the control block)
    uint64_t bytes() const
    {
        uint64_t t = ctl ? sizeof(Control) : 0;
        for (const Buf *b : {&codes, &dscr, &unit_tot, &unit_off, &unit_part, &unit_exc, &lane_bits, &chunk_off, &faces,
                             &scan_part, &qint, &excm, &zbits, &hist, &cw64, &cw32, &codes_only, &keyA, &keyB, &nodef, &parent,
                             &distA, &distB, &parA, &parB, &lut, &lutf, &first, &count, &start, &sorted})
            t += b->cap;
        return t;
    }
    // frees the scratch sized by field (kept: the fixed-size tables)
    void release_field_scratch()
    {
        for (Buf *b : {&codes, &dscr, &unit_tot, &unit_off, &unit_part, &unit_exc, &lane_bits, &chunk_off, &faces,
                       &scan_part, &qint, &excm, &zbits})
            b->release();
    }
    void release()
    {
        for (Buf *b : {&codes, &dscr, &unit_tot, &unit_off, &unit_part, &unit_exc, &lane_bits, &chunk_off, &faces, &scan_part,
                       &qint, &excm, &zbits, &hist, &cw64,
                       &cw32, &codes_only, &keyA, &keyB, &nodef, &parent, &distA, &distB, &parA, &parB, &lut, &lutf,
                       &first, &count, &start, &sorted})
            b->release();
        if (ctl) cudaFree(ctl);
        ctl = nullptr;
        if (stream) cudaStreamDestroy(stream);
        stream = nullptr;
        if (done) cudaEventDestroy(done);
        done = nullptr;
        if (aux) cudaStreamDestroy(aux);
        aux = nullptr;
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        fork = join = nullptr;
    }
};

}  // namespace

// what gbsz_autotune chose for one key: the chunk (part of the archive), and
// two knobs that leave the bytes alone -- the decoder (1 thread, 2 warp per
// chunk) and the rows / planes each dual-quant tile sweeps (0: the rule)
struct Tuned {
    uint32_t chunk, decoder, slab;
};

struct gbsz_ctx {
    int device = 0;
    int num_sms = 152;
    cudaStream_t last_stream = nullptr;
    std::vector<Slot *> slots;       // slot 0 always exists
    HostBuf<Control> ctl_host;       // one control block per field of the last call
    HostBuf<uint8_t> h_header;       // kHeaderBytes per field of the last call
    // the header the last successful single-field compress wrote, copied back
    // inside that call; a decompress of the same buffer and size plans from
    // it and checks it on the device instead of reading it back first
    HostBuf<uint8_t> hdr_last;
    const void *hdr_ptr = nullptr;
    size_t hdr_bytes = 0;
    bool hdr_valid = false;
    cudaEvent_t fork = nullptr;
    // staging of the host-buffer API
    Buf stage_field, stage_archive;
    // the pending asynchronous host decompress: its own slot, staging,
    // control copy and completion event, so that synchronous calls on the
    // context can run while it is in flight
    Slot *aslot = nullptr;
    Buf astage_field, astage_archive;
    HostBuf<Control> actl;
    cudaEvent_t adone = nullptr;
    bool apending = false;
    uint64_t azeros = 0;  // outliers the pending call's archive declares
    // last call (debug copies)
    uint64_t last_n = 0, last_dn = 0;
    uint32_t last_nbins = 0;
    float last_sc[3] = {0, 0, 0};  // error-bound scalars of the last compress
    bool have_compress = false, have_decompress = false;
    bool decoded_codes = false;  // the last decompress left its codes in slot 0's buffer
    // options
    uint32_t cw64_only = 0;  // GBSZ_OPT_CODEWORD_BITS = 64
    uint32_t decoder = 0;    // GBSZ_OPT_DECODER
    uint32_t slab = 0;       // GBSZ_OPT_LORENZO_SLAB
    uint32_t hold_chunk = ~0u;  // GBSZ_OPT_TEST_HOLD_CHUNK (~0u: none)
    // captured batch calls, and captured single-field calls
    BatchGraph gcomp, gdecomp, gsc, gsd, ggcomp, ggdecomp;
    // grouped batch calls: every field's scratch in one arena, the launch
    // plan (items and block tables) built in pinned memory and copied over
    Buf garena, gplan_dev;
    HostBuf<uint8_t> gplan_host;
    uint32_t batch_mode = 0;  // GBSZ_OPT_BATCH_MODE: 0 grouped launches where possible, 1 slot streams
    // autotuned knobs, keyed by (ndim, dims, radius, lorenzo_block, lorenzo_order)
    std::vector<std::pair<std::array<uint64_t, 8>, Tuned>> tuned;
    uint64_t tuned_gen = 0;  // bumped when an entry is added (captured graphs depend on it)
    Buf tune_arc, tune_out;
    // timing
    bool profiling = false;
    std::vector<StageRec> recs;
    std::vector<cudaEvent_t> pool;
    uint64_t launches = 0;
    double prof_ms[GBSZ_NSTAGE] = {};     // stage times collected from graph replays
    uint64_t prof_n[GBSZ_NSTAGE] = {};
    BatchGraph *prof_pending = nullptr;  // replayed graph whose stage events await collection

    cudaEvent_t ev()
    {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }

    bool ensure_slots(int k)
    {
        while ((int)slots.size() < k) {
            Slot *s = new (std::nothrow) Slot();
            if (!s) return false;
            if (!s->init()) {
                s->release();
                delete s;
                return false;
            }
            slots.push_back(s);
        }
        return true;
    }
};

namespace {

bool valid_params(const gbsz_params *p, uint64_t *n_out)
{
    if (!p || p->ndim < 1 || p->ndim > 4) return false;
    uint64_t n = 1;
    for (uint32_t i = 0; i < 4; i++) {
        const uint64_t d = p->dims[i];
        if (d == 0 || d >= (1ull << 32)) return false;
        if (i >= p->ndim && d != 1) return false;
        n *= d;
        if (n >= (1ull << 32)) return false;
    }
    if (!(p->eb > 0.0) || !std::isfinite(p->eb)) return false;
    if (p->eb_mode != GBSZ_EB_ABS && p->eb_mode != GBSZ_EB_REL) return false;
    if (p->radius < 2 || p->radius > 32768) return false;
    if (p->chunk != 0 && (p->chunk < 64 || p->chunk > 65536 || (p->chunk & (p->chunk - 1)))) return false;
    if (p->lorenzo_block > 1 || p->lorenzo_order > 3) return false;
    if (p->lorenzo_block && p->lorenzo_order > 1) return false;
    *n_out = n;
    return true;
}

uint32_t order_of(const gbsz_params &p) { return p.lorenzo_order ? p.lorenzo_order : 1u; }

// The predictor's geometry: a 4D field is predicted as 3D with its two
// slowest extents folded into one.
uint32_t lorenzo_geom(const gbsz_params &p, uint64_t d[3])
{
    d[0] = p.dims[0];
    d[1] = p.dims[1];
    d[2] = p.ndim == 4 ? p.dims[2] * p.dims[3] : p.dims[2];
    return p.ndim == 4 ? 3u : p.ndim;
}

uint32_t auto_chunk(uint64_t n)
{
    // Decoding is sequential inside a chunk, one thread per chunk, and the
    // decoders keep 1024 threads resident per SM: the smallest power of two
    // (64..4096 symbols) whose chunks fit in one such wave on a 152-SM GB300,
    // so no partial second wave trails the first.  Depends on n only, so
    // equal inputs always give equal archives.
    const uint64_t wave = 152ull * 1024ull;
    uint32_t c = 64;
    while (c < 4096 && (uint64_t)c * wave < n) c *= 2;
    return c;
}

gbsz_status map_device_error(uint32_t e)
{
    if (e & DERR_BOUNDS) return GBSZ_ERR_BOUNDS;
    if (e & DERR_INTERNAL) return GBSZ_ERR_CUDA;
    if (e & DERR_TIMEOUT) return GBSZ_ERR_TIMEOUT;
    if (e & (DERR_EB | DERR_RANGE)) return GBSZ_ERR_INVALID_ARG;
    if (e & DERR_CORRUPT) return GBSZ_ERR_CORRUPT;
    if (e & DERR_CAPACITY) return GBSZ_ERR_CAPACITY;
    return GBSZ_OK;
}

// A stage event.  In a stream that is being captured, a plain record would
// only order the captured work; an external record becomes an event-record
// node of the graph, recorded again by every replay.
void record_stage_event(cudaEvent_t e, cudaStream_t st)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
        cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else
        cudaEventRecord(e, st);
}

void stage_begin(gbsz_ctx *c, cudaStream_t st, cudaEvent_t *e)
{
    *e = nullptr;
    if (!c->profiling) return;
    *e = c->ev();
    record_stage_event(*e, st);
}

void stage_end(gbsz_ctx *c, cudaStream_t st, int stage, cudaEvent_t a)
{
    if (!c->profiling || !a) return;
    cudaEvent_t b = c->ev();
    record_stage_event(b, st);
    c->recs.push_back({stage, a, b});
}

CodebookArgs codebook_args(Slot *s)
{
    CodebookArgs a{};
    a.cw64 = s->cw64.as<uint64_t>();
    a.cw32 = s->cw32.as<uint32_t>();
    a.codes_only = s->codes_only.as<uint64_t>();
    a.lut = s->lut.as<uint32_t>();
    a.lutf = s->lutf.p;
    a.first = s->first.as<unsigned long long>();
    a.count = s->count.as<uint32_t>();
    a.start = s->start.as<uint32_t>();
    a.sorted = s->sorted.as<uint16_t>();
    a.keyA = s->keyA.as<unsigned long long>();
    a.keyB = s->keyB.as<unsigned long long>();
    a.nodef = s->nodef.as<uint32_t>();
    a.parent = s->parent.as<uint32_t>();
    a.distA = s->distA.as<uint32_t>();
    a.distB = s->distB.as<uint32_t>();
    a.parA = s->parA.as<uint32_t>();
    a.parB = s->parB.as<uint32_t>();
    a.ctl = s->ctl;
    return a;
}

struct Header {
    gbsz_params p;
    uint64_t n, nchunk, m, e, w, total;
    float eb, ebx2, inv2eb;
    uint32_t maxlen;
    Layout L;
};

template <typename T> T rd(const uint8_t *b, size_t off)
{
    T v;
    std::memcpy(&v, b + off, sizeof(T));
    return v;
}

gbsz_status parse_header(const uint8_t *b, size_t bytes, Header *h)
{
    if (bytes < kHeaderBytes) return GBSZ_ERR_CORRUPT;
    if (rd<uint32_t>(b, H_MAGIC) != kMagic || rd<uint16_t>(b, H_VERSION) != kVersion ||
        rd<uint16_t>(b, H_HDRBYTES) != kHeaderBytes)
        return GBSZ_ERR_CORRUPT;
    gbsz_params p{};
    p.ndim = rd<uint32_t>(b, H_NDIM);
    p.eb_mode = rd<uint32_t>(b, H_EBMODE);
    for (int i = 0; i < 3; i++) p.dims[i] = rd<uint64_t>(b, H_DIMS + 8 * i);
    p.dims[3] = rd<uint32_t>(b, H_DIM3);
    p.lorenzo_order = rd<uint32_t>(b, H_ORDER);
    if (p.lorenzo_order < 1) return GBSZ_ERR_CORRUPT;  // written as 1..3
    p.eb = rd<double>(b, H_EB);
    p.radius = rd<uint32_t>(b, H_RADIUS);
    p.chunk = rd<uint32_t>(b, H_CHUNK);
    p.lorenzo_block = rd<uint32_t>(b, H_LBLOCK);  // validated with the other parameters
    uint64_t n;
    if (!valid_params(&p, &n) || p.chunk == 0) return GBSZ_ERR_CORRUPT;
    if (rd<uint64_t>(b, H_N) != n) return GBSZ_ERR_CORRUPT;
    h->p = p;
    h->n = n;
    h->nchunk = rd<uint32_t>(b, H_NCHUNK);
    if (h->nchunk != (n + p.chunk - 1) / p.chunk) return GBSZ_ERR_CORRUPT;
    h->eb = rd<float>(b, H_EBF);
    h->ebx2 = rd<float>(b, H_EBX2);
    h->inv2eb = rd<float>(b, H_INV2EB);
    if (!(h->eb > 0.0f) || !std::isfinite(h->eb) || !std::isfinite(h->ebx2) || h->ebx2 != h->eb * 2.0f)
        return GBSZ_ERR_CORRUPT;
    h->m = rd<uint64_t>(b, H_M);
    h->e = rd<uint64_t>(b, H_E);
    h->w = rd<uint64_t>(b, H_W);
    h->maxlen = rd<uint32_t>(b, H_MAXLEN);
    h->total = rd<uint64_t>(b, H_TOTAL);
    if (h->m > n || h->e > h->m || h->maxlen < 1 || h->maxlen > kMaxLen) return GBSZ_ERR_CORRUPT;
    if (h->w > h->nchunk + (kMaxLen * n + 31) / 32) return GBSZ_ERR_CORRUPT;
    h->L = make_layout(p.radius, h->nchunk, h->m, h->e, h->w,
                       anchored(p.ndim, p.lorenzo_order, p.lorenzo_block, p.chunk));
    if (h->total != h->L.total || h->total > bytes) return GBSZ_ERR_CORRUPT;
    return GBSZ_OK;
}

// Host-side checks of one compress request; resolves chunk = 0.
gbsz_status check_compress(const float *d_field, const gbsz_params *pin, const void *d_archive, size_t capacity,
                           gbsz_params *p, uint64_t *n, size_t *need)
{
    if (!d_field || !d_archive || !valid_params(pin, n)) return GBSZ_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_archive) & 15) return GBSZ_ERR_INVALID_ARG;
    *p = *pin;
    if (p->chunk == 0) p->chunk = auto_chunk(*n);
    const uint64_t nchunk = (*n + p->chunk - 1) / p->chunk;
    const Layout Lmin =
        make_layout(p->radius, nchunk, 0, 0, 0, anchored(p->ndim, p->lorenzo_order, p->lorenzo_block, p->chunk));
    if (capacity < Lmin.stream) {
        *need = Lmin.stream;
        return GBSZ_ERR_CAPACITY;
    }
    return GBSZ_OK;
}

// bytes a Buf holds after ensure(bytes)
inline uint64_t buf_bytes(uint64_t bytes) { return std::max<uint64_t>(bytes, 256); }

// Single-field compression of a 1D order-1 field of at least this many
// points leaves its outlier and exception records to k_encode_outliers, fed
// by a code-0 bitmap (n/8 bytes) that the count phase writes; smaller fields
// keep the records in pack (one launch fewer).  Measured crossover on a
// random walk with 1.6% outliers: pack stage 0.0163 vs 0.0155 ms at 2^22
// points, 0.0188 vs 0.0204 at 2^23, 0.252 vs 0.339 at 2^28.
constexpr uint64_t kZbitsMin = 1ull << 23;
bool uses_zbits(const gbsz_params &p, uint64_t n)
{
    uint64_t gd[3];
    return n >= kZbitsMin && order_of(p) == 1 && lorenzo_geom(p, gd) == 1;
}
// the bitmap rounded up to whole 128-point lanes (k_encode_outliers reads them whole)
inline uint64_t zbits_bytes(uint64_t n) { return (n + 127) / 128 * 16 + 64; }

// Device bytes of the per-field scratch reserve_compress / reserve_decompress
// allocate in a slot for one field (p resolved: chunk != 0).
uint64_t compress_scratch(const gbsz_params &p, uint64_t n)
{
    const uint64_t nunits = encode_units(n, p.chunk);
    uint64_t t = buf_bytes(n * 2 + 64) + buf_bytes(n * 8 + 64) + buf_bytes(nunits * 16) + buf_bytes((n / 64 + 64) * 4) +
                 buf_bytes(nunits * 16) + buf_bytes(scan_partials(nunits) * 16 + 64) + buf_bytes(nunits * 4);
    if (order_of(p) > 1) t += buf_bytes(n * 4 + 64) + buf_bytes((n / 32 + 1) * 4);
    if (uses_zbits(p, n)) t += buf_bytes(zbits_bytes(n));
    return t;
}

uint64_t decompress_scratch(const gbsz_params &p, uint64_t n)
{
    uint64_t gd[3];
    const uint64_t nchunk = (n + p.chunk - 1) / p.chunk;
    const uint64_t nfaces = recon_faces_entries(lorenzo_geom(p, gd), gd);
    const uint64_t nscan = std::max<uint64_t>(nchunk, nfaces);
    const uint64_t scan_bytes = std::max<uint64_t>({scan_partials(nscan) * 8, order_of(p) > 1 ? scan_partials(n) * 4 : 0,
                                                    scan_partials(n + 1) * 4});
    return buf_bytes(n * 2 + 64) + buf_bytes(n * 8 + 64) + buf_bytes(nchunk * 8 + 8) + buf_bytes(nfaces * 4 + 16) +
           buf_bytes(scan_bytes + 64);
}

// Sizes a slot's scratch for one field (allocates only when it grows).
bool reserve_compress(Slot *s, const gbsz_params &p, uint64_t n)
{
    const uint64_t nunits = encode_units(n, p.chunk);
    if (order_of(p) > 1 && !(s->qint.ensure(n * 4 + 64) && s->excm.ensure((n / 32 + 1) * 4))) return false;
    if (uses_zbits(p, n) && !s->zbits.ensure(zbits_bytes(n))) return false;
    return s->codes.ensure(n * 2 + 64) && s->dscr.ensure(n * 8 + 64) && s->unit_tot.ensure(nunits * 16) &&
           s->lane_bits.ensure((n / 64 + 64) * 4) && s->unit_off.ensure(nunits * 16) &&
           s->unit_part.ensure(scan_partials(nunits) * 16 + 64) && s->unit_exc.ensure(nunits * 4);
}

bool reserve_decompress(Slot *s, const Header &h)
{
    const uint64_t n = h.n;
    uint64_t gd[3];
    const uint64_t nfaces = recon_faces_entries(lorenzo_geom(h.p, gd), gd);
    const uint64_t nscan = std::max<uint64_t>(h.nchunk, nfaces);
    // order > 1 scans the whole 1D field, the warp decoder's fused mode the
    // outlier list (4-byte partials)
    const uint64_t scan_bytes = std::max<uint64_t>({scan_partials(nscan) * 8, order_of(h.p) > 1 ? scan_partials(n) * 4 : 0,
                                                    scan_partials(h.m + 1) * 4});
    return s->codes.ensure(n * 2 + 64) && s->dscr.ensure(n * 8 + 64) && s->chunk_off.ensure(h.nchunk * 8 + 8) &&
           s->faces.ensure(nfaces * 4 + 16) && s->scan_part.ensure(scan_bytes + 64);
}

// the autotuner's key of a field: (ndim, dims, radius, lorenzo_block, lorenzo_order)
std::array<uint64_t, 8> tune_key(const gbsz_params &p)
{
    return {p.ndim, p.dims[0], p.dims[1], p.dims[2], p.dims[3], p.radius, p.lorenzo_block, order_of(p)};
}

const Tuned *find_tuned(const gbsz_ctx *c, const gbsz_params &p)
{
    if (c->tuned.empty()) return nullptr;
    const std::array<uint64_t, 8> k = tune_key(p);
    for (const auto &t : c->tuned)
        if (t.first == k) return &t.second;
    return nullptr;
}

// rows (2D) or planes (3D) each dual-quant tile sweeps: the option, else the
// tuned choice for this field's key, else 0 (the kernels' rule)
uint32_t slab_for(const gbsz_ctx *c, const gbsz_params &p)
{
    if (c->slab) return c->slab;
    const Tuned *t = find_tuned(c, p);
    return t ? t->slab : 0u;
}

// Enqueues S0-S6 of one field on stream st using slot s; no synchronisation.
gbsz_status enqueue_compress(gbsz_ctx *c, Slot *s, const float *d_field, const gbsz_params &p, uint64_t n,
                             void *d_archive, size_t capacity, cudaStream_t st)
{
    const uint32_t nbins = 2 * p.radius;
    const uint64_t nunits = encode_units(n, p.chunk);
    const uint32_t order = order_of(p);
    if (!reserve_compress(s, p, n)) return GBSZ_ERR_OOM;
    cudaMemsetAsync(s->ctl, 0, sizeof(Control), st);
    cudaMemsetAsync(s->hist.p, 0, nbins * 4, st);
    cudaMemsetAsync(s->unit_exc.p, 0, nunits * 4, st);
    if (order > 1) cudaMemsetAsync(s->excm.p, 0, (n / 32 + 1) * 4, st);

    cudaEvent_t e0;
    stage_begin(c, st, &e0);
    launch_minmax_eb(d_field, n, s->ctl, p.eb, p.eb_mode, c->num_sms, st);
    stage_end(c, st, 0, e0);

    QuantArgs q{};
    q.x = d_field;
    q.ndim = lorenzo_geom(p, q.dims);
    q.radius = p.radius;
    q.codes = s->codes.as<uint16_t>();
    q.dscr = s->dscr.as<int2>();
    q.hist = s->hist.as<uint32_t>();
    q.unit_exc = s->unit_exc.as<uint32_t>();
    q.unit_shift = encode_unit_shift(p.chunk);
    q.lblock = p.lorenzo_block;
    q.order = order;
    q.qint = order > 1 ? s->qint.as<int32_t>() : nullptr;
    q.excm = order > 1 ? s->excm.as<uint32_t>() : nullptr;
    q.ctl = s->ctl;
    q.num_sms = c->num_sms;
    q.slab = slab_for(c, p);
    q.chunk = p.chunk;
    if (anchored(p.ndim, order, p.lorenzo_block, p.chunk))  // capacity checked by check_compress
        q.anchors = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(d_archive) +
                                                 make_layout(p.radius, (n + p.chunk - 1) / p.chunk, 0, 0, 0, true).anch);
    stage_begin(c, st, &e0);
    const int nq = launch_dualquant(q, st);
    stage_end(c, st, 1, e0);

    CodebookArgs cb = codebook_args(s);
    cb.hist = s->hist.as<uint32_t>();
    cb.nbins = nbins;
    cb.len_out = static_cast<uint8_t *>(d_archive) + kHeaderBytes;
    stage_begin(c, st, &e0);
    launch_codebook(cb, st);
    stage_end(c, st, 2, e0);

    EncodeArgs en{};
    en.codes = q.codes;
    en.x = d_field;
    en.dscr = q.dscr;
    en.zbits = uses_zbits(p, n) ? s->zbits.as<uint32_t>() : nullptr;
    en.n = n;
    en.chunk = p.chunk;
    en.radius = p.radius;
    en.nbins = nbins;
    en.cw64 = cb.cw64;
    en.cw32 = cb.cw32;
    en.archive = static_cast<uint8_t *>(d_archive);
    en.capacity = capacity;
    en.lane_bits = s->lane_bits.as<uint32_t>();
    en.unit_exc = s->unit_exc.as<uint32_t>();
    en.unit_tot = s->unit_tot.as<ulonglong2>();
    en.unit_off = s->unit_off.as<ulonglong2>();
    en.scan_part = s->unit_part.as<ulonglong2>();
    en.ctl = s->ctl;
    en.ndim = p.ndim;
    en.eb_mode = p.eb_mode;
    en.lblock = p.lorenzo_block;
    en.order = order;
    en.cw64_only = c->cw64_only;
    for (int i = 0; i < 4; i++) en.dims[i] = p.dims[i];
    en.eb = p.eb;
    en.num_sms = c->num_sms;
    int nenc = 0;
    for (int ph = 0; ph < 3; ph++) {
        stage_begin(c, st, &e0);
        nenc += launch_encode(en, st, ph);
        stage_end(c, st, 3 + ph, e0);
    }
    c->launches += 2 + nq + nenc;
    return GBSZ_OK;
}

// Which decoder a field takes: the thread-per-chunk decoders, the
// warp-per-chunk decoder writing codes, or the warp-per-chunk decoder with
// the 1D reconstruction fused in.  By default the warp decoder takes fields
// of at most 32 chunks per SM in chunks of at least 1024 symbols: there a
// thread-per-chunk decoder leaves most of the GPU idle while each thread
// walks its long chunk.  With more chunks, or short ones, the thread
// decoders finish first (fewer instructions per symbol, and no
// re-synchronisation or look-back per chunk).
// ThreadValues: an anchored 1D archive whose codes fit the complete table is
// reconstructed inside the thread-per-chunk decoder itself (each chunk from
// its anchor), so the codes never reach HBM and no separate value pass runs.
enum class WarpUse { Thread, Codes, Fused, ThreadValues };

WarpUse warp_use(const gbsz_ctx *c, const Header &h, uint32_t gnd, uint32_t order)
{
    uint32_t dec = c->decoder;
    if (dec == 0) {  // the tuned choice for this key, when it was measured at this chunk
        const Tuned *t = find_tuned(c, h.p);
        if (t && t->chunk == h.p.chunk) dec = t->decoder;
    }
    const WarpUse thread = dec != 3 && h.L.nanch && fast_lut_bits(h.maxlen, 2 * h.p.radius) != 0
                               ? WarpUse::ThreadValues
                               : WarpUse::Thread;
    if (dec == 1 || dec == 3 || h.p.chunk > kWarpMaxChunk) return thread;
    if (dec == 0 && (h.nchunk > 32ull * (uint64_t)c->num_sms || h.p.chunk < 1024)) return thread;
    // 1D order-1 fields get their tile sums from the thread decoder, or are
    // reconstructed inside the warp decoder
    const bool line = gnd == 1 && !h.p.lorenzo_block && order == 1;
    if (line) return h.n < (1ull << 30) ? WarpUse::Fused : thread;
    return WarpUse::Codes;
}

// Enqueues S7-S8 of one parsed archive on stream st using slot s.
// expect: the header h was parsed from, when it was not read from d_archive
// in this call (checked on the device first; a mismatch sets DERR_STALE)
gbsz_status enqueue_decompress(gbsz_ctx *c, Slot *s, const Header &h, const void *d_archive, float *d_field,
                               cudaStream_t st, const uint8_t *expect = nullptr)
{
    const uint64_t n = h.n;
    uint64_t gd[3];
    const uint32_t gnd = lorenzo_geom(h.p, gd);
    const uint32_t order = order_of(h.p);
    const uint64_t nfaces = recon_faces_entries(gnd, gd);
    const WarpUse wu = warp_use(c, h, gnd, order);
    const bool own_values = wu == WarpUse::Fused || wu == WarpUse::ThreadValues;  // S8 inside the decoder
    if (s == c->slots[0]) c->decoded_codes = !own_values;
    const bool tile_sums = gnd == 1 && !h.p.lorenzo_block && order == 1 && !own_values;
    if (!reserve_decompress(s, h)) return GBSZ_ERR_OOM;
    cudaMemsetAsync(s->ctl, 0, sizeof(Control), st);
    if (expect) {
        launch_header_check(d_archive, expect, s->ctl, st);
        c->launches++;
    }
    if (tile_sums) cudaMemsetAsync(s->faces.p, 0, nfaces * 4, st);
    // fused: the look-back words in the (unused) code buffer
    if (wu == WarpUse::Fused) cudaMemsetAsync(s->codes.p, 0, h.nchunk * 8, st);
    const uint8_t *arc = static_cast<const uint8_t *>(d_archive);

    CodebookArgs cb = codebook_args(s);
    cb.len_in = arc + kHeaderBytes;
    cb.nbins = 2 * h.p.radius;
    cb.expect_maxlen = h.maxlen;
    cb.fast_bits = fast_lut_bits(h.maxlen, cb.nbins);
    cb.fast_pair = 0;  // the decoder builds its own first level from the complete table
    // decoder tables (one CTA) on the slot's second stream, beside the
    // chunk-offset scan below; joined before the symbols are decoded
    cudaEvent_t e0;
    cudaEventRecord(s->fork, st);
    cudaStreamWaitEvent(s->aux, s->fork, 0);
    stage_begin(c, s->aux, &e0);
    launch_decode_tables(cb, s->aux);
    stage_end(c, s->aux, 6, e0);
    cudaEventRecord(s->join, s->aux);

    DecodeArgs d{};
    d.archive = arc;
    d.n = n;
    d.chunk = h.p.chunk;
    d.nchunk = (uint32_t)h.nchunk;
    d.radius = h.p.radius;
    d.maxlen = h.maxlen;
    d.words = h.w;
    d.off_bits = h.L.bits;
    d.off_stream = h.L.stream;
    d.lut = cb.lut;
    d.first = cb.first;
    d.count = cb.count;
    d.start = cb.start;
    d.sorted = cb.sorted;
    d.lutf = cb.lutf;
    d.fast_bits = cb.fast_bits;
    d.fast_pair = cb.fast_pair;
    d.num_sms = c->num_sms;
    d.chunk_off = s->chunk_off.as<unsigned long long>();
    d.scan_partial = s->scan_part.as<unsigned long long>();
    d.tile_sums = tile_sums ? s->faces.as<uint32_t>() : nullptr;
    d.codes = s->codes.as<uint16_t>();
    d.ctl = s->ctl;
    if (wu == WarpUse::ThreadValues) {
        d.out = d_field;
        d.ebx2 = h.ebx2;
        d.anchors = reinterpret_cast<const uint32_t *>(arc + h.L.anch);
        d.outl = reinterpret_cast<const uint2 *>(arc + h.L.outl);
        d.ostart = s->dscr.as<uint32_t>();  // the residual buffer is not otherwise used here
        d.m = h.m;
    }
    int ndec = 0;
    stage_begin(c, st, &e0);
    ndec += launch_decode(d, st, 0);
    if (wu == WarpUse::Fused)
        ndec += launch_outlier_prefix(reinterpret_cast<const uint2 *>(arc + h.L.outl), h.m, s->dscr.as<uint32_t>(),
                                      s->scan_part.as<uint32_t>(), s->ctl, st);
    if (wu == WarpUse::ThreadValues)
        ndec += launch_outlier_chunk_starts(d.outl, h.m, n, h.p.chunk, d.nchunk, s->dscr.as<uint32_t>(), s->ctl, st);
    stage_end(c, st, 7, e0);
    cudaStreamWaitEvent(st, s->join, 0);
    stage_begin(c, st, &e0);
    if (wu == WarpUse::Thread) {
        ndec += launch_decode(d, st, 1);
    } else if (wu == WarpUse::ThreadValues) {
        ndec += launch_decode(d, st, 2);
    } else {
        WarpDecodeArgs w{};
        w.d = d;
        w.outl = reinterpret_cast<const uint2 *>(arc + h.L.outl);
        w.odp = s->dscr.as<uint32_t>();
        w.m = h.m;
        w.ebx2 = h.ebx2;
        w.out = d_field;
        w.look = s->codes.as<unsigned long long>();
        w.hold_chunk = c->hold_chunk;
        if (h.L.nanch) w.anchors = reinterpret_cast<const uint32_t *>(arc + h.L.anch);
        ndec += launch_decode_warp(w, wu == WarpUse::Fused, st);
    }
    stage_end(c, st, 8, e0);
    if (own_values) {  // S8 ran inside the decoder; only the verbatim exceptions remain
        ReconArgs r{};
        r.archive = arc;
        r.off_exc = h.L.exc;
        r.e = h.e;
        r.ndim = 1;
        r.dims[0] = n;
        r.dims[1] = r.dims[2] = 1;
        r.out = d_field;
        r.ctl = s->ctl;
        r.num_sms = c->num_sms;
        stage_begin(c, st, &e0);
        const int nl = launch_exceptions(r, st);
        stage_end(c, st, 9, e0);
        c->launches += 1 + ndec + nl;
        return GBSZ_OK;
    }

    ReconArgs r{};
    r.codes = d.codes;
    r.archive = arc;
    r.off_outl = h.L.outl;
    r.off_exc = h.L.exc;
    r.m = h.m;
    r.e = h.e;
    r.ndim = gnd;
    for (int i = 0; i < 3; i++) r.dims[i] = gd[i];
    r.radius = h.p.radius;
    r.ebx2 = h.ebx2;
    r.dscr = s->dscr.as<int32_t>();
    r.lblock = h.p.lorenzo_block;
    r.order = order;
    r.faces = s->faces.as<uint32_t>();
    r.faces_cap = nfaces;
    r.scan_partial = s->scan_part.as<uint32_t>();
    r.out = d_field;
    r.ctl = s->ctl;
    r.num_sms = c->num_sms;
    if (h.L.nanch) {
        r.anchors = reinterpret_cast<const uint32_t *>(arc + h.L.anch);
        r.chunk = h.p.chunk;
    }
    int nl = 0;
    stage_begin(c, st, &e0);
    launch_reconstruct(r, st, &nl);
    stage_end(c, st, 9, e0);
    c->launches += 1 + ndec + nl;
    return GBSZ_OK;
}

gbsz_status decompress_status(const Control &ctl, const Header &h)
{
    if (ctl.error) return map_device_error(ctl.error);
    if (ctl.zeros != h.m) return GBSZ_ERR_CORRUPT;
    return GBSZ_OK;
}

}  // namespace

namespace {

// Runs `enqueue` (which forks the caller's stream st to the slot streams and
// joins them back) either eagerly, or through the context's graph for this
// kind of batch: replayed if `key` matches the captured one, captured if it
// matches the previous eager call's.  While profiling, the stage events are
// captured as event-record nodes of the graph; the caller collects their
// times (prof_collect) after it has synchronized with the replay.
template <typename F>
gbsz_status run_batch(gbsz_ctx *c, BatchGraph &bg, std::vector<uint64_t> &key, cudaStream_t st, F enqueue)
{
    key.push_back(c->profiling ? 1u : 0u);
    key.push_back(c->decoder);
    key.push_back(c->slab);
    key.push_back(c->hold_chunk);
    key.push_back(c->tuned_gen);
    key.push_back(g_alloc_gen.load());  // last: checked again after a capture
    if (bg.exec && key == bg.key) {
        c->launches += bg.launches;
        bg.replays++;
        if (!bg.recs.empty()) c->prof_pending = &bg;
        return cudaGraphLaunch(bg.exec, st) == cudaSuccess ? GBSZ_OK : GBSZ_ERR_CUDA;
    }
    if (key == bg.seen) {
        bg.drop();
        for (auto &r : bg.recs) {  // the old graph's events
            c->pool.push_back(r.a);
            c->pool.push_back(r.b);
        }
        bg.recs.clear();
        const uint64_t l0 = c->launches;
        const size_t r0 = c->recs.size();
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            const gbsz_status es = enqueue();
            const cudaError_t ce = cudaStreamEndCapture(st, &graph);
            if (es == GBSZ_OK && ce == cudaSuccess && graph &&
                cudaGraphInstantiate(&bg.exec, graph, 0) == cudaSuccess && key.back() == g_alloc_gen.load()) {
                cudaGraphDestroy(graph);
                bg.key = key;
                bg.launches = c->launches - l0;
                bg.captures++;
                bg.recs.assign(c->recs.begin() + r0, c->recs.end());  // now the graph's
                c->recs.resize(r0);
                if (!bg.recs.empty()) c->prof_pending = &bg;
                return cudaGraphLaunch(bg.exec, st) == cudaSuccess ? GBSZ_OK : GBSZ_ERR_CUDA;
            }
            if (graph) cudaGraphDestroy(graph);
            bg.drop();
        }
        cudaGetLastError();  // a failed capture leaves nothing behind; run eagerly
        c->launches = l0;
        for (size_t i = r0; i < c->recs.size(); i++) {  // events of the failed capture
            c->pool.push_back(c->recs[i].a);
            c->pool.push_back(c->recs[i].b);
        }
        c->recs.resize(r0);
    }
    const gbsz_status es = enqueue();
    bg.seen = key;
    return es;
}

// After the caller has synchronized with a replayed graph: its stage times.
void prof_collect(gbsz_ctx *c)
{
    BatchGraph *bg = c->prof_pending;
    c->prof_pending = nullptr;
    if (!bg) return;
    for (const auto &r : bg->recs) {
        float t = 0;
        if (r.stage >= 0 && r.stage < GBSZ_NSTAGE && cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess) {
            c->prof_ms[r.stage] += t;
            c->prof_n[r.stage]++;
        }
    }
    cudaGetLastError();
}

inline void key_add(std::vector<uint64_t> &k, const void *p, size_t bytes)
{
    const uint8_t *b = static_cast<const uint8_t *>(p);
    for (size_t i = 0; i < bytes; i += 8) {
        uint64_t v = 0;
        std::memcpy(&v, b + i, std::min<size_t>(8, bytes - i));
        k.push_back(v);
    }
}

}  // namespace

namespace {

// ---------------------------------------------------------------------------
// Grouped batch compress: every stage of every field in one launch per
// kernel (variant), each field owning a range of the grid's blocks.

struct ZeroRange {
    void *p;
    uint64_t bytes;  // a multiple of 4; p 16-byte aligned
};

// zeroes every range (blocks stride over the ranges)
__global__ void __launch_bounds__(256) k_zero_group(const ZeroRange *r, uint32_t nr)
{
    for (uint32_t i = blockIdx.x; i < nr; i += gridDim.x) {
        uint32_t *p = static_cast<uint32_t *>(r[i].p);
        const uint64_t words = r[i].bytes / 4;
        for (uint64_t w = threadIdx.x; w < words; w += blockDim.x) p[w] = 0;
    }
}

// the fields' control blocks side by side, for one copy to the host
__global__ void k_gather_ctl(Control *const *ctl, uint32_t count, Control *dst)
{
    const uint32_t words = sizeof(Control) / 4;
    for (uint32_t i = blockIdx.x; i < count; i += gridDim.x)
        for (uint32_t w = threadIdx.x; w < words; w += blockDim.x)
            reinterpret_cast<uint32_t *>(dst + i)[w] = reinterpret_cast<const uint32_t *>(ctl[i])[w];
}

inline uint64_t up256(uint64_t v) { return (v + 255) & ~uint64_t(255); }

// One field's scratch in the arena (all 256-byte aligned); base = nullptr
// only sizes it.  Sizes follow the slot buffers, with the codebook scratch
// sized for the field's 2R symbols.
struct FieldScratch {
    Control *ctl;
    uint32_t *hist, *cw32, *nodef, *parent, *distA, *distB, *parA, *parB, *lane_bits, *unit_exc;
    uint64_t *cw64, *codes_only;
    unsigned long long *keyA, *keyB;
    uint16_t *codes;
    int2 *dscr;
    ulonglong2 *unit_tot, *unit_off, *unit_part;
};

uint64_t layout_field(uint8_t *base, const gbsz_params &p, uint64_t n, FieldScratch *f)
{
    const uint64_t nb = 2ull * p.radius, nunits = encode_units(n, p.chunk);
    uint64_t off = 0;
    auto take = [&](uint64_t bytes) -> void * {
        void *q = base ? base + off : nullptr;
        off += up256(bytes);
        return q;
    };
    f->ctl = static_cast<Control *>(take(sizeof(Control)));
    f->hist = static_cast<uint32_t *>(take(nb * 4));
    f->cw64 = static_cast<uint64_t *>(take(nb * 8));
    f->cw32 = static_cast<uint32_t *>(take(nb * 4));
    f->codes_only = static_cast<uint64_t *>(take(nb * 8));
    f->keyA = static_cast<unsigned long long *>(take(nb * 8));
    f->keyB = static_cast<unsigned long long *>(take(nb * 8));
    f->nodef = static_cast<uint32_t *>(take(nb * 4));
    f->parent = static_cast<uint32_t *>(take(2 * nb * 4));
    f->distA = static_cast<uint32_t *>(take(2 * nb * 4));
    f->distB = static_cast<uint32_t *>(take(2 * nb * 4));
    f->parA = static_cast<uint32_t *>(take(2 * nb * 4));
    f->parB = static_cast<uint32_t *>(take(2 * nb * 4));
    f->codes = static_cast<uint16_t *>(take(n * 2 + 64));
    f->dscr = static_cast<int2 *>(take(n * 8 + 64));
    f->unit_tot = static_cast<ulonglong2 *>(take(nunits * 16));
    f->lane_bits = static_cast<uint32_t *>(take((n / 64 + 64) * 4));
    f->unit_off = static_cast<ulonglong2 *>(take(nunits * 16));
    f->unit_part = static_cast<ulonglong2 *>(take(scan_partials(nunits) * 16 + 64));
    f->unit_exc = static_cast<uint32_t *>(take(nunits * 4));
    return off;
}

// host-side plan: arrays appended to one pinned buffer, 16-byte aligned
struct PlanBuilder {
    std::vector<uint8_t> buf;
    template <typename T> uint64_t put(const T *v, size_t count)
    {
        const uint64_t off = (buf.size() + 15) & ~uint64_t(15);
        buf.resize(off + sizeof(T) * count);
        if (count) std::memcpy(buf.data() + off, v, sizeof(T) * count);
        return off;
    }
};

// first[] of a grouped launch from every item's blocks
std::vector<uint32_t> firsts(const std::vector<uint32_t> &blocks)
{
    std::vector<uint32_t> f(blocks.size() + 1, 0);
    for (size_t i = 0; i < blocks.size(); i++) f[i + 1] = f[i] + blocks[i];
    return f;
}

// A batch that the grouped path takes: every field valid, order 1, and
// small on average -- launch latency dominates small fields, while the
// fields' own launches on the slot streams let one field's single-CTA
// codebook overlap another's memory-bound kernels (measured: 16 fields of
// 1800x3600, 0.80 ms on the slot streams against 0.86 ms grouped; 256 fields
// of 64 Ki points, 3.2 ms against 1.0 ms).
constexpr uint64_t kGroupedMeanPoints = 1ull << 21;

bool groupable(uint32_t count, const gbsz_params *rp, const uint64_t *rn, const gbsz_status *statuses)
{
    if (count < 2) return false;
    uint64_t total = 0;
    for (uint32_t i = 0; i < count; i++) {
        if (statuses[i] != GBSZ_OK || order_of(rp[i]) != 1) return false;
        total += rn[i];
    }
    return total <= kGroupedMeanPoints * count;
}

gbsz_status compress_batch_grouped(gbsz_ctx *c, uint32_t count, const float *const *d_fields,
                                   const gbsz_params *rp, const uint64_t *rn, void *const *d_archives,
                                   const size_t *capacities, std::vector<uint64_t> &key, cudaStream_t st)
{
    // arena
    std::vector<uint64_t> foff(count + 1, 0);
    FieldScratch tmp;
    for (uint32_t i = 0; i < count; i++) foff[i + 1] = foff[i] + layout_field(nullptr, rp[i], rn[i], &tmp);
    if (!c->garena.ensure(foff[count])) return GBSZ_ERR_OOM;
    uint8_t *arena = c->garena.as<uint8_t>();
    std::vector<FieldScratch> fs(count);
    for (uint32_t i = 0; i < count; i++) layout_field(arena + foff[i], rp[i], rn[i], &fs[i]);

    // items of every stage
    std::vector<MinmaxItem> mm(count);
    std::vector<uint32_t> mm_b(count), cb_unused;
    std::vector<QuantItem> qi(count);
    std::vector<int> qvar(count);
    std::vector<uint32_t> q_b(count);
    size_t q_smem = 0, enc_smem[2] = {0, 0};
    std::vector<CodebookArgs> cb(count);
    std::vector<EncodeItem> en(count);
    std::vector<uint32_t> cnt_b(count), pack_b(count), scan_b;
    std::vector<ScanItem<UnitScan>> sc;
    std::vector<ZeroRange> zr;
    std::vector<Control *> ctls(count);
    bool vec = true;
    for (uint32_t i = 0; i < count; i++) {
        const gbsz_params &p = rp[i];
        const uint64_t n = rn[i];
        const FieldScratch &f = fs[i];
        const uint32_t nbins = 2 * p.radius;
        const uint64_t nunits = encode_units(n, p.chunk);
        zr.push_back({f.ctl, sizeof(Control)});
        zr.push_back({f.hist, (uint64_t)nbins * 4});
        zr.push_back({f.unit_exc, nunits * 4});
        ctls[i] = f.ctl;
        vec &= (reinterpret_cast<uintptr_t>(d_fields[i]) & 15) == 0;
        mm[i] = MinmaxItem{d_fields[i], n, f.ctl, p.eb, p.eb_mode};
        mm_b[i] = minmax_blocks(n, p.eb_mode, c->num_sms);
        QuantArgs &q = qi[i].a;
        q = QuantArgs{};
        q.x = d_fields[i];
        q.ndim = lorenzo_geom(p, q.dims);
        q.radius = p.radius;
        q.codes = f.codes;
        q.dscr = f.dscr;
        q.hist = f.hist;
        q.unit_exc = f.unit_exc;
        q.unit_shift = encode_unit_shift(p.chunk);
        q.lblock = p.lorenzo_block;
        q.order = 1;
        q.ctl = f.ctl;
        q.num_sms = c->num_sms;
        q.slab = slab_for(c, p);
        q.chunk = p.chunk;
        if (anchored(p.ndim, 1, p.lorenzo_block, p.chunk))  // capacities checked per field beforehand
            q.anchors = reinterpret_cast<uint32_t *>(
                static_cast<uint8_t *>(d_archives[i]) + make_layout(p.radius, (n + p.chunk - 1) / p.chunk, 0, 0, 0, true).anch);
        size_t sm = 0;
        q_b[i] = dualquant_plan(q, qi[i].t, &qvar[i], &sm);
        q_smem = std::max(q_smem, sm);
        CodebookArgs &k = cb[i];
        k = CodebookArgs{};
        k.hist = f.hist;
        k.nbins = nbins;
        k.len_out = static_cast<uint8_t *>(d_archives[i]) + kHeaderBytes;
        k.cw64 = f.cw64;
        k.cw32 = f.cw32;
        k.codes_only = f.codes_only;
        k.keyA = f.keyA;
        k.keyB = f.keyB;
        k.nodef = f.nodef;
        k.parent = f.parent;
        k.distA = f.distA;
        k.distB = f.distB;
        k.parA = f.parA;
        k.parB = f.parB;
        k.ctl = f.ctl;
        EncodeArgs e{};
        e.codes = f.codes;
        e.x = d_fields[i];
        e.dscr = f.dscr;
        e.n = n;
        e.chunk = p.chunk;
        e.radius = p.radius;
        e.nbins = nbins;
        e.cw64 = f.cw64;
        e.cw32 = f.cw32;
        e.archive = static_cast<uint8_t *>(d_archives[i]);
        e.capacity = capacities[i];
        e.lane_bits = f.lane_bits;
        e.unit_exc = f.unit_exc;
        e.unit_tot = f.unit_tot;
        e.unit_off = f.unit_off;
        e.scan_part = f.unit_part;
        e.ctl = f.ctl;
        e.ndim = p.ndim;
        e.eb_mode = p.eb_mode;
        e.lblock = p.lorenzo_block;
        e.order = 1;
        e.cw64_only = c->cw64_only;
        for (int d = 0; d < 4; d++) e.dims[d] = p.dims[d];
        e.eb = p.eb;
        e.num_sms = c->num_sms;
        uint32_t bl[2];
        size_t sm2[2];
        uint64_t units;
        encode_plan(e, &en[i], bl, sm2, &units);
        cnt_b[i] = bl[0];
        pack_b[i] = bl[1];
        enc_smem[0] = std::max(enc_smem[0], sm2[0]);
        enc_smem[1] = std::max(enc_smem[1], sm2[1]);
        sc.push_back(ScanItem<UnitScan>{UnitScan{f.unit_tot, f.unit_off}, units, f.unit_part});
        scan_b.push_back((uint32_t)scan_blocks(units));
    }
    // dual-quant items ordered by kernel variant, one launch per variant
    std::vector<uint32_t> order(count);
    for (uint32_t i = 0; i < count; i++) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t b) { return qvar[a] < qvar[b]; });
    PlanBuilder pb;
    const uint64_t o_mm = pb.put(mm.data(), count);
    const std::vector<uint32_t> mmf = firsts(mm_b);
    const uint64_t o_mmf = pb.put(mmf.data(), mmf.size());
    struct QGroup {
        int variant;
        uint32_t ni, blocks;
        uint64_t o_items, o_first;
    };
    std::vector<QGroup> qg;
    for (uint32_t a = 0; a < count;) {
        uint32_t b = a;
        std::vector<QuantItem> items;
        std::vector<uint32_t> bl;
        while (b < count && qvar[order[b]] == qvar[order[a]]) {
            items.push_back(qi[order[b]]);
            bl.push_back(q_b[order[b]]);
            b++;
        }
        const std::vector<uint32_t> f = firsts(bl);
        QGroup g{qvar[order[a]], (uint32_t)items.size(), f.back(), 0, 0};
        g.o_items = pb.put(items.data(), items.size());
        g.o_first = pb.put(f.data(), f.size());
        qg.push_back(g);
        a = b;
    }
    const uint64_t o_cb = pb.put(cb.data(), count);
    const uint64_t o_en = pb.put(en.data(), count);
    const std::vector<uint32_t> cf = firsts(cnt_b), pf = firsts(pack_b), sf = firsts(scan_b);
    const uint64_t o_cf = pb.put(cf.data(), cf.size());
    const uint64_t o_pf = pb.put(pf.data(), pf.size());
    const uint64_t o_sc = pb.put(sc.data(), sc.size());
    const uint64_t o_sf = pb.put(sf.data(), sf.size());
    const uint64_t o_zr = pb.put(zr.data(), zr.size());
    const uint64_t o_ctl = pb.put(ctls.data(), ctls.size());
    const uint64_t o_cdst = pb.put<uint8_t>(nullptr, 0);
    pb.buf.resize(o_cdst + (uint64_t)count * sizeof(Control));  // the gathered control blocks (device side)
    const uint64_t plan_bytes = pb.buf.size();
    if (!c->gplan_host.ensure(plan_bytes) || !c->gplan_dev.ensure(plan_bytes)) return GBSZ_ERR_OOM;
    std::memcpy(c->gplan_host.p, pb.buf.data(), plan_bytes);
    uint8_t *dp = c->gplan_dev.as<uint8_t>();
    key.push_back(0x6Eu);  // grouped
    key.push_back((uint64_t)(uintptr_t)c->gplan_host.p);
    key.push_back((uint64_t)(uintptr_t)dp);
    key.push_back((uint64_t)(uintptr_t)arena);

    auto enqueue = [&]() -> gbsz_status {
        int nl = 0;
        cudaEvent_t e0;
        cudaMemcpyAsync(dp, c->gplan_host.p, plan_bytes, cudaMemcpyHostToDevice, st);
        k_zero_group<<<(unsigned)std::min<size_t>(zr.size(), (size_t)c->num_sms * 8), 256, 0, st>>>(
            reinterpret_cast<const ZeroRange *>(dp + o_zr), (uint32_t)zr.size());
        stage_begin(c, st, &e0);
        launch_minmax_group(reinterpret_cast<const MinmaxItem *>(dp + o_mm), reinterpret_cast<const uint32_t *>(dp + o_mmf),
                            count, mmf.back(), vec, st);
        stage_end(c, st, 0, e0);
        stage_begin(c, st, &e0);
        for (const QGroup &g : qg) {
            launch_dualquant_group(g.variant, reinterpret_cast<const QuantItem *>(dp + g.o_items),
                                   reinterpret_cast<const uint32_t *>(dp + g.o_first), g.ni, g.blocks, q_smem, st);
            nl++;
        }
        stage_end(c, st, 1, e0);
        stage_begin(c, st, &e0);
        launch_codebook_group(reinterpret_cast<const CodebookArgs *>(dp + o_cb), count, st);
        stage_end(c, st, 2, e0);
        const EncodeItem *ei = reinterpret_cast<const EncodeItem *>(dp + o_en);
        stage_begin(c, st, &e0);
        launch_encode_group(0, ei, reinterpret_cast<const uint32_t *>(dp + o_cf), count, cf.back(), enc_smem[0], st);
        stage_end(c, st, 3, e0);
        stage_begin(c, st, &e0);
        nl += launch_unit_scan_group(reinterpret_cast<const ScanItem<UnitScan> *>(dp + o_sc),
                                     reinterpret_cast<const uint32_t *>(dp + o_sf), count, sf.back(), st);
        stage_end(c, st, 4, e0);
        stage_begin(c, st, &e0);
        launch_encode_group(1, ei, reinterpret_cast<const uint32_t *>(dp + o_pf), count, pf.back(), enc_smem[1], st);
        stage_end(c, st, 5, e0);
        Control *cdst = reinterpret_cast<Control *>(dp + o_cdst);
        k_gather_ctl<<<(unsigned)std::min<uint32_t>(count, (uint32_t)c->num_sms * 4), 64, 0, st>>>(
            reinterpret_cast<Control *const *>(dp + o_ctl), count, cdst);
        cudaMemcpyAsync(c->ctl_host.p, cdst, (size_t)count * sizeof(Control), cudaMemcpyDeviceToHost, st);
        c->launches += 7 + nl;
        return cudaGetLastError() == cudaSuccess ? GBSZ_OK : GBSZ_ERR_CUDA;
    };
    return run_batch(c, c->ggcomp, key, st, enqueue);
}

// One field's decompress scratch in the arena (base = nullptr only sizes it).
struct FieldDScratch {
    Control *ctl;
    uint32_t *lut, *count, *start;
    void *lutf;
    unsigned long long *first;
    uint16_t *sorted, *codes;
    int2 *dscr;
    unsigned long long *chunk_off;
    uint32_t *faces;
    void *scan_part;
};

uint64_t layout_dfield(uint8_t *base, const Header &h, FieldDScratch *f)
{
    const uint64_t n = h.n, nb = 2ull * h.p.radius;
    uint64_t gd[3];
    const uint64_t nfaces = recon_faces_entries(lorenzo_geom(h.p, gd), gd);
    uint64_t off = 0;
    auto take = [&](uint64_t bytes) -> void * {
        void *q = base ? base + off : nullptr;
        off += up256(bytes);
        return q;
    };
    f->ctl = static_cast<Control *>(take(sizeof(Control)));
    f->lut = static_cast<uint32_t *>(take(((1u << kLutBits) + kLut2Words) * 4));
    f->lutf = take(kFastLutBytes);
    f->first = static_cast<unsigned long long *>(take((kMaxLen + 2) * 8));
    f->count = static_cast<uint32_t *>(take((kMaxLen + 2) * 4));
    f->start = static_cast<uint32_t *>(take((kMaxLen + 2) * 4));
    f->sorted = static_cast<uint16_t *>(take(nb * 2));
    f->codes = static_cast<uint16_t *>(take(n * 2 + 64));
    f->dscr = static_cast<int2 *>(take(n * 8 + 64));
    f->chunk_off = static_cast<unsigned long long *>(take(h.nchunk * 8 + 8));
    f->faces = static_cast<uint32_t *>(take(nfaces * 4 + 16));
    f->scan_part = take(scan_partials(std::max<uint64_t>(h.nchunk, nfaces)) * 8 + 64);
    return off;
}

bool dgroupable(uint32_t count, const std::vector<Header> &hs, const gbsz_status *statuses)
{
    if (count < 2) return false;
    uint64_t total = 0;
    for (uint32_t i = 0; i < count; i++) {
        if (statuses[i] != GBSZ_OK || order_of(hs[i].p) != 1) return false;
        total += hs[i].n;
    }
    return total <= kGroupedMeanPoints * count;
}

gbsz_status decompress_batch_grouped(gbsz_ctx *c, uint32_t count, const std::vector<Header> &hs,
                                     const void *const *d_archives, float *const *d_fields,
                                     std::vector<uint64_t> &key, cudaStream_t st)
{
    std::vector<uint64_t> foff(count + 1, 0);
    FieldDScratch tmp;
    for (uint32_t i = 0; i < count; i++) foff[i + 1] = foff[i] + layout_dfield(nullptr, hs[i], &tmp);
    if (!c->garena.ensure(foff[count])) return GBSZ_ERR_OOM;
    uint8_t *arena = c->garena.as<uint8_t>();
    std::vector<FieldDScratch> fs(count);
    for (uint32_t i = 0; i < count; i++) layout_dfield(arena + foff[i], hs[i], &fs[i]);

    std::vector<CodebookArgs> tab(count);
    std::vector<ScanItem<ChunkWords>> osc;
    std::vector<uint32_t> osc_b;
    std::vector<DecodeItem> di(count);
    std::vector<int> dvar(count);
    std::vector<uint32_t> d_b(count);
    size_t d_smem[4] = {0, 0, 0, 0};
    std::vector<ReconArgs> ra(count);
    std::vector<ZeroRange> zr;
    std::vector<Control *> ctls(count);
    for (uint32_t i = 0; i < count; i++) {
        const Header &h = hs[i];
        const FieldDScratch &f = fs[i];
        const uint8_t *arc = static_cast<const uint8_t *>(d_archives[i]);
        uint64_t gd[3];
        const uint32_t gnd = lorenzo_geom(h.p, gd);
        const uint64_t nfaces = recon_faces_entries(gnd, gd);
        const bool tile_sums = gnd == 1 && !h.p.lorenzo_block;
        zr.push_back({f.ctl, sizeof(Control)});
        if (tile_sums) zr.push_back({f.faces, nfaces * 4});
        ctls[i] = f.ctl;
        CodebookArgs &cb = tab[i];
        cb = CodebookArgs{};
        cb.len_in = arc + kHeaderBytes;
        cb.nbins = 2 * h.p.radius;
        cb.expect_maxlen = h.maxlen;
        cb.fast_bits = fast_lut_bits(h.maxlen, cb.nbins);
        cb.fast_pair = 0;
        cb.lut = f.lut;
        cb.lutf = f.lutf;
        cb.first = f.first;
        cb.count = f.count;
        cb.start = f.start;
        cb.sorted = f.sorted;
        cb.ctl = f.ctl;
        DecodeArgs d{};
        d.archive = arc;
        d.n = h.n;
        d.chunk = h.p.chunk;
        d.nchunk = (uint32_t)h.nchunk;
        d.radius = h.p.radius;
        d.maxlen = h.maxlen;
        d.words = h.w;
        d.off_bits = h.L.bits;
        d.off_stream = h.L.stream;
        d.lut = f.lut;
        d.first = f.first;
        d.count = f.count;
        d.start = f.start;
        d.sorted = f.sorted;
        d.lutf = f.lutf;
        d.fast_bits = cb.fast_bits;
        d.fast_pair = 0;
        d.num_sms = c->num_sms;
        d.chunk_off = f.chunk_off;
        d.scan_partial = static_cast<unsigned long long *>(f.scan_part);
        d.tile_sums = tile_sums ? f.faces : nullptr;
        d.codes = f.codes;
        d.ctl = f.ctl;
        osc.push_back(ScanItem<ChunkWords>{chunk_words_op(d), h.nchunk, d.scan_partial});
        osc_b.push_back((uint32_t)scan_blocks(h.nchunk));
        size_t dyn = 0;
        d_b[i] = decode_plan(d, &di[i], &dvar[i], &dyn);
        d_smem[dvar[i]] = std::max(d_smem[dvar[i]], dyn);
        ReconArgs &r = ra[i];
        r = ReconArgs{};
        r.codes = f.codes;
        r.archive = arc;
        r.off_outl = h.L.outl;
        r.off_exc = h.L.exc;
        r.m = h.m;
        r.e = h.e;
        r.ndim = gnd;
        for (int k = 0; k < 3; k++) r.dims[k] = gd[k];
        r.radius = h.p.radius;
        r.ebx2 = h.ebx2;
        r.dscr = reinterpret_cast<int32_t *>(f.dscr);
        r.lblock = h.p.lorenzo_block;
        r.order = 1;
        r.faces = f.faces;
        r.faces_cap = nfaces;
        r.scan_partial = static_cast<uint32_t *>(f.scan_part);
        r.out = d_fields[i];
        r.ctl = f.ctl;
        r.num_sms = c->num_sms;
        if (h.L.nanch) {
            r.anchors = reinterpret_cast<const uint32_t *>(arc + h.L.anch);
            r.chunk = h.p.chunk;
        }
    }
    PlanBuilder pb;
    const uint64_t o_zr = pb.put(zr.data(), zr.size());
    const uint64_t o_tab = pb.put(tab.data(), count);
    const uint64_t o_osc = pb.put(osc.data(), osc.size());
    const std::vector<uint32_t> oscf = firsts(osc_b);
    const uint64_t o_oscf = pb.put(oscf.data(), oscf.size());
    struct DGroup {
        int variant;
        uint32_t ni, blocks;
        uint64_t o_items, o_first;
    };
    std::vector<DGroup> dg;
    for (int v = 0; v < 4; v++) {
        std::vector<DecodeItem> items;
        std::vector<uint32_t> bl;
        for (uint32_t i = 0; i < count; i++)
            if (dvar[i] == v) {
                items.push_back(di[i]);
                bl.push_back(d_b[i]);
            }
        if (items.empty()) continue;
        const std::vector<uint32_t> f = firsts(bl);
        DGroup g{v, (uint32_t)items.size(), f.back(), 0, 0};
        g.o_items = pb.put(items.data(), items.size());
        g.o_first = pb.put(f.data(), f.size());
        dg.push_back(g);
    }
    std::vector<GroupLaunch> recon;
    plan_reconstruct_group(ra.data(), count, pb.buf, recon);
    const uint64_t o_ctl = pb.put(ctls.data(), ctls.size());
    const uint64_t o_cdst = pb.put<uint8_t>(nullptr, 0);
    pb.buf.resize(o_cdst + (uint64_t)count * sizeof(Control));
    const uint64_t plan_bytes = pb.buf.size();
    if (!c->gplan_host.ensure(plan_bytes) || !c->gplan_dev.ensure(plan_bytes)) return GBSZ_ERR_OOM;
    std::memcpy(c->gplan_host.p, pb.buf.data(), plan_bytes);
    uint8_t *dp = c->gplan_dev.as<uint8_t>();
    key.push_back(0x6Du);  // grouped
    key.push_back((uint64_t)(uintptr_t)c->gplan_host.p);
    key.push_back((uint64_t)(uintptr_t)dp);
    key.push_back((uint64_t)(uintptr_t)arena);

    auto enqueue = [&]() -> gbsz_status {
        int nl = 0;
        cudaEvent_t e0;
        cudaMemcpyAsync(dp, c->gplan_host.p, plan_bytes, cudaMemcpyHostToDevice, st);
        k_zero_group<<<(unsigned)std::min<size_t>(zr.size(), (size_t)c->num_sms * 8), 256, 0, st>>>(
            reinterpret_cast<const ZeroRange *>(dp + o_zr), (uint32_t)zr.size());
        stage_begin(c, st, &e0);
        launch_decode_tables_group(reinterpret_cast<const CodebookArgs *>(dp + o_tab), count, st);
        stage_end(c, st, 6, e0);
        stage_begin(c, st, &e0);
        nl += launch_offsets_scan_group(reinterpret_cast<const ScanItem<ChunkWords> *>(dp + o_osc),
                                        reinterpret_cast<const uint32_t *>(dp + o_oscf), count, oscf.back(), st);
        stage_end(c, st, 7, e0);
        stage_begin(c, st, &e0);
        for (const DGroup &g : dg) {
            launch_decode_group(g.variant, reinterpret_cast<const DecodeItem *>(dp + g.o_items),
                                reinterpret_cast<const uint32_t *>(dp + g.o_first), g.ni, g.blocks,
                                d_smem[g.variant], st);
            nl++;
        }
        stage_end(c, st, 8, e0);
        stage_begin(c, st, &e0);
        for (const GroupLaunch &l : recon) nl += l(dp, st);
        stage_end(c, st, 9, e0);
        Control *cdst = reinterpret_cast<Control *>(dp + o_cdst);
        k_gather_ctl<<<(unsigned)std::min<uint32_t>(count, (uint32_t)c->num_sms * 4), 64, 0, st>>>(
            reinterpret_cast<Control *const *>(dp + o_ctl), count, cdst);
        cudaMemcpyAsync(c->ctl_host.p, cdst, (size_t)count * sizeof(Control), cudaMemcpyDeviceToHost, st);
        c->launches += 3 + nl;
        return cudaGetLastError() == cudaSuccess ? GBSZ_OK : GBSZ_ERR_CUDA;
    };
    return run_batch(c, c->ggdecomp, key, st, enqueue);
}

}  // namespace

namespace {
// An NVTX range named after the entry point, open for the duration of the
// call (header-only NVTX 3: a no-op unless a profiler such as Nsight
// Systems has attached its NVTX library).
struct ApiRange {
    explicit ApiRange(const char *name) { nvtxRangePushA(name); }
    ~ApiRange() { nvtxRangePop(); }
    ApiRange(const ApiRange &) = delete;
    ApiRange &operator=(const ApiRange &) = delete;
};
}  // namespace

extern "C" {

const char *gbsz_status_str(gbsz_status s)
{
    switch (s) {
    case GBSZ_OK: return "ok";
    case GBSZ_ERR_INVALID_ARG: return "invalid argument";
    case GBSZ_ERR_CAPACITY: return "output capacity too small";
    case GBSZ_ERR_CORRUPT: return "corrupt archive";
    case GBSZ_ERR_OOM: return "out of memory";
    case GBSZ_ERR_CUDA: return "CUDA error";
    case GBSZ_ERR_TIMEOUT: return "bounded device wait timed out";
    case GBSZ_ERR_UNSUPPORTED: return "unsupported device";
    case GBSZ_ERR_BOUNDS: return "index check failed (bounds-checking build)";
    }
    return "unknown status";
}

gbsz_status gbsz_create(gbsz_ctx **out, int device)
{
    if (!out) return GBSZ_ERR_INVALID_ARG;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return GBSZ_ERR_UNSUPPORTED;
    }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return GBSZ_ERR_CUDA;
    if (prop.major != 10 || prop.minor != 3) return GBSZ_ERR_UNSUPPORTED;
    DevGuard g(device);
    gbsz_ctx *c = new (std::nothrow) gbsz_ctx();
    if (!c) return GBSZ_ERR_OOM;
    c->device = device;
    c->num_sms = prop.multiProcessorCount;
    if (!c->ensure_slots(1) || !c->ctl_host.ensure(1) || !c->h_header.ensure(kHeaderBytes) ||
        !c->hdr_last.ensure(kHeaderBytes) || cudaEventCreateWithFlags(&c->fork, cudaEventDisableTiming) != cudaSuccess) {
        gbsz_destroy(c);
        cudaGetLastError();
        return GBSZ_ERR_OOM;
    }
    *out = c;
    return GBSZ_OK;
}

void gbsz_destroy(gbsz_ctx *c)
{
    if (!c) return;
    DevGuard g(c->device);
    cudaDeviceSynchronize();
    for (Slot *s : c->slots) {
        s->release();
        delete s;
    }
    c->slots.clear();
    if (c->aslot) {
        c->aslot->release();
        delete c->aslot;
    }
    c->astage_field.release();
    c->astage_archive.release();
    c->actl.release();
    if (c->adone) cudaEventDestroy(c->adone);
    c->gcomp.drop();
    c->gdecomp.drop();
    c->gsc.drop();
    c->gsd.drop();
    c->ggcomp.drop();
    c->ggdecomp.drop();
    c->garena.release();
    c->gplan_dev.release();
    c->gplan_host.release();
    c->tune_arc.release();
    c->tune_out.release();
    c->stage_field.release();
    c->stage_archive.release();
    c->ctl_host.release();
    c->h_header.release();
    for (auto &r : c->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (BatchGraph *bg : {&c->gcomp, &c->gdecomp, &c->gsc, &c->gsd, &c->ggcomp, &c->ggdecomp})
        for (auto &r : bg->recs) {
            cudaEventDestroy(r.a);
            cudaEventDestroy(r.b);
        }
    for (auto e : c->pool) cudaEventDestroy(e);
    if (c->fork) cudaEventDestroy(c->fork);
    delete c;
}

gbsz_status gbsz_set_option(gbsz_ctx *c, int option, int64_t value)
{
    if (!c) return GBSZ_ERR_INVALID_ARG;
    if (option == GBSZ_OPT_BATCH_MODE) {
        if (value != 0 && value != 1) return GBSZ_ERR_INVALID_ARG;
        c->batch_mode = (uint32_t)value;
        return GBSZ_OK;
    }
    if (option == GBSZ_OPT_TEST_HOLD_CHUNK) {
        if (value < -1 || value >= 0xFFFFFFFFll) return GBSZ_ERR_INVALID_ARG;
        c->hold_chunk = value < 0 ? ~0u : (uint32_t)value;
        return GBSZ_OK;
    }
    if (option == GBSZ_OPT_LORENZO_SLAB) {
        if (value < 0 || value > 65536) return GBSZ_ERR_INVALID_ARG;
        c->slab = (uint32_t)value;
        return GBSZ_OK;
    }
    if (option == GBSZ_OPT_DECODER) {
        if (value < 0 || value > 3) return GBSZ_ERR_INVALID_ARG;
        c->decoder = (uint32_t)value;
        return GBSZ_OK;
    }
    if (option == GBSZ_OPT_CODEWORD_BITS) {
        if (value != 0 && value != 64) return GBSZ_ERR_INVALID_ARG;
        c->cw64_only = value == 64 ? 1u : 0u;
        return GBSZ_OK;
    }
    return GBSZ_ERR_INVALID_ARG;
}

uint32_t gbsz_auto_chunk(const gbsz_params *p)
{
    uint64_t n;
    if (!valid_params(p, &n)) return 0;
    return p->chunk ? p->chunk : auto_chunk(n);
}

gbsz_status gbsz_autotune(gbsz_ctx *c, const float *d_field, const gbsz_params *p, gbsz_params *out, float *ms,
                          void *stream)
{
    const ApiRange nvtx_range("gbsz_autotune");
    uint64_t n;
    if (!c || !d_field || !p || !out || !valid_params(p, &n)) return GBSZ_ERR_INVALID_ARG;
    DevGuard g(c->device);
    *out = *p;
    if (ms) *ms = 0.0f;
    if (const Tuned *t = find_tuned(c, *p)) {
        out->chunk = t->chunk;
        return GBSZ_OK;
    }
    std::vector<uint32_t> cand{256, 512, 1024, 2048, 4096};
    const uint32_t rule = auto_chunk(n);
    if (std::find(cand.begin(), cand.end(), rule) == cand.end()) cand.push_back(rule);
    gbsz_params q = *p;
    size_t cap = 0;
    for (uint32_t C : cand) {
        q.chunk = C;
        cap = std::max(cap, gbsz_compress_bound(&q));
    }
    if (!c->tune_arc.ensure(cap) || !c->tune_out.ensure(n * 4)) return GBSZ_ERR_OOM;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = c->ev(), e1 = c->ev();
    gbsz_status status = GBSZ_OK;
    size_t nb = 0;
    // best of two timed runs after a warm-up; what = 1 compress, 2 decompress, 3 both
    auto timed = [&](int what) -> float {
        float tmin = -1.0f;
        for (int rep = 0; rep < 3 && status == GBSZ_OK; rep++) {
            cudaEventRecord(e0, st);
            if (what & 1) status = gbsz_compress(c, d_field, &q, c->tune_arc.p, cap, &nb, stream);
            if (status == GBSZ_OK && (what & 2))
                status = gbsz_decompress(c, c->tune_arc.p, nb, c->tune_out.as<float>(), n, stream);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) status = GBSZ_ERR_CUDA;
            float t = 0.0f;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0 && (tmin < 0.0f || t < tmin)) tmin = t;
        }
        return tmin;
    };
    // 1. the Huffman chunk (changes the archive), with the knobs as they are
    float best = -1.0f;
    Tuned tu{rule, 0, 0};
    for (uint32_t C : cand) {
        q.chunk = C;
        const float t = timed(3);
        if (status != GBSZ_OK) break;
        if (best < 0.0f || t < best) {
            best = t;
            tu.chunk = C;
        }
    }
    q.chunk = tu.chunk;
    const uint32_t save_dec = c->decoder, save_slab = c->slab;
    // 2. the decoder's granularity: a thread or a warp per chunk (same floats)
    if (status == GBSZ_OK && tu.chunk <= kWarpMaxChunk) {
        status = gbsz_compress(c, d_field, &q, c->tune_arc.p, cap, &nb, stream);
        float bt = -1.0f;
        for (uint32_t dec : {1u, 2u}) {
            c->decoder = dec;
            const float t = timed(2);
            if (status != GBSZ_OK) break;
            if (bt < 0.0f || t < bt) {
                bt = t;
                tu.decoder = dec;
            }
        }
        c->decoder = save_dec;
    }
    // 3. the dual-quant tile's extent along y (2D) or z (3D) (same bytes)
    uint64_t gd[3];
    const uint32_t gnd = lorenzo_geom(*p, gd);
    if (status == GBSZ_OK && gnd > 1 && order_of(*p) == 1) {
        float bt = -1.0f;
        for (uint32_t sl : {0u, 4u, 8u, 16u, 32u, 64u}) {
            if (sl > gd[gnd - 1]) break;
            c->slab = sl;
            const float t = timed(1);
            if (status != GBSZ_OK) break;
            if (bt < 0.0f || t < bt) {
                bt = t;
                tu.slab = sl;
            }
        }
        c->slab = save_slab;
    }
    c->pool.push_back(e0);
    c->pool.push_back(e1);
    if (status != GBSZ_OK) return status;
    c->tuned.push_back({tune_key(*p), tu});
    c->tuned_gen++;
    out->chunk = tu.chunk;
    if (ms) *ms = best;
    return GBSZ_OK;
}

gbsz_status gbsz_tuned_knobs(gbsz_ctx *c, const gbsz_params *p, uint32_t knobs[3])
{
    if (!c || !p || !knobs) return GBSZ_ERR_INVALID_ARG;
    const Tuned *t = find_tuned(c, *p);
    if (!t) return GBSZ_ERR_INVALID_ARG;
    knobs[0] = t->chunk;
    knobs[1] = t->decoder;
    knobs[2] = t->slab;
    return GBSZ_OK;
}

size_t gbsz_compress_bound(const gbsz_params *p)
{
    uint64_t n;
    if (!valid_params(p, &n)) return 0;
    const uint32_t C = p->chunk ? p->chunk : auto_chunk(n);
    const uint64_t nc = (n + C - 1) / C;
    const uint64_t words_max = nc + (kMaxLen * n + 31) / 32;
    return (size_t)(208 + 2ull * p->radius + 12 * nc + 16 * n + 4 * words_max);  // anchors included
}

gbsz_status gbsz_compress(gbsz_ctx *c, const float *d_field, const gbsz_params *pin, void *d_archive,
                          size_t capacity, size_t *out_bytes, void *stream)
{
    const ApiRange nvtx_range("gbsz_compress");
    if (!c || !out_bytes) return GBSZ_ERR_INVALID_ARG;
    *out_bytes = 0;
    gbsz_params p;
    uint64_t n;
    size_t need = 0;
    gbsz_status s = check_compress(d_field, pin, d_archive, capacity, &p, &n, &need);
    if (s != GBSZ_OK) {
        *out_bytes = need;
        return s;
    }
    DevGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    Slot *sl = c->slots[0];
    // a call repeated with the same buffers and parameters is replayed as a
    // CUDA graph (captured on its second identical occurrence; not on the
    // legacy default stream, which cannot be captured)
    std::vector<uint64_t> key{0x5Cu, (uint64_t)(uintptr_t)c->ctl_host.p, (uint64_t)(uintptr_t)c->hdr_last.p};
    key_add(key, &d_field, sizeof(void *));
    key_add(key, &d_archive, sizeof(void *));
    key_add(key, &capacity, sizeof(size_t));
    key.insert(key.end(), {p.ndim, p.dims[0], p.dims[1], p.dims[2], p.dims[3], p.eb_mode, p.radius, p.chunk,
                           p.lorenzo_block, p.lorenzo_order, c->cw64_only});
    key_add(key, &p.eb, sizeof(double));
    auto enqueue = [&]() -> gbsz_status {
        gbsz_status es = enqueue_compress(c, sl, d_field, p, n, d_archive, capacity, st);
        if (es == GBSZ_OK &&
            (cudaMemcpyAsync(c->ctl_host.p, sl->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
             cudaMemcpyAsync(c->hdr_last.p, d_archive, kHeaderBytes, cudaMemcpyDeviceToHost, st) != cudaSuccess))
            es = GBSZ_ERR_CUDA;
        return es;
    };
    c->hdr_valid = false;
    s = run_batch(c, c->gsc, key, st, enqueue);
    if (s != GBSZ_OK) return s;
    c->last_n = n;
    c->last_nbins = 2 * p.radius;
    c->have_compress = true;
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GBSZ_ERR_CUDA;
    prof_collect(c);
    const Control &ch = c->ctl_host.p[0];
    *out_bytes = (size_t)ch.total;
    c->last_sc[0] = ch.eb;
    c->last_sc[1] = ch.ebx2;
    c->last_sc[2] = ch.inv2eb;
    const gbsz_status ds = map_device_error(ch.error);
    if (ds == GBSZ_OK) {
        c->hdr_valid = true;
        c->hdr_ptr = d_archive;
        c->hdr_bytes = (size_t)ch.total;
    }
    return ds;
}

gbsz_status gbsz_archive_info(const void *h_archive, size_t bytes, gbsz_params *out, uint64_t *n)
{
    if (!h_archive) return GBSZ_ERR_INVALID_ARG;
    Header h;
    gbsz_status s = parse_header(static_cast<const uint8_t *>(h_archive), bytes, &h);
    if (s != GBSZ_OK) return s;
    if (out) *out = h.p;
    if (n) *n = h.n;
    return GBSZ_OK;
}

gbsz_status gbsz_decompress(gbsz_ctx *c, const void *d_archive, size_t bytes, float *d_field,
                            uint64_t capacity_elems, void *stream)
{
    const ApiRange nvtx_range("gbsz_decompress");
    if (!c || !d_archive || !d_field) return GBSZ_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(d_archive) & 15) || (reinterpret_cast<uintptr_t>(d_field) & 15))
        return GBSZ_ERR_INVALID_ARG;
    if (bytes < kHeaderBytes) return GBSZ_ERR_CORRUPT;
    DevGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    // the archive this context just wrote: plan from the header copied back
    // by that compress, check it on the device (no round trip to the host
    // before the launch); otherwise read the header first
    const bool cached = c->hdr_valid && c->hdr_ptr == d_archive && c->hdr_bytes == bytes;
    if (cached) {
        memcpy(c->h_header.p, c->hdr_last.p, kHeaderBytes);
    } else if (cudaMemcpyAsync(c->h_header.p, d_archive, kHeaderBytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
               cudaStreamSynchronize(st) != cudaSuccess) {
        return GBSZ_ERR_CUDA;
    }
    Header h;
    gbsz_status s = parse_header(c->h_header.p, bytes, &h);
    if (s == GBSZ_OK && h.n > capacity_elems) s = GBSZ_ERR_CAPACITY;
    if (s != GBSZ_OK) {
        if (!cached) return s;
        c->hdr_valid = false;  // judged by the archive's own header instead
        return gbsz_decompress(c, d_archive, bytes, d_field, capacity_elems, stream);
    }
    Slot *sl = c->slots[0];
    std::vector<uint64_t> key{0x5Du, (uint64_t)(uintptr_t)c->ctl_host.p, cached ? 1u : 0u};
    key_add(key, &d_archive, sizeof(void *));
    key_add(key, &d_field, sizeof(void *));
    key_add(key, &bytes, sizeof(size_t));
    key_add(key, c->h_header.p, kHeaderBytes);
    auto enqueue = [&]() -> gbsz_status {
        gbsz_status es = enqueue_decompress(c, sl, h, d_archive, d_field, st, cached ? c->h_header.p : nullptr);
        if (es == GBSZ_OK &&
            cudaMemcpyAsync(c->ctl_host.p, sl->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            es = GBSZ_ERR_CUDA;
        return es;
    };
    s = run_batch(c, c->gsd, key, st, enqueue);
    if (s != GBSZ_OK) return s;
    c->last_dn = h.n;
    c->have_decompress = true;
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GBSZ_ERR_CUDA;
    prof_collect(c);
    if (cached && (c->ctl_host.p[0].error & DERR_STALE)) {
        // the buffer holds another archive now: run again from its own header
        // (the stale run stayed inside the buffers, as a corrupt archive does)
        c->hdr_valid = false;
        return gbsz_decompress(c, d_archive, bytes, d_field, capacity_elems, stream);
    }
    return decompress_status(c->ctl_host.p[0], h);
}

gbsz_status gbsz_compress_batch(gbsz_ctx *c, uint32_t count, const float *const *d_fields,
                                const gbsz_params *params, void *const *d_archives, const size_t *capacities,
                                size_t *out_bytes, gbsz_status *statuses, void *stream)
{
    const ApiRange nvtx_range("gbsz_compress_batch");
    if (!c || !d_fields || !params || !d_archives || !capacities || !out_bytes || !statuses)
        return GBSZ_ERR_INVALID_ARG;
    if (count == 0) return GBSZ_OK;
    DevGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    const int K = (int)std::min<uint32_t>(count, kMaxSlots);
    if (!c->ensure_slots(K) || !c->ctl_host.ensure(count)) return GBSZ_ERR_OOM;
    std::vector<gbsz_params> rp(count);
    std::vector<uint64_t> rn(count);
    for (uint32_t i = 0; i < count; i++) {
        size_t need = 0;
        out_bytes[i] = 0;
        statuses[i] = check_compress(d_fields[i], &params[i], d_archives[i], capacities[i], &rp[i], &rn[i], &need);
        if (statuses[i] == GBSZ_ERR_CAPACITY) out_bytes[i] = need;
    }
    const bool grouped = c->batch_mode == 0 && groupable(count, rp.data(), rn.data(), statuses);
    // slot scratch is sized before any capture (a graph must not allocate)
    for (uint32_t i = 0; i < count && !grouped; i++)
        if (statuses[i] == GBSZ_OK && !reserve_compress(c->slots[i % K], rp[i], rn[i])) statuses[i] = GBSZ_ERR_OOM;
    std::vector<uint64_t> key{0xC0u, count, (uint64_t)K, (uint64_t)(uintptr_t)c->ctl_host.p};
    for (uint32_t i = 0; i < count; i++) {
        key_add(key, &d_fields[i], sizeof(void *));
        key_add(key, &d_archives[i], sizeof(void *));
        key_add(key, &capacities[i], sizeof(size_t));
        key.insert(key.end(), {rp[i].ndim, rp[i].dims[0], rp[i].dims[1], rp[i].dims[2], rp[i].dims[3],
                               rp[i].eb_mode, rp[i].radius, rp[i].chunk, rp[i].lorenzo_block,
                               rp[i].lorenzo_order, c->cw64_only});
        key_add(key, &rp[i].eb, sizeof(double));
        key.push_back((uint64_t)statuses[i]);
    }
    if (grouped) {
        const gbsz_status gs = compress_batch_grouped(c, count, d_fields, rp.data(), rn.data(), d_archives,
                                                      capacities, key, st);
        if (gs != GBSZ_OK) return gs;
        if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GBSZ_ERR_CUDA;
        prof_collect(c);
        gbsz_status first = GBSZ_OK;
        for (uint32_t i = 0; i < count; i++) {
            out_bytes[i] = (size_t)c->ctl_host.p[i].total;
            statuses[i] = map_device_error(c->ctl_host.p[i].error);
            if (first == GBSZ_OK) first = statuses[i];
        }
        return first;
    }
    auto enqueue = [&]() -> gbsz_status {
        cudaEventRecord(c->fork, st);
        for (int k = 0; k < K; k++) cudaStreamWaitEvent(c->slots[k]->stream, c->fork, 0);
        gbsz_status es = GBSZ_OK;
        for (uint32_t i = 0; i < count && es == GBSZ_OK; i++) {
            if (statuses[i] != GBSZ_OK) continue;
            Slot *sl = c->slots[i % K];
            es = enqueue_compress(c, sl, d_fields[i], rp[i], rn[i], d_archives[i], capacities[i], sl->stream);
            if (es == GBSZ_OK)
                cudaMemcpyAsync(&c->ctl_host.p[i], sl->ctl, sizeof(Control), cudaMemcpyDeviceToHost, sl->stream);
        }
        for (int k = 0; k < K; k++) {  // always joined, so a capture can end cleanly
            cudaEventRecord(c->slots[k]->done, c->slots[k]->stream);
            cudaStreamWaitEvent(st, c->slots[k]->done, 0);
        }
        return es;
    };
    const gbsz_status es = run_batch(c, c->gcomp, key, st, enqueue);
    if (es != GBSZ_OK) return es;
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GBSZ_ERR_CUDA;
    prof_collect(c);
    gbsz_status first = GBSZ_OK;
    for (uint32_t i = 0; i < count; i++) {
        if (statuses[i] == GBSZ_OK) {
            out_bytes[i] = (size_t)c->ctl_host.p[i].total;
            statuses[i] = map_device_error(c->ctl_host.p[i].error);
        }
        if (first == GBSZ_OK) first = statuses[i];
    }
    return first;
}

gbsz_status gbsz_decompress_batch(gbsz_ctx *c, uint32_t count, const void *const *d_archives, const size_t *bytes,
                                  float *const *d_fields, const uint64_t *capacities, gbsz_status *statuses,
                                  void *stream)
{
    const ApiRange nvtx_range("gbsz_decompress_batch");
    if (!c || !d_archives || !bytes || !d_fields || !capacities || !statuses) return GBSZ_ERR_INVALID_ARG;
    if (count == 0) return GBSZ_OK;
    DevGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    const int K = (int)std::min<uint32_t>(count, kMaxSlots);
    if (!c->ensure_slots(K) || !c->ctl_host.ensure(count) || !c->h_header.ensure((size_t)count * kHeaderBytes))
        return GBSZ_ERR_OOM;
    for (uint32_t i = 0; i < count; i++) {
        statuses[i] = GBSZ_OK;
        if (!d_archives[i] || !d_fields[i] || (reinterpret_cast<uintptr_t>(d_archives[i]) & 15) ||
            (reinterpret_cast<uintptr_t>(d_fields[i]) & 15)) {
            statuses[i] = GBSZ_ERR_INVALID_ARG;
            continue;
        }
        if (bytes[i] < kHeaderBytes) {
            statuses[i] = GBSZ_ERR_CORRUPT;
            continue;
        }
        cudaMemcpyAsync(c->h_header.p + (size_t)i * kHeaderBytes, d_archives[i], kHeaderBytes,
                        cudaMemcpyDeviceToHost, st);
    }
    if (cudaStreamSynchronize(st) != cudaSuccess) return GBSZ_ERR_CUDA;
    std::vector<Header> hs(count);
    for (uint32_t i = 0; i < count; i++) {
        if (statuses[i] != GBSZ_OK) continue;
        statuses[i] = parse_header(c->h_header.p + (size_t)i * kHeaderBytes, bytes[i], &hs[i]);
        if (statuses[i] == GBSZ_OK && hs[i].n > capacities[i]) statuses[i] = GBSZ_ERR_CAPACITY;
    }
    const bool grouped = c->batch_mode == 0 && dgroupable(count, hs, statuses);
    for (uint32_t i = 0; i < count && !grouped; i++)
        if (statuses[i] == GBSZ_OK && !reserve_decompress(c->slots[i % K], hs[i])) statuses[i] = GBSZ_ERR_OOM;
    std::vector<uint64_t> key{0xDEu, count, (uint64_t)K, (uint64_t)(uintptr_t)c->ctl_host.p};
    for (uint32_t i = 0; i < count; i++) {
        key_add(key, &d_archives[i], sizeof(void *));
        key_add(key, &d_fields[i], sizeof(void *));
        key_add(key, &bytes[i], sizeof(size_t));
        key.push_back((uint64_t)statuses[i]);
        if (statuses[i] == GBSZ_OK) key_add(key, c->h_header.p + (size_t)i * kHeaderBytes, kHeaderBytes);
    }
    if (grouped) {
        const gbsz_status gs = decompress_batch_grouped(c, count, hs, d_archives, d_fields, key, st);
        if (gs != GBSZ_OK) return gs;
        if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GBSZ_ERR_CUDA;
        prof_collect(c);
        gbsz_status first = GBSZ_OK;
        for (uint32_t i = 0; i < count; i++) {
            statuses[i] = decompress_status(c->ctl_host.p[i], hs[i]);
            if (first == GBSZ_OK) first = statuses[i];
        }
        return first;
    }
    auto enqueue = [&]() -> gbsz_status {
        cudaEventRecord(c->fork, st);
        for (int k = 0; k < K; k++) cudaStreamWaitEvent(c->slots[k]->stream, c->fork, 0);
        gbsz_status es = GBSZ_OK;
        for (uint32_t i = 0; i < count && es == GBSZ_OK; i++) {
            if (statuses[i] != GBSZ_OK) continue;
            Slot *sl = c->slots[i % K];
            es = enqueue_decompress(c, sl, hs[i], d_archives[i], d_fields[i], sl->stream);
            if (es == GBSZ_OK)
                cudaMemcpyAsync(&c->ctl_host.p[i], sl->ctl, sizeof(Control), cudaMemcpyDeviceToHost, sl->stream);
        }
        for (int k = 0; k < K; k++) {  // always joined, so a capture can end cleanly
            cudaEventRecord(c->slots[k]->done, c->slots[k]->stream);
            cudaStreamWaitEvent(st, c->slots[k]->done, 0);
        }
        return es;
    };
    const gbsz_status es = run_batch(c, c->gdecomp, key, st, enqueue);
    if (es != GBSZ_OK) return es;
    if (cudaStreamSynchronize(st) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GBSZ_ERR_CUDA;
    prof_collect(c);
    gbsz_status first = GBSZ_OK;
    for (uint32_t i = 0; i < count; i++) {
        if (statuses[i] == GBSZ_OK) statuses[i] = decompress_status(c->ctl_host.p[i], hs[i]);
        if (first == GBSZ_OK) first = statuses[i];
    }
    return first;
}

gbsz_status gbsz_compress_host(gbsz_ctx *c, const float *h_field, const gbsz_params *p, void *h_archive,
                               size_t capacity, size_t *out_bytes, void *stream)
{
    const ApiRange nvtx_range("gbsz_compress_host");
    uint64_t n;
    if (!c || !h_field || !h_archive || !out_bytes || !valid_params(p, &n)) return GBSZ_ERR_INVALID_ARG;
    DevGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bound = gbsz_compress_bound(p);
    if (!c->stage_field.ensure(n * 4) || !c->stage_archive.ensure(bound)) return GBSZ_ERR_OOM;
    if (cudaMemcpyAsync(c->stage_field.p, h_field, n * 4, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return GBSZ_ERR_CUDA;
    gbsz_status s = gbsz_compress(c, c->stage_field.as<float>(), p, c->stage_archive.p, bound, out_bytes, stream);
    if (s != GBSZ_OK) return s;
    if (*out_bytes > capacity) return GBSZ_ERR_CAPACITY;
    if (cudaMemcpyAsync(h_archive, c->stage_archive.p, *out_bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return GBSZ_ERR_CUDA;
    return GBSZ_OK;
}

gbsz_status gbsz_decompress_host(gbsz_ctx *c, const void *h_archive, size_t bytes, float *h_field,
                                 uint64_t capacity_elems, void *stream)
{
    const ApiRange nvtx_range("gbsz_decompress_host");
    if (!c || !h_archive || !h_field) return GBSZ_ERR_INVALID_ARG;
    Header h;
    gbsz_status s = parse_header(static_cast<const uint8_t *>(h_archive), bytes, &h);
    if (s != GBSZ_OK) return s;
    if (h.n > capacity_elems) return GBSZ_ERR_CAPACITY;
    DevGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!c->stage_field.ensure(h.n * 4) || !c->stage_archive.ensure(h.total)) return GBSZ_ERR_OOM;
    if (cudaMemcpyAsync(c->stage_archive.p, h_archive, h.total, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return GBSZ_ERR_CUDA;
    s = gbsz_decompress(c, c->stage_archive.p, h.total, c->stage_field.as<float>(), h.n, stream);
    if (s != GBSZ_OK) return s;
    if (cudaMemcpyAsync(h_field, c->stage_field.p, h.n * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return GBSZ_ERR_CUDA;
    return GBSZ_OK;
}

gbsz_status gbsz_decompress_host_async(gbsz_ctx *c, const void *h_archive, size_t bytes, float *h_field,
                                       uint64_t capacity_elems, void *stream)
{
    const ApiRange nvtx_range("gbsz_decompress_host_async");
    if (!c || !h_archive || !h_field || c->apending) return GBSZ_ERR_INVALID_ARG;
    Header h;
    gbsz_status s = parse_header(static_cast<const uint8_t *>(h_archive), bytes, &h);
    if (s != GBSZ_OK) return s;
    if (h.n > capacity_elems) return GBSZ_ERR_CAPACITY;
    DevGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!c->aslot) {
        c->aslot = new Slot();
        if (!c->aslot->init()) {
            c->aslot->release();
            delete c->aslot;
            c->aslot = nullptr;
            return GBSZ_ERR_OOM;
        }
    }
    if (!c->adone && cudaEventCreateWithFlags(&c->adone, cudaEventDisableTiming) != cudaSuccess) return GBSZ_ERR_CUDA;
    if (!c->actl.ensure(1) || !c->astage_field.ensure(h.n * 4) || !c->astage_archive.ensure(h.total))
        return GBSZ_ERR_OOM;
    if (cudaMemcpyAsync(c->astage_archive.p, h_archive, h.total, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return GBSZ_ERR_CUDA;
    s = enqueue_decompress(c, c->aslot, h, c->astage_archive.p, c->astage_field.as<float>(), st);
    if (s != GBSZ_OK) return s;
    if (cudaMemcpyAsync(h_field, c->astage_field.p, h.n * 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(c->actl.p, c->aslot->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaEventRecord(c->adone, st) != cudaSuccess)
        return GBSZ_ERR_CUDA;
    c->azeros = h.m;
    c->apending = true;
    return GBSZ_OK;
}

gbsz_status gbsz_async_wait(gbsz_ctx *c)
{
    const ApiRange nvtx_range("gbsz_async_wait");
    if (!c) return GBSZ_ERR_INVALID_ARG;
    if (!c->apending) return GBSZ_OK;
    DevGuard g(c->device);
    c->apending = false;
    if (cudaEventSynchronize(c->adone) != cudaSuccess || cudaGetLastError() != cudaSuccess) return GBSZ_ERR_CUDA;
    const Control &ctl = c->actl.p[0];
    if (ctl.error) return map_device_error(ctl.error);
    return ctl.zeros == c->azeros ? GBSZ_OK : GBSZ_ERR_CORRUPT;
}

gbsz_status gbsz_debug_copy(gbsz_ctx *c, int which, void *h_dst, size_t bytes)
{
    if (!c || !h_dst) return GBSZ_ERR_INVALID_ARG;
    DevGuard g(c->device);
    Slot *sl = c->slots[0];
    const void *src = nullptr;
    size_t need = 0;
    switch (which) {
    case 0: src = sl->codes.p; need = c->have_compress ? c->last_n * 2 : 0; break;
    case 1: src = sl->hist.p; need = c->have_compress ? c->last_nbins * 4 : 0; break;
    case 2:
        if (!c->have_compress || bytes != 12) return GBSZ_ERR_INVALID_ARG;
        std::memcpy(h_dst, c->last_sc, 12);
        return GBSZ_OK;
    case 3: src = sl->codes.p; need = c->have_decompress && c->decoded_codes ? c->last_dn * 2 : 0; break;
    case 4: src = sl->codes_only.p; need = c->have_compress ? c->last_nbins * 8 : 0; break;
    case 5:
    case 6: {
        if (bytes != 32) return GBSZ_ERR_INVALID_ARG;
        const BatchGraph &gc = which == 5 ? c->gcomp : c->gsc, &gd = which == 5 ? c->gdecomp : c->gsd;
        // batch compress: the slot-stream graphs and the grouped ones together
        const uint64_t cap = gc.captures + (which == 5 ? c->ggcomp.captures : 0);
        const uint64_t rep = gc.replays + (which == 5 ? c->ggcomp.replays : 0);
        const uint64_t dcap = gd.captures + (which == 5 ? c->ggdecomp.captures : 0);
        const uint64_t drep = gd.replays + (which == 5 ? c->ggdecomp.replays : 0);
        const uint64_t v[4] = {cap, rep, dcap, drep};
        std::memcpy(h_dst, v, 32);
        return GBSZ_OK;
    }
    default: return GBSZ_ERR_INVALID_ARG;
    }
    if (need == 0 || bytes != need) return GBSZ_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(c->last_stream) != cudaSuccess) return GBSZ_ERR_CUDA;
    if (cudaMemcpy(h_dst, src, need, cudaMemcpyDeviceToHost) != cudaSuccess) return GBSZ_ERR_CUDA;
    return GBSZ_OK;
}

gbsz_status gbsz_memory_usage(gbsz_ctx *c, uint64_t *device_bytes, uint32_t *slots)
{
    if (!c || !device_bytes) return GBSZ_ERR_INVALID_ARG;
    uint64_t t = 0;
    for (const Slot *sl : c->slots) t += sl->bytes();
    if (c->aslot) t += c->aslot->bytes();
    for (const Buf *b : {&c->stage_field, &c->stage_archive, &c->astage_field, &c->astage_archive, &c->tune_arc,
                         &c->tune_out, &c->garena, &c->gplan_dev})
        t += b->cap;
    *device_bytes = t;
    if (slots) *slots = (uint32_t)c->slots.size();
    return GBSZ_OK;
}

gbsz_status gbsz_release_scratch(gbsz_ctx *c)
{
    if (!c) return GBSZ_ERR_INVALID_ARG;
    if (c->apending) return GBSZ_ERR_INVALID_ARG;
    DevGuard g(c->device);
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        return GBSZ_ERR_CUDA;
    }
    for (BatchGraph *bg : {&c->gcomp, &c->gdecomp, &c->gsc, &c->gsd, &c->ggcomp, &c->ggdecomp}) {
        bg->drop();
        bg->seen.clear();
    }
    c->garena.release();
    c->gplan_dev.release();
    while (c->slots.size() > 1) {
        c->slots.back()->release();
        delete c->slots.back();
        c->slots.pop_back();
    }
    c->slots[0]->release_field_scratch();
    if (c->aslot) {
        c->aslot->release();
        delete c->aslot;
        c->aslot = nullptr;
    }
    for (Buf *b : {&c->stage_field, &c->stage_archive, &c->astage_field, &c->astage_archive, &c->tune_arc,
                   &c->tune_out})
        b->release();
    c->have_compress = c->have_decompress = false;
    return GBSZ_OK;
}

gbsz_status gbsz_scratch_bytes(const gbsz_params *p, int for_decompress, uint64_t *field_bytes,
                               uint64_t *slot_bytes)
{
    uint64_t n;
    if (!p || !valid_params(p, &n)) return GBSZ_ERR_INVALID_ARG;
    gbsz_params q = *p;
    if (q.chunk == 0) q.chunk = auto_chunk(n);
    if (field_bytes) *field_bytes = for_decompress ? decompress_scratch(q, n) : compress_scratch(q, n);
    if (slot_bytes) {
        const uint64_t B = kMaxBins;
        uint64_t t = sizeof(Control);
        for (uint64_t b : {B * 4, B * 8, B * 4, B * 8, B * 8, B * 8, B * 4, 2 * B * 4, 2 * B * 4, 2 * B * 4, 2 * B * 4,
                           2 * B * 4, (uint64_t)((1u << kLutBits) + kLut2Words) * 4, (uint64_t)kFastLutBytes,
                           (uint64_t)(kMaxLen + 2) * 8, (uint64_t)(kMaxLen + 2) * 4, (uint64_t)(kMaxLen + 2) * 4,
                           B * 2})
            t += buf_bytes(b);
        *slot_bytes = t;
    }
    return GBSZ_OK;
}

gbsz_status gbsz_profile_enable(gbsz_ctx *c, int enable)
{
    if (!c) return GBSZ_ERR_INVALID_ARG;
    c->profiling = enable != 0;
    return GBSZ_OK;
}

gbsz_status gbsz_profile_read(gbsz_ctx *c, double *ms, uint64_t *calls, uint64_t *kernel_launches)
{
    if (!c) return GBSZ_ERR_INVALID_ARG;
    DevGuard g(c->device);
    double acc[GBSZ_NSTAGE] = {0};
    uint64_t cnt[GBSZ_NSTAGE] = {0};
    gbsz_status s = GBSZ_OK;
    for (auto &r : c->recs) {
        if (cudaEventSynchronize(r.b) != cudaSuccess) s = GBSZ_ERR_CUDA;
        float t = 0;
        if (cudaEventElapsedTime(&t, r.a, r.b) == cudaSuccess && r.stage >= 0 && r.stage < GBSZ_NSTAGE) {
            acc[r.stage] += t;
            cnt[r.stage]++;
        }
        c->pool.push_back(r.a);
        c->pool.push_back(r.b);
    }
    c->recs.clear();
    for (int i = 0; i < GBSZ_NSTAGE; i++) {
        acc[i] += c->prof_ms[i];
        cnt[i] += c->prof_n[i];
        c->prof_ms[i] = 0;
        c->prof_n[i] = 0;
    }
    if (ms)
        for (int i = 0; i < GBSZ_NSTAGE; i++) ms[i] = acc[i];
    if (calls)
        for (int i = 0; i < GBSZ_NSTAGE; i++) calls[i] = cnt[i];
    if (kernel_launches) *kernel_launches = c->launches;
    c->launches = 0;
    return s;
}

}  // extern "C"
