// gbsz_api.cu -- host side of the C ABI declared in include/gbsz.h:
// context with resident device scratch, argument validation, archive header
// parsing, stage orchestration on the caller's stream, stage timing.
#include "../../include/gbsz.h"
#include "common.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

using namespace gbsz;

namespace {

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

struct Buf {
    void *p = nullptr;
    size_t cap = 0;
    bool ensure(size_t bytes)
    {
        if (bytes <= cap && p) return true;
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
        if (p) cudaFree(p);
        p = nullptr;
        cap = 0;
    }
    template <typename T> T *as() const { return static_cast<T *>(p); }
};

struct StageRec {
    int stage;
    cudaEvent_t a, b;
};

}  // namespace

struct gbsz_ctx {
    int device = 0;
    int num_sms = 152;
    cudaStream_t last_stream = nullptr;
    Control *ctl = nullptr;
    Control *ctl_host = nullptr;  // pinned
    uint8_t *h_header = nullptr;  // pinned, kHeaderBytes
    // per-field scratch (grown on demand)
    Buf codes, dscr, lb_flag, lb_agg, lb_inc, chunk_off, faces;
    // fixed-size scratch
    Buf hist, cw64, cw32, codes_only, keyA, keyB, nodef, parent, distA, distB, parA, parB;
    Buf lut, first, count, start, sorted;
    // staging of the host-buffer API
    Buf stage_field, stage_archive;
    uint32_t epoch = 0;
    size_t lb_units = 0;
    // last call (debug copies)
    uint64_t last_n = 0, last_dn = 0;
    uint32_t last_nbins = 0;
    float last_sc[3] = {0, 0, 0};  // error-bound scalars of the last compress
    bool have_compress = false, have_decompress = false;
    // timing
    bool profiling = false;
    std::vector<StageRec> recs;
    std::vector<cudaEvent_t> pool;
    uint64_t launches = 0;

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
};

namespace {

constexpr uint32_t kUnitSymbols = 4096;  // encoder work unit (symbols)

bool valid_params(const gbsz_params *p, uint64_t *n_out)
{
    if (!p || p->ndim < 1 || p->ndim > 3) return false;
    uint64_t n = 1;
    for (uint32_t i = 0; i < 3; i++) {
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
    *n_out = n;
    return true;
}

uint32_t auto_chunk(uint64_t n)
{
    // about 128 chunks per SM of a 152-SM GB300, between 64 and 4096 symbols
    uint64_t target = n / (152ull * 128ull);
    uint32_t c = 64;
    while (c < 4096 && (uint64_t)c * 2 <= target) c *= 2;
    return c;
}

gbsz_status map_device_error(uint32_t e)
{
    if (e & DERR_INTERNAL) return GBSZ_ERR_CUDA;
    if (e & DERR_TIMEOUT) return GBSZ_ERR_TIMEOUT;
    if (e & DERR_EB) return GBSZ_ERR_INVALID_ARG;
    if (e & DERR_CORRUPT) return GBSZ_ERR_CORRUPT;
    if (e & DERR_CAPACITY) return GBSZ_ERR_CAPACITY;
    return GBSZ_OK;
}

void stage_begin(gbsz_ctx *c, cudaStream_t st, cudaEvent_t *e)
{
    *e = nullptr;
    if (!c->profiling) return;
    *e = c->ev();
    cudaEventRecord(*e, st);
}

void stage_end(gbsz_ctx *c, cudaStream_t st, int stage, cudaEvent_t a)
{
    if (!c->profiling || !a) return;
    cudaEvent_t b = c->ev();
    cudaEventRecord(b, st);
    c->recs.push_back({stage, a, b});
}

bool ensure_fixed(gbsz_ctx *c)
{
    const size_t B = kMaxBins;
    return c->hist.ensure(B * 4) && c->cw64.ensure(B * 8) && c->cw32.ensure(B * 4) &&
           c->codes_only.ensure(B * 8) && c->keyA.ensure(B * 8) && c->keyB.ensure(B * 8) &&
           c->nodef.ensure(B * 4) && c->parent.ensure(2 * B * 4) && c->distA.ensure(2 * B * 4) &&
           c->distB.ensure(2 * B * 4) && c->parA.ensure(2 * B * 4) && c->parB.ensure(2 * B * 4) &&
           c->lut.ensure((1u << kLutBits) * 4) && c->first.ensure((kMaxLen + 2) * 8) &&
           c->count.ensure((kMaxLen + 2) * 4) && c->start.ensure((kMaxLen + 2) * 4) && c->sorted.ensure(B * 2);
}

CodebookArgs codebook_args(gbsz_ctx *c)
{
    CodebookArgs a{};
    a.cw64 = c->cw64.as<uint64_t>();
    a.cw32 = c->cw32.as<uint32_t>();
    a.codes_only = c->codes_only.as<uint64_t>();
    a.lut = c->lut.as<uint32_t>();
    a.first = c->first.as<unsigned long long>();
    a.count = c->count.as<uint32_t>();
    a.start = c->start.as<uint32_t>();
    a.sorted = c->sorted.as<uint16_t>();
    a.keyA = c->keyA.as<unsigned long long>();
    a.keyB = c->keyB.as<unsigned long long>();
    a.nodef = c->nodef.as<uint32_t>();
    a.parent = c->parent.as<uint32_t>();
    a.distA = c->distA.as<uint32_t>();
    a.distB = c->distB.as<uint32_t>();
    a.parA = c->parA.as<uint32_t>();
    a.parB = c->parB.as<uint32_t>();
    a.ctl = c->ctl;
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
    p.eb = rd<double>(b, H_EB);
    p.radius = rd<uint32_t>(b, H_RADIUS);
    p.chunk = rd<uint32_t>(b, H_CHUNK);
    uint64_t n;
    if (!valid_params(&p, &n) || p.chunk == 0) return GBSZ_ERR_CORRUPT;
    if (rd<uint64_t>(b, H_N) != n || rd<uint32_t>(b, H_LBLOCK) != 0) return GBSZ_ERR_CORRUPT;
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
    h->L = make_layout(p.radius, h->nchunk, h->m, h->e, h->w);
    if (h->total != h->L.total || h->total > bytes) return GBSZ_ERR_CORRUPT;
    return GBSZ_OK;
}

gbsz_status finish(gbsz_ctx *c, cudaStream_t st)
{
    if (cudaMemcpyAsync(c->ctl_host, c->ctl, sizeof(Control), cudaMemcpyDeviceToHost, st) != cudaSuccess)
        return GBSZ_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return GBSZ_ERR_CUDA;
    if (cudaGetLastError() != cudaSuccess) return GBSZ_ERR_CUDA;
    return GBSZ_OK;
}

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
    if (cudaMalloc(&c->ctl, sizeof(Control)) != cudaSuccess ||
        cudaMallocHost(&c->ctl_host, sizeof(Control)) != cudaSuccess ||
        cudaMallocHost(&c->h_header, kHeaderBytes) != cudaSuccess || !ensure_fixed(c)) {
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
    for (Buf *b : {&c->codes, &c->dscr, &c->lb_flag, &c->lb_agg, &c->lb_inc, &c->chunk_off, &c->faces, &c->hist,
                   &c->cw64, &c->cw32, &c->codes_only, &c->keyA, &c->keyB, &c->nodef, &c->parent, &c->distA,
                   &c->distB, &c->parA, &c->parB, &c->lut, &c->first, &c->count, &c->start, &c->sorted,
                   &c->stage_field, &c->stage_archive})
        b->release();
    for (auto &r : c->recs) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : c->pool) cudaEventDestroy(e);
    if (c->ctl) cudaFree(c->ctl);
    if (c->ctl_host) cudaFreeHost(c->ctl_host);
    if (c->h_header) cudaFreeHost(c->h_header);
    delete c;
}

uint32_t gbsz_auto_chunk(const gbsz_params *p)
{
    uint64_t n;
    if (!valid_params(p, &n)) return 0;
    return p->chunk ? p->chunk : auto_chunk(n);
}

size_t gbsz_compress_bound(const gbsz_params *p)
{
    uint64_t n;
    if (!valid_params(p, &n)) return 0;
    const uint32_t C = p->chunk ? p->chunk : auto_chunk(n);
    const uint64_t nc = (n + C - 1) / C;
    const uint64_t words_max = nc + (kMaxLen * n + 31) / 32;
    return (size_t)(192 + 2ull * p->radius + 8 * nc + 16 * n + 4 * words_max);
}

gbsz_status gbsz_compress(gbsz_ctx *c, const float *d_field, const gbsz_params *pin, void *d_archive,
                          size_t capacity, size_t *out_bytes, void *stream)
{
    uint64_t n;
    if (!c || !d_field || !d_archive || !out_bytes || !valid_params(pin, &n)) return GBSZ_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_archive) & 15) return GBSZ_ERR_INVALID_ARG;
    gbsz_params p = *pin;
    if (p.chunk == 0) p.chunk = auto_chunk(n);
    *out_bytes = 0;
    DevGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    const uint32_t nbins = 2 * p.radius;
    const uint64_t nchunk = (n + p.chunk - 1) / p.chunk;
    const Layout Lmin = make_layout(p.radius, nchunk, 0, 0, 0);
    if (capacity < Lmin.stream) {
        *out_bytes = Lmin.stream;
        return GBSZ_ERR_CAPACITY;
    }
    const uint64_t U = p.chunk > kUnitSymbols ? p.chunk : kUnitSymbols;
    const uint64_t nunits = (n + U - 1) / U;
    if (!c->codes.ensure(n * 2 + 64) || !c->dscr.ensure(n * 4 + 64)) return GBSZ_ERR_OOM;
    if (nunits > c->lb_units) {
        if (!c->lb_flag.ensure(nunits * 4) || !c->lb_agg.ensure(nunits * 16) || !c->lb_inc.ensure(nunits * 16))
            return GBSZ_ERR_OOM;
        cudaMemsetAsync(c->lb_flag.p, 0, c->lb_flag.cap, st);
        // capacity in units is that of the smallest of the three arrays
        c->lb_units = std::min(c->lb_flag.cap / 4, std::min(c->lb_agg.cap, c->lb_inc.cap) / 16);
        c->epoch = 0;
    }
    if (++c->epoch >= (1u << 29)) {
        cudaMemsetAsync(c->lb_flag.p, 0, c->lb_flag.cap, st);
        c->epoch = 1;
    }
    cudaMemsetAsync(c->ctl, 0, sizeof(Control), st);
    cudaMemsetAsync(c->hist.p, 0, nbins * 4, st);

    cudaEvent_t e0;
    stage_begin(c, st, &e0);
    launch_minmax_eb(d_field, n, c->ctl, p.eb, p.eb_mode, c->num_sms, st);
    stage_end(c, st, 0, e0);

    QuantArgs q{};
    q.x = d_field;
    for (int i = 0; i < 3; i++) q.dims[i] = p.dims[i];
    q.ndim = p.ndim;
    q.radius = p.radius;
    q.codes = c->codes.as<uint16_t>();
    q.dscr = c->dscr.as<int32_t>();
    q.hist = c->hist.as<uint32_t>();
    q.ctl = c->ctl;
    q.num_sms = c->num_sms;
    stage_begin(c, st, &e0);
    launch_dualquant(q, st);
    stage_end(c, st, 1, e0);

    CodebookArgs cb = codebook_args(c);
    cb.hist = c->hist.as<uint32_t>();
    cb.nbins = nbins;
    cb.len_out = static_cast<uint8_t *>(d_archive) + kHeaderBytes;
    stage_begin(c, st, &e0);
    launch_codebook(cb, st);
    stage_end(c, st, 2, e0);

    EncodeArgs en{};
    en.codes = q.codes;
    en.x = d_field;
    en.dscr = q.dscr;
    en.n = n;
    en.chunk = p.chunk;
    en.radius = p.radius;
    en.nbins = nbins;
    en.cw64 = cb.cw64;
    en.cw32 = cb.cw32;
    en.archive = static_cast<uint8_t *>(d_archive);
    en.capacity = capacity;
    en.lb_flag = c->lb_flag.as<uint32_t>();
    en.lb_agg = c->lb_agg.as<ulonglong2>();
    en.lb_inc = c->lb_inc.as<ulonglong2>();
    en.epoch = c->epoch;
    en.ctl = c->ctl;
    en.ndim = p.ndim;
    en.eb_mode = p.eb_mode;
    for (int i = 0; i < 3; i++) en.dims[i] = p.dims[i];
    en.eb = p.eb;
    en.num_sms = c->num_sms;
    stage_begin(c, st, &e0);
    launch_encode(en, st);
    stage_end(c, st, 3, e0);
    c->launches += 4;

    c->last_n = n;
    c->last_nbins = nbins;
    c->have_compress = true;
    gbsz_status s = finish(c, st);
    if (s != GBSZ_OK) return s;
    const uint32_t derr = c->ctl_host->error;
    *out_bytes = (size_t)c->ctl_host->total;
    c->last_sc[0] = c->ctl_host->eb;
    c->last_sc[1] = c->ctl_host->ebx2;
    c->last_sc[2] = c->ctl_host->inv2eb;
    return map_device_error(derr);
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
    if (!c || !d_archive || !d_field) return GBSZ_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(d_archive) & 15) || (reinterpret_cast<uintptr_t>(d_field) & 15))
        return GBSZ_ERR_INVALID_ARG;
    if (bytes < kHeaderBytes) return GBSZ_ERR_CORRUPT;
    DevGuard g(c->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    c->last_stream = st;
    if (cudaMemcpyAsync(c->h_header, d_archive, kHeaderBytes, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return GBSZ_ERR_CUDA;
    Header h;
    gbsz_status s = parse_header(c->h_header, bytes, &h);
    if (s != GBSZ_OK) return s;
    if (h.n > capacity_elems) return GBSZ_ERR_CAPACITY;
    const uint64_t n = h.n;
    const uint64_t nfaces = recon_faces_entries(h.p.ndim, h.p.dims);
    if (!c->codes.ensure(n * 2 + 64) || !c->dscr.ensure(n * 4 + 64) || !c->chunk_off.ensure(h.nchunk * 8 + 8) ||
        !c->faces.ensure(nfaces * 4 + 16))
        return GBSZ_ERR_OOM;
    cudaMemsetAsync(c->ctl, 0, sizeof(Control), st);
    const uint8_t *arc = static_cast<const uint8_t *>(d_archive);

    CodebookArgs cb = codebook_args(c);
    cb.len_in = arc + kHeaderBytes;
    cb.nbins = 2 * h.p.radius;
    cb.expect_maxlen = h.maxlen;
    cudaEvent_t e0;
    stage_begin(c, st, &e0);
    launch_decode_tables(cb, st);
    stage_end(c, st, 4, e0);

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
    d.chunk_off = c->chunk_off.as<unsigned long long>();
    d.codes = c->codes.as<uint16_t>();
    d.ctl = c->ctl;
    stage_begin(c, st, &e0);
    launch_decode(d, st);
    stage_end(c, st, 5, e0);

    ReconArgs r{};
    r.codes = d.codes;
    r.archive = arc;
    r.off_outl = h.L.outl;
    r.off_exc = h.L.exc;
    r.m = h.m;
    r.e = h.e;
    r.ndim = h.p.ndim;
    for (int i = 0; i < 3; i++) r.dims[i] = h.p.dims[i];
    r.radius = h.p.radius;
    r.ebx2 = h.ebx2;
    r.dscr = c->dscr.as<int32_t>();
    r.faces = c->faces.as<uint32_t>();
    r.faces_cap = nfaces;
    r.out = d_field;
    r.ctl = c->ctl;
    r.num_sms = c->num_sms;
    int nl = 0;
    stage_begin(c, st, &e0);
    launch_reconstruct(r, st, &nl);
    stage_end(c, st, 6, e0);
    c->launches += 3 + nl;

    c->last_dn = n;
    c->have_decompress = true;
    s = finish(c, st);
    if (s != GBSZ_OK) return s;
    const uint32_t derr = c->ctl_host->error;
    if (derr) return map_device_error(derr);
    if (c->ctl_host->zeros != h.m) return GBSZ_ERR_CORRUPT;
    return GBSZ_OK;
}

gbsz_status gbsz_compress_host(gbsz_ctx *c, const float *h_field, const gbsz_params *p, void *h_archive,
                               size_t capacity, size_t *out_bytes, void *stream)
{
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

gbsz_status gbsz_debug_copy(gbsz_ctx *c, int which, void *h_dst, size_t bytes)
{
    if (!c || !h_dst) return GBSZ_ERR_INVALID_ARG;
    DevGuard g(c->device);
    const void *src = nullptr;
    size_t need = 0;
    switch (which) {
    case 0: src = c->codes.p; need = c->have_compress ? c->last_n * 2 : 0; break;
    case 1: src = c->hist.p; need = c->have_compress ? c->last_nbins * 4 : 0; break;
    case 2:
        if (!c->have_compress || bytes != 12) return GBSZ_ERR_INVALID_ARG;
        std::memcpy(h_dst, c->last_sc, 12);
        return GBSZ_OK;
    case 3: src = c->codes.p; need = c->have_decompress ? c->last_dn * 2 : 0; break;
    case 4: src = c->codes_only.p; need = c->have_compress ? c->last_nbins * 8 : 0; break;
    default: return GBSZ_ERR_INVALID_ARG;
    }
    if (need == 0 || bytes != need) return GBSZ_ERR_INVALID_ARG;
    if (cudaStreamSynchronize(c->last_stream) != cudaSuccess) return GBSZ_ERR_CUDA;
    if (cudaMemcpy(h_dst, src, need, cudaMemcpyDeviceToHost) != cudaSuccess) return GBSZ_ERR_CUDA;
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
    if (ms)
        for (int i = 0; i < GBSZ_NSTAGE; i++) ms[i] = acc[i];
    if (calls)
        for (int i = 0; i < GBSZ_NSTAGE; i++) calls[i] = cnt[i];
    if (kernel_launches) *kernel_launches = c->launches;
    c->launches = 0;
    return s;
}

}  // extern "C"
