// server.cu -- the serving loop behind the C ABI (gbsz_server_*): requests
// are queued, admitted against a device-memory budget and run in batches by
// worker threads, each with its own context and stream, through the batch
// entry points; the queueing logic is server_core.h.
#include "gbsz.h"
#include "server_core.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <new>

static_assert(sizeof(gbsz_params) <= sizeof(((gbsz_srv::Request *)nullptr)->params), "params do not fit");

namespace {

struct CudaWorker {
    gbsz_ctx *ctx = nullptr;
    cudaStream_t st = nullptr;
};

class CudaExecutor final : public gbsz_srv::Executor {
public:
    explicit CudaExecutor(int dev) : dev_(dev) {}

    void *new_worker() override
    {
        CudaWorker *w = new (std::nothrow) CudaWorker();
        if (!w) return nullptr;
        if (gbsz_create(&w->ctx, dev_) != GBSZ_OK) {
            delete w;
            return nullptr;
        }
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(dev_);
        const cudaError_t e = cudaStreamCreateWithFlags(&w->st, cudaStreamNonBlocking);
        cudaSetDevice(prev);
        if (e != cudaSuccess) {
            cudaGetLastError();
            gbsz_destroy(w->ctx);
            delete w;
            return nullptr;
        }
        return w;
    }

    void free_worker(void *p) override
    {
        CudaWorker *w = static_cast<CudaWorker *>(p);
        if (!w) return;
        gbsz_destroy(w->ctx);  // waits for the context's work
        if (w->st) cudaStreamDestroy(w->st);
        delete w;
    }

    // compress requests in one batch call, decompress requests in another
    void run(void *p, std::vector<gbsz_srv::Request *> &batch) override
    {
        CudaWorker *w = static_cast<CudaWorker *>(p);
        std::vector<gbsz_srv::Request *> rc, rd;
        for (auto *r : batch) (r->kind == gbsz_srv::kCompress ? rc : rd).push_back(r);
        if (!rc.empty()) {
            const size_t k = rc.size();
            std::vector<const float *> f(k);
            std::vector<gbsz_params> ps(k);
            std::vector<void *> arcs(k);
            std::vector<size_t> caps(k), nb(k, 0);
            std::vector<gbsz_status> sts(k, GBSZ_OK);
            for (size_t i = 0; i < k; i++) {
                f[i] = static_cast<const float *>(rc[i]->in);
                std::memcpy(&ps[i], rc[i]->params, sizeof(gbsz_params));
                arcs[i] = rc[i]->out;
                caps[i] = rc[i]->cap;
            }
            const gbsz_status s = gbsz_compress_batch(w->ctx, (uint32_t)k, f.data(), ps.data(), arcs.data(),
                                                      caps.data(), nb.data(), sts.data(), w->st);
            for (size_t i = 0; i < k; i++) {
                rc[i]->status = s == GBSZ_ERR_CUDA || s == GBSZ_ERR_OOM ? s : sts[i];
                rc[i]->out_bytes = nb[i];
            }
        }
        if (!rd.empty()) {
            const size_t k = rd.size();
            std::vector<const void *> arcs(k);
            std::vector<size_t> bytes(k);
            std::vector<float *> outs(k);
            std::vector<uint64_t> caps(k);
            std::vector<gbsz_status> sts(k, GBSZ_OK);
            for (size_t i = 0; i < k; i++) {
                arcs[i] = rd[i]->in;
                bytes[i] = rd[i]->in_bytes;
                outs[i] = static_cast<float *>(rd[i]->out);
                caps[i] = rd[i]->cap;
            }
            const gbsz_status s = gbsz_decompress_batch(w->ctx, (uint32_t)k, arcs.data(), bytes.data(), outs.data(),
                                                        caps.data(), sts.data(), w->st);
            for (size_t i = 0; i < k; i++) {
                rd[i]->status = s == GBSZ_ERR_CUDA || s == GBSZ_ERR_OOM ? s : sts[i];
                rd[i]->out_bytes = rd[i]->n * 4;
            }
        }
    }

    uint64_t resident(void *p) override
    {
        CudaWorker *w = static_cast<CudaWorker *>(p);
        uint64_t b = 0;
        gbsz_memory_usage(w->ctx, &b, nullptr);
        return b;
    }

    // now + every request's field scratch + the fixed tables of the slots
    // the batch calls add (a batch uses up to 8 slots)
    uint64_t estimate(void *p, const std::vector<gbsz_srv::Request *> &batch) override
    {
        CudaWorker *w = static_cast<CudaWorker *>(p);
        uint64_t b = 0;
        uint32_t slots = 1;
        gbsz_memory_usage(w->ctx, &b, &slots);
        size_t nc = 0, nd = 0;
        for (auto *r : batch) {
            b += r->mem;
            (r->kind == gbsz_srv::kCompress ? nc : nd)++;
        }
        const uint32_t want = (uint32_t)std::min<size_t>(std::max(nc, nd), 8);
        if (want > slots) b += (uint64_t)(want - slots) * slot_bytes();
        return b;
    }

    void trim(void *p) override { gbsz_release_scratch(static_cast<CudaWorker *>(p)->ctx); }

    uint64_t least(uint64_t mem) override { return slot_bytes() + mem; }

private:
    static uint64_t slot_bytes()
    {
        gbsz_params q{};
        q.ndim = 1;
        q.dims[0] = 1;
        q.dims[1] = q.dims[2] = q.dims[3] = 1;
        q.eb = 1.0;
        q.radius = 2;
        uint64_t sb = 0;
        gbsz_scratch_bytes(&q, 0, nullptr, &sb);
        return sb;
    }
    int dev_;
};

}  // namespace

struct gbsz_server {
    CudaExecutor ex;
    gbsz_srv::Core core;
    gbsz_server(int dev, uint32_t workers, uint32_t max_batch, uint64_t budget)
        : ex(dev), core(&ex, workers, max_batch, budget)
    {
    }
};

extern "C" {

gbsz_status gbsz_server_create(gbsz_server **out, int device, uint32_t workers, uint32_t max_batch,
                               uint64_t mem_budget)
{
    if (!out || workers < 1 || workers > 64 || max_batch < 1 || max_batch > 1024 || mem_budget == 0)
        return GBSZ_ERR_INVALID_ARG;
    *out = nullptr;
    gbsz_server *s = new (std::nothrow) gbsz_server(device, workers, max_batch, mem_budget);
    if (!s) return GBSZ_ERR_OOM;
    if (!s->core.start()) {
        delete s;
        // a worker's context could not be created: report what gbsz_create says
        gbsz_ctx *probe = nullptr;
        const gbsz_status st = gbsz_create(&probe, device);
        gbsz_destroy(probe);
        return st == GBSZ_OK ? GBSZ_ERR_OOM : st;
    }
    *out = s;
    return GBSZ_OK;
}

void gbsz_server_destroy(gbsz_server *s)
{
    if (!s) return;
    s->core.stop();
    delete s;
}

gbsz_status gbsz_server_submit_compress(gbsz_server *s, const float *d_field, const gbsz_params *p,
                                        void *d_archive, size_t capacity, uint64_t *ticket)
{
    if (!s || !d_field || !p || !d_archive || !ticket || gbsz_compress_bound(p) == 0) return GBSZ_ERR_INVALID_ARG;
    gbsz_srv::Request r;
    r.kind = gbsz_srv::kCompress;
    r.in = d_field;
    r.out = d_archive;
    r.cap = capacity;
    r.n = 1;
    for (uint32_t i = 0; i < p->ndim; i++) r.n *= p->dims[i];
    std::memcpy(r.params, p, sizeof(gbsz_params));
    if (gbsz_scratch_bytes(p, 0, &r.mem, nullptr) != GBSZ_OK) return GBSZ_ERR_INVALID_ARG;
    *ticket = s->core.submit(r);
    return *ticket ? GBSZ_OK : GBSZ_ERR_CAPACITY;
}

gbsz_status gbsz_server_submit_decompress(gbsz_server *s, const void *d_archive, size_t bytes, float *d_field,
                                          uint64_t capacity_elems, uint64_t *ticket)
{
    if (!s || !d_archive || !d_field || !ticket || capacity_elems == 0) return GBSZ_ERR_INVALID_ARG;
    gbsz_srv::Request r;
    r.kind = gbsz_srv::kDecompress;
    r.in = d_archive;
    r.in_bytes = bytes;
    r.out = d_field;
    r.cap = capacity_elems;
    // the archive's parameters fix the scratch its decompression takes
    unsigned char hdr[128];
    if (bytes < sizeof(hdr)) return GBSZ_ERR_CORRUPT;
    if (cudaMemcpy(hdr, d_archive, sizeof(hdr), cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaGetLastError();
        return GBSZ_ERR_CUDA;
    }
    gbsz_params hp;
    uint64_t n = 0;
    const gbsz_status hs = gbsz_archive_info(hdr, bytes, &hp, &n);
    if (hs != GBSZ_OK) return hs;
    r.n = n;
    if (gbsz_scratch_bytes(&hp, 1, &r.mem, nullptr) != GBSZ_OK) return GBSZ_ERR_CORRUPT;
    *ticket = s->core.submit(r);
    return *ticket ? GBSZ_OK : GBSZ_ERR_CAPACITY;
}

gbsz_status gbsz_server_poll(gbsz_server *s, uint64_t ticket, int *done, gbsz_status *status, size_t *out_bytes)
{
    if (!s || !done) return GBSZ_ERR_INVALID_ARG;
    int st = 0;
    uint64_t ob = 0;
    const int r = s->core.poll(ticket, &st, &ob);
    if (r < 0) return GBSZ_ERR_INVALID_ARG;
    *done = r;
    if (r && status) *status = static_cast<gbsz_status>(st);
    if (r && out_bytes) *out_bytes = (size_t)ob;
    return GBSZ_OK;
}

gbsz_status gbsz_server_wait(gbsz_server *s, uint64_t ticket, double timeout_s, gbsz_status *status,
                             size_t *out_bytes)
{
    if (!s) return GBSZ_ERR_INVALID_ARG;
    int st = 0;
    uint64_t ob = 0;
    const int r = s->core.wait(ticket, timeout_s, &st, &ob);
    if (r < 0) return GBSZ_ERR_INVALID_ARG;
    if (r == 0) return GBSZ_ERR_TIMEOUT;
    if (status) *status = static_cast<gbsz_status>(st);
    if (out_bytes) *out_bytes = (size_t)ob;
    return GBSZ_OK;
}

gbsz_status gbsz_server_stats(gbsz_server *s, double *out6)
{
    if (!s || !out6) return GBSZ_ERR_INVALID_ARG;
    s->core.stats(out6);
    return GBSZ_OK;
}

gbsz_status gbsz_server_memory(gbsz_server *s, uint64_t *out4)
{
    if (!s || !out4) return GBSZ_ERR_INVALID_ARG;
    out4[0] = s->core.in_use();
    out4[1] = s->core.peak();
    out4[2] = s->core.trims();
    out4[3] = s->core.overruns();
    return GBSZ_OK;
}

}  // extern "C"
