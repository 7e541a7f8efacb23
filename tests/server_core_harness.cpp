// Test harness of the serving loop's host logic (server_core.h) with a
// stand-in executor: no GPU.  Each "request" sleeps for a fixed time; the
// executor records how many ran at once, the counted memory it saw, and
// every request's start and end times.  A stand-in worker holds `fixed`
// bytes plus, after a batch, the scratch of the largest request it ran (as
// a context's slots keep the size of the largest field), until trimmed.
#include "server_core.h"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <map>
#include <mutex>
#include <thread>

namespace {

struct FakeWorker {
    uint64_t held = 0;
};

struct Fake final : gbsz_srv::Executor {
    gbsz_srv::Core *core = nullptr;
    int delay_ms = 20;
    uint64_t fixed = 0;
    std::mutex mu;
    int running = 0, max_running = 0, max_batch_seen = 0;
    uint64_t max_mem = 0;
    std::map<uint64_t, std::pair<double, double>> times;
    void *new_worker() override
    {
        FakeWorker *w = new FakeWorker();
        w->held = fixed;
        return w;
    }
    void free_worker(void *w) override { delete static_cast<FakeWorker *>(w); }
    uint64_t resident(void *w) override { return static_cast<FakeWorker *>(w)->held; }
    uint64_t estimate(void *w, const std::vector<gbsz_srv::Request *> &b) override
    {
        uint64_t e = static_cast<FakeWorker *>(w)->held;
        for (auto *r : b) e += r->mem;
        return e;
    }
    void trim(void *w) override { static_cast<FakeWorker *>(w)->held = fixed; }
    uint64_t least(uint64_t mem) override { return fixed + mem; }
    void run(void *wp, std::vector<gbsz_srv::Request *> &b) override
    {
        FakeWorker *fw = static_cast<FakeWorker *>(wp);
        uint64_t big = 0;
        for (auto *r : b) big = std::max(big, r->mem);
        fw->held = std::max(fw->held, fixed + big);
        const double t0 = gbsz_srv::now_s();
        {
            std::lock_guard<std::mutex> g(mu);
            running += (int)b.size();
            max_running = std::max(max_running, running);
            max_batch_seen = std::max(max_batch_seen, (int)b.size());
            max_mem = std::max(max_mem, core->in_use());
        }
        std::this_thread::sleep_for(std::chrono::milliseconds(delay_ms));
        const double t1 = gbsz_srv::now_s();
        std::lock_guard<std::mutex> g(mu);
        running -= (int)b.size();
        for (auto *r : b) {
            r->status = 0;
            r->out_bytes = r->n * 2 + (uint64_t)r->kind;
            times[r->id] = {t0, t1};
        }
    }
};

struct Harness {
    Fake fake;
    gbsz_srv::Core core;
    Harness(uint32_t w, uint32_t b, uint64_t budget, int delay, uint64_t fixed) : core(&fake, w, b, budget)
    {
        fake.core = &core;
        fake.delay_ms = delay;
        fake.fixed = fixed;
    }
};

}  // namespace

extern "C" {
void *h_new(uint32_t workers, uint32_t max_batch, uint64_t budget, int delay_ms, uint64_t fixed)
{
    Harness *h = new Harness(workers, max_batch, budget, delay_ms, fixed);
    if (!h->core.start()) {
        delete h;
        return nullptr;
    }
    return h;
}
uint64_t h_submit(void *p, int kind, uint64_t n, uint64_t mem)
{
    gbsz_srv::Request r;
    r.kind = kind;
    r.n = n;
    r.mem = mem;
    return static_cast<Harness *>(p)->core.submit(r);
}
int h_wait(void *p, uint64_t t, double timeout, int *status, uint64_t *out_bytes)
{
    return static_cast<Harness *>(p)->core.wait(t, timeout, status, out_bytes);
}
int h_poll(void *p, uint64_t t, int *status, uint64_t *out_bytes)
{
    return static_cast<Harness *>(p)->core.poll(t, status, out_bytes);
}
void h_stats(void *p, double *out6) { static_cast<Harness *>(p)->core.stats(out6); }
void h_times(void *p, uint64_t t, double *t0, double *t1)
{
    Harness *h = static_cast<Harness *>(p);
    std::lock_guard<std::mutex> g(h->fake.mu);
    *t0 = h->fake.times[t].first;
    *t1 = h->fake.times[t].second;
}
void h_limits(void *p, int *max_running, int *max_batch, uint64_t *max_mem)
{
    Harness *h = static_cast<Harness *>(p);
    std::lock_guard<std::mutex> g(h->fake.mu);
    *max_running = h->fake.max_running;
    *max_batch = h->fake.max_batch_seen;
    *max_mem = h->fake.max_mem;
}
void h_memory(void *p, uint64_t *in_use, uint64_t *peak, uint64_t *trims, uint64_t *overruns)
{
    Harness *h = static_cast<Harness *>(p);
    *in_use = h->core.in_use();
    *peak = h->core.peak();
    *trims = h->core.trims();
    *overruns = h->core.overruns();
}
void h_stop(void *p) { static_cast<Harness *>(p)->core.stop(); }
void h_free(void *p) { delete static_cast<Harness *>(p); }
}
