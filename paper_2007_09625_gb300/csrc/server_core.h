// server_core.h -- host logic of the continuous-batching request loop:
// a FIFO queue, admission by a device-memory budget (every worker's resident
// context memory counted), batches of at most
// max_batch requests taken by worker threads, completion tickets and latency
// statistics.  Pure C++ (no CUDA): the work itself is done by an Executor,
// which the library implements with its batch entry points (server.cu) and
// the host-logic tests with a stand-in.
#pragma once

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

namespace gbsz_srv {

enum Kind : int { kCompress = 0, kDecompress = 1 };

struct Request {
    uint64_t id = 0;
    int kind = kCompress;
    const void *in = nullptr;  // compress: field; decompress: archive
    void *out = nullptr;       // compress: archive; decompress: field
    uint64_t in_bytes = 0;     // decompress: archive bytes
    uint64_t cap = 0;          // compress: archive bytes; decompress: field elements
    uint64_t n = 0;            // field elements
    unsigned char params[96];  // the executor's parameters (opaque here)
    uint64_t mem = 0;          // device bytes the request holds while it runs
    double t_arrive = 0, t_start = 0, t_done = 0;
    int status = 0;
    uint64_t out_bytes = 0;
    bool done = false;
};

// Device memory of a worker is its resident state: what its context holds
// between batches (fixed tables and scratch grown for the largest fields it
// ran).  The core counts every worker's resident bytes against the budget
// at all times, and admits a batch only if the worker's resident bytes after
// it -- estimated from above before, measured after -- keep the total within
// the budget.  A worker that cannot admit the oldest request because of
// memory releases its own scratch first.
class Executor {
public:
    virtual ~Executor() = default;
    virtual void *new_worker() = 0;  // per-thread state (nullptr = failure)
    virtual void free_worker(void *w) = 0;
    // runs a batch; sets status and out_bytes of every request
    virtual void run(void *w, std::vector<Request *> &batch) = 0;
    // device bytes the worker holds now
    virtual uint64_t resident(void *w) = 0;
    // an upper bound of resident(w) after running the batch
    virtual uint64_t estimate(void *w, const std::vector<Request *> &batch) = 0;
    // releases the worker's scratch, keeping what it needs to exist
    virtual void trim(void *w) = 0;
    // the least a worker holds after running one request of `mem` scratch bytes
    virtual uint64_t least(uint64_t mem) = 0;
};

inline double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

class Core {
public:
    Core(Executor *ex, uint32_t workers, uint32_t max_batch, uint64_t budget)
        : ex_(ex), nworkers_(workers), max_batch_(max_batch), budget_(budget)
    {
    }
    ~Core() { stop(); }

    // starts the worker threads; false if a worker's state could not be made
    bool start()
    {
        std::vector<void *> states;
        for (uint32_t i = 0; i < nworkers_; i++) {
            void *w = ex_->new_worker();
            if (!w) {
                for (void *s : states) ex_->free_worker(s);
                return false;
            }
            states.push_back(w);
        }
        held_.assign(states.size(), 0);
        for (size_t i = 0; i < states.size(); i++) {
            held_[i] = ex_->resident(states[i]);
            in_use_ += held_[i];
        }
        for (size_t i = 0; i < states.size(); i++) {
            void *w = states[i];
            threads_.emplace_back([this, w, i] { worker_loop(w, i); });
        }
        return true;
    }

    // queues a request; returns its ticket, or 0 if it needs more memory
    // than the whole budget (rejected) or the server is stopping
    uint64_t submit(const Request &r)
    {
        std::lock_guard<std::mutex> g(mu_);
        if (stopping_ || ex_->least(r.mem) > budget_) return 0;
        Request *q = new Request(r);
        q->id = next_id_++;
        q->t_arrive = now_s();
        q->done = false;
        all_[q->id] = q;
        queue_.push_back(q);
        cv_work_.notify_one();
        return q->id;
    }

    // -1: unknown ticket; 0: pending; 1: done (the ticket is then released)
    int poll(uint64_t id, int *status, uint64_t *out_bytes)
    {
        std::lock_guard<std::mutex> g(mu_);
        return take_if_done(id, status, out_bytes);
    }

    // waits up to timeout_s seconds (< 0: no limit); same results as poll
    int wait(uint64_t id, double timeout_s, int *status, uint64_t *out_bytes)
    {
        std::unique_lock<std::mutex> g(mu_);
        const auto pred = [&] {
            auto it = all_.find(id);
            return it == all_.end() || it->second->done;
        };
        if (timeout_s < 0) cv_done_.wait(g, pred);
        else cv_done_.wait_for(g, std::chrono::duration<double>(timeout_s), pred);
        return take_if_done(id, status, out_bytes);
    }

    // requests, p50 ms, p99 ms, mean batch, throughput GB/s of input floats,
    // span s (first arrival to last completion), all over completed requests
    void stats(double out[6])
    {
        std::lock_guard<std::mutex> g(mu_);
        for (int i = 0; i < 6; i++) out[i] = 0;
        if (lat_.empty()) return;
        std::vector<double> l = lat_;
        std::sort(l.begin(), l.end());
        auto pct = [&](double p) {  // linear interpolation between order statistics
            const double pos = p / 100.0 * (double)(l.size() - 1);
            const size_t lo = (size_t)pos, hi = std::min(lo + 1, l.size() - 1);
            return l[lo] + (l[hi] - l[lo]) * (pos - (double)lo);
        };
        double nb = 0;
        for (uint32_t b : batches_) nb += b;
        out[0] = (double)l.size();
        out[1] = pct(50) * 1e3;
        out[2] = pct(99) * 1e3;
        out[3] = batches_.empty() ? 0 : nb / (double)batches_.size();
        out[5] = t_last_ - t_first_;
        out[4] = out[5] > 0 ? (double)in_bytes_ / out[5] / 1e9 : 0;
    }

    // counted device memory now, and its peak (for tests)
    uint64_t in_use()
    {
        std::lock_guard<std::mutex> g(mu_);
        return in_use_;
    }
    uint64_t peak()
    {
        std::lock_guard<std::mutex> g(mu_);
        return peak_;
    }
    // times a worker released its scratch to admit a request; batches after
    // which a worker held more than estimated (should stay 0)
    uint64_t trims()
    {
        std::lock_guard<std::mutex> g(mu_);
        return trims_;
    }
    uint64_t overruns()
    {
        std::lock_guard<std::mutex> g(mu_);
        return over_;
    }

    // finishes every queued request, then joins the workers
    void stop()
    {
        {
            std::lock_guard<std::mutex> g(mu_);
            stopping_ = true;
            cv_work_.notify_all();
        }
        for (auto &t : threads_) t.join();
        threads_.clear();
        std::lock_guard<std::mutex> g(mu_);
        for (auto &kv : all_) delete kv.second;
        all_.clear();
    }

private:
    int take_if_done(uint64_t id, int *status, uint64_t *out_bytes)
    {
        auto it = all_.find(id);
        if (it == all_.end()) return -1;
        Request *r = it->second;
        if (!r->done) return 0;
        if (status) *status = r->status;
        if (out_bytes) *out_bytes = r->out_bytes;
        all_.erase(it);
        delete r;
        return 1;
    }

    // The oldest requests, as many as fit the budget and max_batch, for
    // worker i; *charged = the worker's resident bytes counted while they run
    // (the estimate).  Empty when stopping with nothing queued.
    std::vector<Request *> take_batch(void *w, size_t i, uint64_t *charged)
    {
        std::unique_lock<std::mutex> g(mu_);
        bool trimmed = false;  // released this worker's scratch since its last batch
        for (;;) {
            std::vector<Request *> b;
            uint64_t est = held_[i];
            while (!queue_.empty() && b.size() < max_batch_) {
                b.push_back(queue_.front());
                const uint64_t e = ex_->estimate(w, b);
                if (in_use_ - held_[i] + e > budget_) {
                    b.pop_back();
                    break;
                }
                est = e;
                queue_.pop_front();
            }
            if (!b.empty()) {
                in_use_ += est - held_[i];
                *charged = est;
                peak_ = std::max(peak_, in_use_);
                return b;
            }
            if (stopping_ && queue_.empty()) return b;
            if (!queue_.empty() && !trimmed && held_[i] > ex_->least(0)) {
                // blocked by memory: release this worker's scratch, then retry
                g.unlock();
                ex_->trim(w);
                const uint64_t now = ex_->resident(w);
                g.lock();
                in_use_ = in_use_ - held_[i] + now;
                held_[i] = now;
                trims_++;
                trimmed = true;
                cv_work_.notify_all();
                continue;
            }
            cv_work_.wait_for(g, std::chrono::milliseconds(50));
        }
    }

    void worker_loop(void *w, size_t i)
    {
        for (;;) {
            uint64_t charged = 0;
            std::vector<Request *> b = take_batch(w, i, &charged);
            if (b.empty()) break;
            const double t0 = now_s();
            for (Request *r : b) r->t_start = t0;
            ex_->run(w, b);
            const uint64_t now = ex_->resident(w);
            const double t1 = now_s();
            std::lock_guard<std::mutex> g(mu_);
            // count what the worker holds now (the estimate bounded it from above)
            in_use_ = in_use_ - charged + now;
            held_[i] = now;
            if (now > charged) over_++;
            peak_ = std::max(peak_, in_use_);
            batches_.push_back((uint32_t)b.size());
            for (Request *r : b) {
                r->t_done = t1;
                r->done = true;
                if (r->status == 0) {
                    lat_.push_back(t1 - r->t_arrive);
                    in_bytes_ += 4 * r->n;
                    if (t_first_ == 0 || r->t_arrive < t_first_) t_first_ = r->t_arrive;
                    t_last_ = std::max(t_last_, t1);
                }
            }
            cv_work_.notify_all();
            cv_done_.notify_all();
        }
        ex_->free_worker(w);
    }

    Executor *ex_;
    uint32_t nworkers_, max_batch_;
    uint64_t budget_;
    std::mutex mu_;
    std::condition_variable cv_work_, cv_done_;
    std::deque<Request *> queue_;
    std::unordered_map<uint64_t, Request *> all_;
    std::vector<std::thread> threads_;
    uint64_t next_id_ = 1, in_use_ = 0, in_bytes_ = 0, peak_ = 0, trims_ = 0, over_ = 0;
    std::vector<uint64_t> held_;  // resident bytes of every worker between batches
    bool stopping_ = false;
    std::vector<double> lat_;
    std::vector<uint32_t> batches_;
    double t_first_ = 0, t_last_ = 0;
};

}  // namespace gbsz_srv
