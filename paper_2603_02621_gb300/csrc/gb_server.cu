// gb_server.cu -- serving: a request loop with continuous batching over
// several GPU lanes (GoldbachGPU, arXiv 2603.02621: range verification,
// Sec. 2.3, and single-n checks, Sec. 2.4, served as a stream of requests).
//
// Ranges to verify enter one FIFO queue, single-n queries another.  Each
// range lane is a context sharing the base primes (gb_init_shared) with its
// own stream and arenas, driven by its own host thread: whenever a lane is
// free it admits the ranges at the head of the queue, as many as fit in the
// free part of the device-memory budget (at most max_batch), and runs them as
// one gb_verify_batch call.  Ranges that arrive while other lanes have work on
// the GPU are admitted by the next free lane, so their work overlaps on the
// device.  Queries take microseconds each and should not wait behind ranges:
// one more lane, on a stream of the highest priority, serves only them, every
// queued query as one gb_query_batch call.  A request's result does not
// depend on what it was batched with.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include "gb.h"
#include "gb_internal.cuh"

struct gb_server {
    struct Pending {
        uint64_t ticket;
        gb_request req;
        uint64_t bytes;
        double t_submit;
    };
    gb_ctx* parent = nullptr;
    std::vector<gb_ctx*> lanes;
    std::vector<cudaStream_t> streams;
    std::vector<std::thread> threads;
    uint64_t budget = 0;
    uint32_t max_batch = 0;
    uint64_t base_limit = 0;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

    std::mutex mu;
    std::condition_variable cv_work, cv_query, cv_done;
    std::deque<Pending> queue;      // ranges
    std::deque<Pending> qqueue;     // single-n queries
    std::unordered_map<uint64_t, gb_response> done;
    uint64_t next_ticket = 1;
    uint64_t in_flight = 0, in_flight_max = 0;
    uint64_t n_submitted = 0, n_done = 0, n_batches = 0;
    bool stop = false;

    double now_us() const
    {
        return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
    }
};

namespace {

// device bytes a request holds while it runs (the batch's q window share,
// histogram row, key and counters; a query's input and output)
uint64_t request_bytes(const gb_request& r, uint32_t p1)
{
    if (r.kind == GB_REQ_QUERY) return 16;
    const uint64_t n = (r.hi - r.lo) / 2;
    const uint64_t halo_words = (uint64_t)p1 / 128 + 4;
    return ((n + 63) / 64 + halo_words) * 8 + 4ull * 8192 + 64;
}

int check_request(const gb_server* s, const gb_request& r)
{
    if (r.kind == GB_REQ_QUERY) return ((r.lo & 1) || r.lo < 4 || r.lo >= (1ull << 63)) ? GB_EINVAL : GB_OK;
    if (r.kind != GB_REQ_RANGE) return GB_EINVAL;
    if ((r.lo & 1) || (r.hi & 1) || r.lo < 4 || r.hi <= r.lo || r.hi > GB_MAX_HI) return GB_EINVAL;
    if ((r.hi - r.lo) / 2 > (1ull << 32)) return GB_EINVAL;
    const double lim = (double)s->base_limit * (double)s->base_limit;
    if ((double)r.hi > lim) return GB_EINVAL;
    return GB_OK;
}

void post(gb_server* s, const std::vector<gb_server::Pending>& batch, int rc, double t_start,
          const std::vector<gb_segment_result>& recs, const std::vector<uint32_t>& pm)
{
    const double t_done = s->now_us();
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (size_t i = 0; i < batch.size(); ++i) {
            const gb_server::Pending& p = batch[i];
            gb_response r{};
            r.t_submit_us = p.t_submit;
            r.t_start_us = t_start;
            r.t_done_us = t_done;
            r.status = rc;
            if (p.req.kind == GB_REQ_RANGE) r.range = recs[i];
            else r.p_min = pm[i];
            s->done[p.ticket] = r;
            s->in_flight -= p.bytes;
        }
        s->n_done += batch.size();
    }
    s->cv_done.notify_all();
    s->cv_work.notify_all();
}

// with s->mu held: take the ticket's request out of its queue and post a
// GB_ECANCELED response; GB_EBUSY if it is no longer queued
int cancel_locked(gb_server* s, uint64_t ticket)
{
    for (std::deque<gb_server::Pending>* q : {&s->queue, &s->qqueue}) {
        for (auto it = q->begin(); it != q->end(); ++it) {
            if (it->ticket != ticket) continue;
            gb_response r{};
            r.status = GB_ECANCELED;
            r.t_submit_us = it->t_submit;
            r.t_start_us = r.t_done_us = s->now_us();
            if (it->req.kind == GB_REQ_RANGE) {
                r.range.lo = it->req.lo;
                r.range.hi = it->req.hi;
            }
            s->done[ticket] = r;
            s->n_done += 1;
            q->erase(it);
            return GB_OK;
        }
    }
    return GB_EBUSY;
}

// a range lane: admits ranges from the head of the queue within the budget
void range_loop(gb_server* s, size_t lane)
{
    gb_ctx* ctx = s->lanes[lane];
    std::vector<gb_server::Pending> batch;
    std::vector<uint64_t> lo, hi;
    std::vector<gb_segment_result> recs;
    const std::vector<uint32_t> none;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_work.wait(lk, [&] { return s->stop || !s->queue.empty(); });
            if (s->queue.empty()) return;                           // stopping and drained
            // the head of the queue while it fits the free budget (the first
            // request always, if nothing else is in flight)
            batch.clear();
            uint64_t held = 0;
            while (!s->queue.empty() && batch.size() < s->max_batch) {
                const gb_server::Pending& p = s->queue.front();
                const bool fits = s->in_flight + held + p.bytes <= s->budget;
                if (!fits && !(batch.empty() && s->in_flight == 0)) break;
                held += p.bytes;
                batch.push_back(p);
                s->queue.pop_front();
            }
            if (batch.empty()) {
                // everything queued waits for memory held by other lanes
                s->cv_done.wait(lk, [&] { return s->in_flight == 0 || s->queue.empty() ||
                                                 s->in_flight + s->queue.front().bytes <= s->budget; });
                continue;
            }
            s->in_flight += held;
            s->in_flight_max = std::max(s->in_flight_max, s->in_flight);
            s->n_batches += 1;
        }
        const double t_start = s->now_us();
        lo.clear();
        hi.clear();
        for (const auto& p : batch) {
            lo.push_back(p.req.lo);
            hi.push_back(p.req.hi);
        }
        recs.assign(lo.size(), gb_segment_result{});
        const int rc = gb_verify_batch(ctx, lo.data(), hi.data(), (uint32_t)lo.size(), 0, recs.data(), nullptr, 0);
        post(s, batch, rc, t_start, recs, none);
    }
}

// the query lane: every queued query (at most max_batch) as one batch
void query_loop(gb_server* s, size_t lane)
{
    gb_ctx* ctx = s->lanes[lane];
    std::vector<gb_server::Pending> batch;
    std::vector<uint64_t> qn;
    std::vector<uint32_t> pm;
    const std::vector<gb_segment_result> none;
    for (;;) {
        {
            std::unique_lock<std::mutex> lk(s->mu);
            s->cv_query.wait(lk, [&] { return s->stop || !s->qqueue.empty(); });
            if (s->qqueue.empty()) return;
            batch.clear();
            uint64_t held = 0;
            while (!s->qqueue.empty() && batch.size() < s->max_batch) {
                held += s->qqueue.front().bytes;
                batch.push_back(s->qqueue.front());
                s->qqueue.pop_front();
            }
            s->in_flight += held;
            s->in_flight_max = std::max(s->in_flight_max, s->in_flight);
            s->n_batches += 1;
        }
        const double t_start = s->now_us();
        qn.clear();
        for (const auto& p : batch) qn.push_back(p.req.lo);
        pm.assign(qn.size(), 0u);
        const int rc = gb_query_batch(ctx, qn.data(), (uint32_t)qn.size(), 0, pm.data());
        post(s, batch, rc, t_start, none, pm);
    }
}

}  // namespace

extern "C" int gb_server_create(gb_server** out, gb_ctx* ctx, uint32_t lanes, uint64_t hbm_budget_bytes,
                                uint32_t max_batch)
{
    if (!out || !ctx) return GB_EINVAL;
    *out = nullptr;
    if (lanes == 0 || lanes > 16) return GB_EINVAL;
    gb_config cfg{};
    int rc = gb_get_config(ctx, &cfg);
    if (rc) return rc;
    gb_server* s = new gb_server();
    s->parent = ctx;
    if (hbm_budget_bytes == 0) {
        // admission by free device memory: half of what is free now
        size_t free_b = 0, total_b = 0;
        cudaSetDevice(cfg.device);
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            cudaGetLastError();
            free_b = 16ull << 30;
        }
        hbm_budget_bytes = free_b / 2;
    }
    s->budget = hbm_budget_bytes;
    s->max_batch = max_batch ? max_batch : 256;
    s->base_limit = cfg.base_limit;
    cudaSetDevice(cfg.device);
    int prio_lo = 0, prio_hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi) != cudaSuccess) {
        cudaGetLastError();
        prio_lo = prio_hi = 0;
    }
    // lanes 0..lanes-1 verify ranges; lane `lanes` answers queries on a
    // stream of the highest priority
    for (uint32_t i = 0; i <= lanes; ++i) {
        cudaStream_t st = nullptr;
        gb_ctx* lc = nullptr;
        const int prio = i == lanes ? prio_hi : prio_lo;
        if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio) != cudaSuccess ||
            (rc = gb_init_shared(&lc, ctx, st)) != GB_OK) {
            if (st) cudaStreamDestroy(st);
            gb_server_destroy(s);
            return rc ? rc : GB_ECUDA;
        }
        s->streams.push_back(st);
        s->lanes.push_back(lc);
    }
    for (uint32_t i = 0; i < lanes; ++i) s->threads.emplace_back(range_loop, s, (size_t)i);
    s->threads.emplace_back(query_loop, s, (size_t)lanes);
    *out = s;
    return GB_OK;
}

extern "C" int gb_server_submit(gb_server* s, const gb_request* req, uint64_t* ticket)
{
    if (!s || !req || !ticket) return GB_EINVAL;
    const int rc = check_request(s, *req);
    if (rc) return rc;
    if (gb::fault_hit(GB_FAULT_SUBMIT)) return GB_EBUSY;            // refused at admission (injected)
    const bool cancel_now = gb::fault_hit(GB_FAULT_CANCEL);         // cancelled once queued (injected)
    gb_config cfg{};
    gb_get_config(s->lanes[0], &cfg);
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (s->stop) return GB_EBUSY;
        *ticket = s->next_ticket++;
        const gb_server::Pending p{*ticket, *req, request_bytes(*req, std::max(cfg.p1, cfg.p2)), s->now_us()};
        (req->kind == GB_REQ_QUERY ? s->qqueue : s->queue).push_back(p);
        s->n_submitted += 1;
        if (cancel_now) cancel_locked(s, *ticket);
    }
    if (cancel_now) s->cv_done.notify_all();
    if (req->kind == GB_REQ_QUERY) s->cv_query.notify_one();
    else s->cv_work.notify_one();
    return GB_OK;
}

extern "C" int gb_server_cancel(gb_server* s, uint64_t ticket)
{
    if (!s) return GB_EINVAL;
    int rc;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        if (ticket == 0 || ticket >= s->next_ticket) return GB_EINVAL;
        rc = cancel_locked(s, ticket);
    }
    if (rc == GB_OK) {
        s->cv_done.notify_all();
        s->cv_work.notify_all();
    }
    return rc;
}

extern "C" int gb_server_wait(gb_server* s, uint64_t ticket, gb_response* out, uint32_t timeout_ms)
{
    if (!s || !out) return GB_EINVAL;
    std::unique_lock<std::mutex> lk(s->mu);
    if (ticket == 0 || ticket >= s->next_ticket) return GB_EINVAL;
    const auto ready = [&] { return s->done.count(ticket) != 0; };
    if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
        return GB_ETIMEOUT;
    }
    *out = s->done[ticket];
    s->done.erase(ticket);
    return GB_OK;
}

extern "C" int gb_server_stats(gb_server* s, uint64_t* submitted, uint64_t* completed, uint64_t* batches,
                               uint64_t* in_flight_max)
{
    if (!s) return GB_EINVAL;
    std::lock_guard<std::mutex> lk(s->mu);
    if (submitted) *submitted = s->n_submitted;
    if (completed) *completed = s->n_done;
    if (batches) *batches = s->n_batches;
    if (in_flight_max) *in_flight_max = s->in_flight_max;
    return GB_OK;
}

extern "C" void gb_server_destroy(gb_server* s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    s->cv_query.notify_all();
    s->cv_done.notify_all();
    for (auto& t : s->threads) t.join();
    for (gb_ctx* c : s->lanes) gb_destroy(c);
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
}
