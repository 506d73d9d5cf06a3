// Continuous-batching server (gd_serve_*).  One execution lane: a host thread
// takes every queued request of the head request's kind (up to max_batch,
// within the memory budget) and runs them as one persistent launch on the
// whole GPU, on a private execution context with buffers sized from the
// budget; requests that arrive meanwhile are admitted into the next launch
// as soon as this one ends.  One request alone runs as a single query (the
// same launch as gd_min_distance / gd_max_distance); a batch's queries are
// read by the kernel from pinned memory and its results written back there,
// so neither path copies or synchronises on the way.
//
// Only one cooperative grid is ever in flight: CUDA does not promise that
// cooperative grids launched on different streams are resident together, and
// a grid whose CTAs wait at a grid barrier for CTAs that cannot be scheduled
// can only time out.
//
// Admission is by HBM footprint: each request holds a predicted number of
// work-buffer bytes (footprint(), a model of the measured front, leaf-pair
// and candidate peaks of single queries) from submission until its result is
// published; a submission that would take the held bytes beyond the budget
// is refused with GD_ERR_BUSY, and a batch holds at most a budget's worth.
// A request whose work outgrows its share of the lane's buffers anyway is run
// again alone, where the buffers grow as far as it needs.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "gd_launch.h"
#include "gd_serve.h"

using namespace gd;

namespace {

struct Request {
    uint64_t ticket;
    gd_query q;
    long long foot;
};

// Predicted work-buffer bytes of one query: 16 B per front entry in each of
// the two front buffers at the largest level, 16 B per leaf pair, 72 B per
// float64 candidate (record, distance, witness points), plus 1 KB of
// per-query records.  The counts are power laws c s^p in s = sqrt(T_A) +
// sqrt(T_B) (a surface-contact front grows with the contact patch, not with
// T_A T_B).  Fitted to 800 single queries on the 64-mesh serving pool (random
// pairs and placements, one in four a max query; largest front, leaf pairs
// and candidates from gd_stats): p by least squares in log-log, c the 99th
// percentile of the residuals, so that 99% of those queries lie below each
// curve (the largest query measured needed 438 MB).
long long footprint(const gd_query& q) {
    const double ta = (double)serve_mesh_tris(q.a), tb = (double)serve_mesh_tris(q.b);
    const double sq = std::sqrt(ta) + std::sqrt(tb);
    const double front = 349.0 * std::pow(sq, 1.223);
    const double leaf = 71.5 * std::pow(sq, 1.514);
    const double cand = 570.0 * std::pow(sq, 0.642);
    const double bytes = 16.0 * (2.0 * front + leaf) + 72.0 * cand + 1024.0;
    return (long long)std::ceil(bytes);
}

}  // namespace

struct gd_server {
    gd_ctx* ctx = nullptr;   // the user's context (validation of submissions)
    gd_ctx* exec = nullptr;  // private execution context: stream, buffers, pinned records
    gd_serve_opts opts{};
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> queue;
    std::atomic<long long> queued{0};  // queue length, read without the lock by the loop
    std::unordered_map<uint64_t, gd_result> done;
    std::unordered_map<uint64_t, int> pending;
    long long held_foot = 0;  // predicted bytes of queued and running requests
    uint64_t next_ticket = 1;
    std::atomic<bool> stop{false};
    std::thread loop;
};

namespace {

// Run one batch (all of one kind) on the lane; results land in res.
void run_batch(gd_server* S, const std::vector<Request>& take, std::vector<gd_result>& res) {
    const size_t m = take.size();
    res.assign(m, gd_result{});
    if (m == 1) {
        gd_status st = serve_single(S->exec, take[0].q, &res[0]);
        if (st != GD_OK) res[0].status = st;
        return;
    }
    std::vector<gd_query> qs(m);
    for (size_t j = 0; j < m; ++j) qs[j] = take[j].q;
    gd_status st = serve_batch(S->exec, qs.data(), (long long)m, (int)qs[0].kind, res.data());
    if (st == GD_ERR_TIMEOUT) {
        // a bounded device wait gave up: each query runs again alone below
        for (gd_result& r : res) { r = gd_result{}; r.status = GD_ERR_TIMEOUT; }
    } else if (st != GD_OK) {
        for (gd_result& r : res) { r = gd_result{}; r.status = st; }
        return;
    }
    // a query that outgrew its share of the queues (or a launch whose
    // bounded waits gave up) runs again alone, with buffers grown for it
    for (size_t j = 0; j < m; ++j) {
        if (res[j].status != GD_ERR_OVERFLOW && res[j].status != GD_ERR_TIMEOUT) continue;
        gd_result r{};
        gd_status s1 = serve_single(S->exec, take[j].q, &r);
        if (s1 != GD_OK) r.status = s1;
        res[j] = r;
    }
}

constexpr long long kBatchFrom = 8;
constexpr int kPipeline = 2;  // single-query launches in flight on the lane

struct InFlight {
    Request req;
    int slot;
    unsigned long long seq;
};

void publish(gd_server* S, const Request& r, const gd_result& res) {
    std::lock_guard<std::mutex> g(S->mu);
    S->pending.erase(r.ticket);
    S->done[r.ticket] = res;
    S->held_foot -= r.foot;
}

void run_loop(gd_server* S) {
    cudaSetDevice(serve_device(S->ctx));
    // the loop stays awake (yielding) this long after its last work, so that
    // a request arriving in a steady stream is not delayed by a thread wake-up
    const auto kStayAwake = std::chrono::milliseconds(20);
    auto last_work = std::chrono::steady_clock::now();
    std::vector<Request> take;
    std::vector<gd_result> res;
    std::deque<InFlight> fl;  // pipelined single queries, oldest first
    int next_slot = 0;
    for (;;) {
        bool worked = false;
        // collect the oldest single query once its record is stamped
        if (!fl.empty() && serve_single_ready(S->exec, fl.front().slot, fl.front().seq)) {
            gd_result r{};
            const InFlight f = fl.front();
            fl.pop_front();
            gd_status st = serve_single_finish(S->exec, f.req.q, f.slot, f.seq, &r);
            if (st != GD_OK && r.status == GD_OK) r.status = st;
            publish(S, f.req, r);
            worked = true;
        }
        take.clear();
        bool batch = false;
        if (S->queued.load(std::memory_order_acquire) > 0 && (long long)fl.size() < kPipeline) {
            std::unique_lock<std::mutex> g(S->mu);
            if (S->opts.linger_us > 0 && fl.empty() && (long long)S->queue.size() < S->opts.max_batch &&
                !S->stop.load()) {
                // wait (once) for more requests to fill the batch
                S->cv.wait_for(g, std::chrono::microseconds(S->opts.linger_us),
                               [&] { return (long long)S->queue.size() >= S->opts.max_batch || S->stop.load(); });
            }
            // a short queue runs one request at a time as a single query (the
            // single-query launch has the background probes, the CTA-shared
            // bound and the one-warp setup that a batch launch lacks, so the
            // heaviest requests, which set the tail, run fastest alone), with
            // the next one already launched behind it on the stream; from
            // kBatchFrom waiting requests on, a batch's throughput pays for
            // that (a batch starts once the pipelined launches are collected)
            batch = (long long)S->queue.size() >= kBatchFrom;
            if (!S->queue.empty() && (!batch || fl.empty())) {
                const gd_kind kind = S->queue.front().q.kind;
                const long long cap = batch ? S->opts.max_batch : 1;
                long long foot = 0;
                for (auto it = S->queue.begin(); it != S->queue.end() && (long long)take.size() < cap;) {
                    if (it->q.kind != kind) { ++it; continue; }
                    if (!take.empty() && foot + it->foot > S->opts.memory_budget) break;
                    foot += it->foot;
                    take.push_back(*it);
                    it = S->queue.erase(it);
                }
                S->queued.store((long long)S->queue.size(), std::memory_order_release);
            }
        }
        if (take.size() == 1 && !batch) {
            InFlight f{take[0], next_slot, 0ull};
            gd_status st = serve_single_launch(S->exec, f.req.q, f.slot, &f.seq);
            if (st == GD_OK) {
                fl.push_back(f);
                next_slot = (next_slot + 1) % kPipeline;
            } else {
                gd_result r{};
                r.status = st;
                publish(S, f.req, r);
            }
            worked = true;
        } else if (!take.empty()) {
            run_batch(S, take, res);
            for (size_t j = 0; j < take.size(); ++j) publish(S, take[j], res[j]);
            worked = true;
        }
        if (worked) {
            last_work = std::chrono::steady_clock::now();
            continue;
        }
        if (!fl.empty()) continue;  // wait for the stamp
        if (S->stop.load()) {
            std::lock_guard<std::mutex> g(S->mu);
            if (S->queue.empty()) break;
            continue;
        }
        if (std::chrono::steady_clock::now() - last_work > kStayAwake) {
            std::unique_lock<std::mutex> g(S->mu);
            S->cv.wait_for(g, std::chrono::milliseconds(2), [&] { return !S->queue.empty() || S->stop.load(); });
        } else {
            std::this_thread::yield();
        }
    }
}

}  // namespace

extern "C" {

GD_API gd_status gd_query_footprint(const gd_query* q, int64_t* bytes) {
    if (!q || !bytes || !q->a || !q->b) return GD_ERR_INVALID_ARG;
    *bytes = footprint(*q);
    return GD_OK;
}

GD_API gd_status gd_serve_start(gd_ctx* ctx, const gd_serve_opts* opts, gd_server** out) {
    if (!ctx || !out) return GD_ERR_INVALID_ARG;
    *out = nullptr;
    gd_serve_opts o{};
    o.slots = 1;
    o.max_batch = 16;
    o.memory_budget = 8ll << 30;
    o.linger_us = 0;
    if (opts) {
        if (opts->max_batch > 0) o.max_batch = opts->max_batch;
        if (opts->memory_budget > 0) o.memory_budget = opts->memory_budget;
        if (opts->linger_us > 0) o.linger_us = opts->linger_us;
    }
    const int device = serve_device(ctx);
    gd_ctx* exec = nullptr;
    gd_status s = gd_ctx_create(device, &exec);
    if (s != GD_OK) return s;
    // the lane's work buffers come out of the budget: two fronts and the leaf
    // queue of n entries (16 B each) and n / 4 candidates (72 B each)
    gd_tunables t = serve_tunables(ctx);
    const long long n = std::max<long long>(o.memory_budget / (3 * 16 + 72 / 4), 1 << 16);
    t.front_capacity = n;
    t.leaf_capacity = n;
    t.cand_capacity = std::max<long long>(n / 4, 1 << 14);
    t.max_capacity = std::max<long long>(t.max_capacity, n);
    t.batch_budget = 0;
    s = gd_ctx_set_tunables(exec, &t);
    if (s == GD_OK) s = serve_prepare(exec, o.max_batch);
    if (s != GD_OK) {
        gd_ctx_destroy(exec);
        return s;
    }
    gd_server* S = new gd_server();
    S->ctx = ctx;
    S->exec = exec;
    S->opts = o;
    S->loop = std::thread(run_loop, S);
    *out = S;
    return GD_OK;
}

GD_API gd_status gd_serve_submit(gd_server* S, const gd_query* q, uint64_t* ticket) {
    if (!S || !q || !ticket) return GD_ERR_INVALID_ARG;
    std::string why;
    if (!serve_query_ok(S->ctx, *q, &why)) return GD_ERR_INVALID_ARG;
    Request r;
    r.q = *q;
    r.foot = footprint(*q);
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->stop.load()) return GD_ERR_BUSY;
        const long long qmax = std::max(4096ll, 16ll * S->opts.max_batch);
        // a request larger than the whole budget is admitted only onto an
        // empty lane (it then runs alone, its buffers grown for it)
        const bool fits = S->held_foot + r.foot <= S->opts.memory_budget || S->held_foot == 0;
        if ((long long)S->queue.size() >= qmax || !fits) return GD_ERR_BUSY;
        r.ticket = S->next_ticket++;
        S->held_foot += r.foot;
        S->queue.push_back(r);
        S->queued.store((long long)S->queue.size(), std::memory_order_release);
        S->pending[r.ticket] = 1;
    }
    S->cv.notify_all();
    *ticket = r.ticket;
    return GD_OK;
}

GD_API gd_status gd_serve_poll(gd_server* S, uint64_t ticket, gd_result* out) {
    if (!S || !out) return GD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->done.find(ticket);
    if (it != S->done.end()) {
        *out = it->second;
        S->done.erase(it);
        return GD_OK;
    }
    if (S->pending.count(ticket)) return GD_ERR_NOT_READY;
    return GD_ERR_INVALID_ARG;
}

GD_API gd_status gd_serve_drain(gd_server* S, uint64_t* tickets, gd_result* out, int64_t max, int64_t* n) {
    if (!S || !n || max < 0 || (max > 0 && (!tickets || !out))) return GD_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(S->mu);
    int64_t k = 0;
    for (auto it = S->done.begin(); it != S->done.end() && k < max;) {
        tickets[k] = it->first;
        out[k] = it->second;
        ++k;
        it = S->done.erase(it);
    }
    *n = k;
    return GD_OK;
}

GD_API gd_status gd_serve_stop(gd_server* S) {
    if (!S) return GD_ERR_INVALID_ARG;
    S->stop.store(true);
    S->cv.notify_all();
    if (S->loop.joinable()) S->loop.join();
    gd_ctx_destroy(S->exec);
    delete S;
    return GD_OK;
}

}  // extern "C"
