// Continuous-batching server (gd_serve_*): a host thread admits queued
// requests into free slots (each slot: a stream and its own work buffers),
// launches one persistent traversal per slot batch, and harvests finished
// slots while others are still running, so requests that arrive during a
// launch overlap with it on the device.  Admission is by an HBM footprint
// estimate against the slot's buffer budget.
#include <algorithm>
#include <atomic>
#include <chrono>
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

struct Slot {
    SlotBuffers b;
    bool busy = false;
    bool whole = false;  // launched on the whole GPU: no other slot starts meanwhile
    int kind = 0;
    std::vector<Request> reqs;
};

// Estimated device bytes of one query: its per-query records plus a front
// share that grows with the square root of the leaf counts (surface-contact
// fronts scale with the contact patch, not with the volume of pairs).
long long footprint(const gd_query& q) {
    long long ta = serve_mesh_tris(q.a), tb = serve_mesh_tris(q.b);
    double s = std::sqrt((double)ta) + std::sqrt((double)tb);
    return 1024 + (long long)(s * 64.0);
}

}  // namespace

struct gd_server {
    gd_ctx* ctx = nullptr;
    gd_serve_opts opts{};
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request> queue;
    std::unordered_map<uint64_t, gd_result> done;
    std::unordered_map<uint64_t, int> pending;
    long long queued_foot = 0;
    long long slot_budget = 0;
    uint64_t next_ticket = 1;
    int whole_grid = 0;  // co-resident CTAs of the whole GPU
    std::atomic<bool> stop{false};
    std::thread loop;
    gd_status loop_error = GD_OK;
};

namespace {

void free_slot(Slot& s) {
    SlotBuffers& b = s.b;
    if (b.stream) cudaStreamSynchronize(b.stream);
    cudaFree(b.front[0]); cudaFree(b.front[1]); cudaFree(b.leafq); cudaFree(b.cand); cudaFree(b.cand_d); cudaFree(b.cand_pts);
    cudaFree(b.qs); cudaFree(b.qin_dev); cudaFree(b.out_dev); cudaFree(b.mb_dev_ctr); cudaFree(b.stats_dev);
    cudaFree(b.rbox); cudaFree(b.jobs); cudaFree(b.slot_of);
    cudaFreeHost(b.qin_host); cudaFreeHost(b.out_host); cudaFreeHost(b.ctr_host);
    if (b.stream) cudaStreamDestroy(b.stream);
    b = SlotBuffers{};
}

bool alloc_slot(Slot& s, long long budget, long long max_batch, int grid) {
    SlotBuffers& b = s.b;
    // queue entries (16 B) for two fronts and the leaf queue, plus candidates (24 B)
    long long per = std::max<long long>(budget / (3 * 16 + 24 / 4), 1 << 16);
    b.cap_front = std::min<long long>(per, 0xffffffffll);
    b.cap_leaf = b.cap_front;
    b.cap_cand = std::max<long long>(b.cap_front / 4, 1 << 14);
    b.cap_q = max_batch;
    b.grid = grid;
    bool ok = cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaMalloc(&b.front[0], sizeof(Item) * b.cap_front) == cudaSuccess;
    ok = ok && cudaMalloc(&b.front[1], sizeof(Item) * b.cap_front) == cudaSuccess;
    ok = ok && cudaMalloc(&b.leafq, sizeof(Item) * b.cap_leaf) == cudaSuccess;
    ok = ok && cudaMalloc(&b.cand, sizeof(Cand) * b.cap_cand) == cudaSuccess;
    ok = ok && cudaMalloc(&b.cand_d, sizeof(double) * b.cap_cand) == cudaSuccess;
    ok = ok && cudaMalloc(&b.cand_pts, sizeof(double) * 6 * b.cap_cand) == cudaSuccess;
    ok = ok && cudaMalloc(&b.qs, sizeof(QState) * b.cap_q) == cudaSuccess;
    ok = ok && cudaMalloc(&b.qin_dev, sizeof(QIn) * b.cap_q) == cudaSuccess;
    ok = ok && cudaMalloc(&b.out_dev, sizeof(gd_result) * b.cap_q) == cudaSuccess;
    ok = ok && cudaMalloc(&b.mb_dev_ctr, sizeof(unsigned) * kCtrWords) == cudaSuccess;
    ok = ok && cudaMemset(b.mb_dev_ctr, 0, sizeof(unsigned) * kCtrWords) == cudaSuccess;
    ok = ok && cudaMalloc(&b.stats_dev, sizeof(StatsDev)) == cudaSuccess;
    ok = ok && cudaMallocHost(&b.qin_host, sizeof(QIn) * b.cap_q) == cudaSuccess;
    ok = ok && cudaMallocHost(&b.out_host, sizeof(gd_result) * b.cap_q) == cudaSuccess;
    ok = ok && cudaMallocHost(&b.ctr_host, sizeof(unsigned) * kCtrWords) == cudaSuccess;
    // refit slots (12 KB each) and root tables for up to 4096 roots per query
    b.cap_slots = 2048;
    b.cap_table = 4096ll * max_batch;
    ok = ok && cudaMalloc(&b.rbox, sizeof(float) * 6 * kRefitBoxes * (size_t)b.cap_slots) == cudaSuccess;
    ok = ok && cudaMalloc(&b.jobs, sizeof(uint2) * (size_t)b.cap_slots) == cudaSuccess;
    ok = ok && cudaMalloc(&b.slot_of, sizeof(unsigned) * (size_t)b.cap_table) == cudaSuccess;
    return ok;
}

void harvest(gd_server* S, Slot& s) {
    std::vector<std::pair<Request, gd_result>> redo;
    bool aborted = s.b.ctr_host[kCtrLastAbort] != 0;
    const bool bad = s.b.ctr_host[kCtrBadIndex] != 0;  // an internal index check failed
    {
        std::lock_guard<std::mutex> g(S->mu);
        for (size_t j = 0; j < s.reqs.size(); ++j) {
            gd_result r = s.b.out_host[j];
            if (aborted) r.status = GD_ERR_TIMEOUT;
            if (bad) r.status = GD_ERR_CUDA;
            // work beyond the slot's buffers, or a slot launch whose bounded
            // waits gave up: rerun alone below
            if (r.status == GD_ERR_OVERFLOW || r.status == GD_ERR_TIMEOUT) {
                redo.push_back({s.reqs[j], r});
                continue;
            }
            S->pending.erase(s.reqs[j].ticket);
            S->done[s.reqs[j].ticket] = r;
        }
    }
    // rerun alone on the context's own buffers, with the device otherwise idle
    // (this runs on the serving thread, so no slot is launched meanwhile)
    if (!redo.empty())
        for (Slot& o : S->slots)
            if (o.busy && &o != &s) cudaStreamSynchronize(o.b.stream);
    for (auto& pr : redo) {
        gd_result r{};
        gd_status st = serve_single(S->ctx, pr.first.q, &r);
        if (st != GD_OK) r.status = st;
        std::lock_guard<std::mutex> g(S->mu);
        S->pending.erase(pr.first.ticket);
        S->done[pr.first.ticket] = r;
    }
    s.reqs.clear();
    s.busy = false;
}

void run_loop(gd_server* S) {
    cudaSetDevice(serve_device(S->ctx));
    // the loop stays awake (yielding) this long after its last work, so that
    // a request arriving in a steady stream is not delayed by a thread wake-up
    const auto kStayAwake = std::chrono::milliseconds(20);
    auto last_work = std::chrono::steady_clock::now();
    for (;;) {
        bool worked = false;
        // harvest finished slots; a slot whose stream reports an error (the
        // context is unusable then) fails its requests instead of being
        // waited for forever
        for (Slot& s : S->slots) {
            if (!s.busy) continue;
            cudaError_t q = cudaStreamQuery(s.b.stream);
            if (q == cudaSuccess) {
                harvest(S, s);
                worked = true;
            } else if (q != cudaErrorNotReady) {
                std::lock_guard<std::mutex> g(S->mu);
                for (auto& r : s.reqs) {
                    gd_result res{};
                    res.status = GD_ERR_CUDA;
                    S->pending.erase(r.ticket);
                    S->done[r.ticket] = res;
                }
                s.reqs.clear();
                s.busy = false;
                S->loop_error = GD_ERR_CUDA;
                worked = true;
            }
        }
        // admit queued requests into free slots (none while a slot holds the
        // whole GPU)
        bool whole_busy = false;
        for (Slot& s : S->slots) whole_busy = whole_busy || (s.busy && s.whole);
        for (Slot& s : S->slots) {
            if (whole_busy) break;
            if (s.busy) continue;
            std::vector<Request> take;
            {
                std::unique_lock<std::mutex> g(S->mu);
                if (S->queue.empty()) break;
                if (S->opts.linger_us > 0 && (long long)S->queue.size() < S->opts.max_batch) {
                    // wait briefly for more requests to fill the batch
                    S->cv.wait_for(g, std::chrono::microseconds(S->opts.linger_us));
                    if (S->queue.empty()) break;
                }
                int kind = (int)S->queue.front().q.kind;
                long long foot = 0;
                for (auto it = S->queue.begin(); it != S->queue.end() && (long long)take.size() < S->opts.max_batch;) {
                    if ((int)it->q.kind != kind) { ++it; continue; }
                    if (!take.empty() && foot + it->foot > S->slot_budget) break;
                    foot += it->foot;
                    S->queued_foot -= it->foot;
                    take.push_back(*it);
                    it = S->queue.erase(it);
                }
            }
            if (take.empty()) break;
            std::vector<gd_query> qs(take.size());
            for (size_t j = 0; j < take.size(); ++j) qs[j] = take[j].q;
            int kind = (int)qs[0].kind;
            // a batch that finds the GPU idle and the queue empty gets the whole
            // GPU (the latency of a lone request is that of a plain query);
            // otherwise the slot's share, so that slots run side by side
            bool idle = true;
            for (Slot& o : S->slots) idle = idle && !o.busy;
            bool solo = false;
            if (idle) {
                std::lock_guard<std::mutex> g(S->mu);
                solo = S->queue.empty();
            }
            const int grid = solo ? S->whole_grid : s.b.grid;
            gd_status st = serve_launch_batch(S->ctx, s.b, qs.data(), (long long)qs.size(), kind, grid);
            if (st != GD_OK) {
                std::lock_guard<std::mutex> g(S->mu);
                for (auto& r : take) {
                    gd_result res{};
                    res.status = st;
                    S->pending.erase(r.ticket);
                    S->done[r.ticket] = res;
                }
                continue;
            }
            s.kind = kind;
            s.whole = solo;
            s.reqs = std::move(take);
            s.busy = true;
            worked = true;
            if (solo) break;
        }
        if (S->stop.load()) {
            bool idle = true;
            for (Slot& s : S->slots) idle = idle && !s.busy;
            std::lock_guard<std::mutex> g(S->mu);
            if (idle && S->queue.empty()) break;
        }
        const auto now = std::chrono::steady_clock::now();
        if (worked) last_work = now;
        if (!worked) {
            std::unique_lock<std::mutex> g(S->mu);
            bool any_busy = false;
            for (Slot& s : S->slots) any_busy = any_busy || s.busy;
            if (S->queue.empty() && !any_busy && !S->stop.load() && now - last_work > kStayAwake) {
                S->cv.wait_for(g, std::chrono::milliseconds(2));
            } else {
                g.unlock();
                std::this_thread::yield();
            }
        }
    }
}

}  // namespace

extern "C" {

GD_API gd_status gd_serve_start(gd_ctx* ctx, const gd_serve_opts* opts, gd_server** out) {
    if (!ctx || !out) return GD_ERR_INVALID_ARG;
    *out = nullptr;
    gd_serve_opts o{};
    // measured on a 64-mesh pool at saturation: 2 slots of 16 queries gave
    // 9.2 K q/s; 4 x 256 gave 5.2 K, 2 x 1024 6.2 K (a launch lasts as long
    // as its slowest query, so small batches keep the slots turning over)
    o.slots = 2;
    o.max_batch = 16;
    o.memory_budget = 8ll << 30;
    o.linger_us = 0;
    if (opts) {
        if (opts->slots > 0) o.slots = std::min(opts->slots, 64);
        if (opts->max_batch > 0) o.max_batch = opts->max_batch;
        if (opts->memory_budget > 0) o.memory_budget = opts->memory_budget;
        if (opts->linger_us > 0) o.linger_us = opts->linger_us;
    }
    cudaSetDevice(serve_device(ctx));
    // make sure the context's own buffers exist for oversized requests
    gd_server* S = new gd_server();
    S->ctx = ctx;
    S->opts = o;
    S->slot_budget = o.memory_budget / o.slots;
    // Every slot's cooperative grid must stay resident while the other slots
    // run theirs.  The CTAs of a grid are spread over the GPU's partitions, so
    // an exact split of the full capacity can leave one partition
    // over-subscribed (a 3-way split, 3 x 101 CTAs, was seen to leave a grid
    // partly unscheduled until its bounded barrier wait gave up): the slots
    // share 90% of the capacity, in grids of a multiple of 16 CTAs.
    int occ = std::max(1, std::min(query_max_blocks_per_sm(0), query_max_blocks_per_sm(1)));
    int cap = occ * serve_sms(ctx);
    int per = cap;
    if (o.slots > 1) {
        per = (cap * 9 / 10) / o.slots;
        per -= per % 16;
        if (per < 16) per = std::min(16, cap);
    }
    S->whole_grid = cap;
    S->slots.resize(o.slots);
    for (Slot& s : S->slots) {
        if (!alloc_slot(s, S->slot_budget, o.max_batch, per)) {
            for (Slot& t : S->slots) free_slot(t);
            delete S;
            return GD_ERR_OOM;
        }
    }
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
        long long cap = S->slot_budget * (long long)S->slots.size();
        const long long qmax = std::max(4096ll, 16ll * S->opts.max_batch * (long long)S->slots.size());
        if ((long long)S->queue.size() >= qmax || S->queued_foot + r.foot > cap)
            return GD_ERR_BUSY;
        r.ticket = S->next_ticket++;
        S->queued_foot += r.foot;
        S->queue.push_back(r);
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
    for (Slot& s : S->slots) free_slot(s);
    delete S;
    return GD_OK;
}

}  // extern "C"
