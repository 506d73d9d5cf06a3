// C ABI of the engine (include/gdist.h): contexts, meshes, synchronous,
// device-resident and batched queries.  Host code only validates, sizes
// buffers and launches; every step of the computation runs in the kernels of
// gd_build.cu and gd_query.cu.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstddef>
#include <cstring>
#include <string>
#include <vector>

#include "gd_internal.cuh"
#include "gd_launch.h"
#include "gd_serve.h"

using namespace gd;

// A single query's result and counters come back after every query (the
// first kResultBytes); its statistics only when gd_get_stats asks.
// single-query launches the server keeps in flight on its stream
constexpr int kPipe = 2;

struct Mailbox {
    gd_result out;
    unsigned ctr[kCtrWords];
    StatsDev stats;
};
constexpr size_t kResultBytes = offsetof(Mailbox, stats);

struct gd_mesh {
    gd_ctx* ctx = nullptr;
    long long nv = 0, nt = 0;
    int L = 0;
    float* d_verts = nullptr;
    int32_t* d_tris = nullptr;
    float* d_box = nullptr;
    float4* d_tri = nullptr;
    unsigned* d_order = nullptr;  // original index of each sorted triangle (leaf order)
    int32_t* d_stris = nullptr;   // vertex indices of each sorted triangle (leaf order), for refits
    MeshDev* d_desc = nullptr;
    MeshDev h_desc{};
    unsigned* d_flags = nullptr;  // validation flags of gd_mesh_update
    bool tree = false;            // box, tri and L hold a sorted tree (refit may run)
    bool built = false;           // ... and its boxes bound the current vertices
    float build_ms = 0.f;         // device time of the last build's kernels
};

struct gd_ctx {
    int device = 0;
    int sms = 0;
    cudaStream_t stream = nullptr;
    std::string err;
    gd_tunables tun{};
    // work buffers
    bool ready = false;
    Item* front[2] = {nullptr, nullptr};
    Item* leafq = nullptr;
    Cand* cand = nullptr;
    double* cand_d = nullptr;
    double* cand_pts = nullptr;
    long long cap_front = 0, cap_leaf = 0, cap_cand = 0;
    Mailbox* mb_dev = nullptr;   // single-query results, stats and counters
    Mailbox* mb_host = nullptr;  // pinned mirror
    HostDone* hd = nullptr;      // pinned result records, written by the kernel: [0] for the
                                 // synchronous calls, [1..kPipe] for the server's pipelined launches
    unsigned long long hd_seq = 0;
    QState* qs = nullptr;
    QIn* qin_dev = nullptr;
    QIn* qin_host = nullptr;
    gd_result* out_dev = nullptr;
    gd_result* out_host = nullptr;
    unsigned long long* done_dev = nullptr;   // per-query completion stamps of a launch
    unsigned long long* done_host = nullptr;  // pinned mirror
    long long cap_q = 0;
    // completion of each query of the last gd_batch_query, device ns since
    // the start of the call's first launch
    std::vector<long long> batch_done;
    unsigned long long batch_t0 = 0;
    bool in_batch = false;
    float* rbox = nullptr;        // refit slots
    uint2* jobs = nullptr;
    long long cap_slots = 0;
    unsigned* slot_of = nullptr;  // refit-root tables
    long long cap_table = 0;
    float* ftree = nullptr;       // refit mode 3: B's whole tree in A's frame
    long long cap_ftree = 0;      // ... its capacity in nodes
    unsigned long long* naive_ws = nullptr;  // scratch of the naive comparator
    unsigned long long* point_ws = nullptr;  // counters of point queries
    double* pts_dev = nullptr;               // staged host points and results
    gd_point_result* pres_dev = nullptr;
    long long cap_pts = 0;
    unsigned long long* pkeys[2] = {nullptr, nullptr};  // Morton ordering of the points
    unsigned* pvals[2] = {nullptr, nullptr};
    unsigned* phist = nullptr;
    long long cap_psort = 0;
    unsigned long long last_point_tests = 0, last_point_exact = 0;  // counters of the last point call
    gd_stats last{};
    bool stats_pending = false;  // last run was device-resident: stats still on the device
    unsigned ws_gen = 0;         // bumped whenever the work buffers or tunables change
    unsigned pending_retries = 0;  // growth retries of the query whose stats are pending
    int last_grid = 0;
};

namespace {

gd_status fail(gd_ctx* ctx, gd_status s, const std::string& msg) {
    if (ctx) ctx->err = msg;
    return s;
}

gd_status cuda_fail(gd_ctx* ctx, cudaError_t e, const char* where) {
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(ctx, GD_ERR_OOM, m);
    return fail(ctx, GD_ERR_CUDA, m);
}

#define GD_CUDA(ctx, call)                                         \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
    } while (0)

bool xform_ok(const double* x, std::string* why) {
    for (int i = 0; i < 12; ++i)
        if (!std::isfinite(x[i])) { *why = "transform has a non-finite entry"; return false; }
    double worst = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = x[i] * x[j] + x[4 + i] * x[4 + j] + x[8 + i] * x[8 + j];
            worst = std::max(worst, std::fabs(s - (i == j ? 1.0 : 0.0)));
        }
    if (worst > 1e-9) { *why = "transform rotation is not orthonormal within 1e-9"; return false; }
    return true;
}

void free_ws(gd_ctx* c) {
    cudaFree(c->front[0]); cudaFree(c->front[1]); cudaFree(c->leafq);
    cudaFree(c->cand); cudaFree(c->cand_d); cudaFree(c->cand_pts);
    cudaFree(c->rbox); cudaFree(c->jobs);
    c->front[0] = c->front[1] = c->leafq = nullptr;
    c->cand = nullptr; c->cand_d = nullptr; c->cand_pts = nullptr;
    c->rbox = nullptr; c->jobs = nullptr;
    c->ready = false;
}

// entries of the refit-root table a query needs (0 when refit is off)
long long table_entries(const gd_ctx* c, const gd_mesh* B) {
    if (c->tun.refit_mode != 1) return 0;
    int dR = B->L > kRefitH ? B->L - kRefitH : 0;
    return 1ll << dR;
}

gd_status ensure_table(gd_ctx* c, long long n) {
    if (n <= c->cap_table) return GD_OK;
    cudaFree(c->slot_of);
    c->slot_of = nullptr;
    c->cap_table = 0;
    long long cap = std::max<long long>(n, 1 << 16);
    GD_CUDA(c, cudaMalloc(&c->slot_of, sizeof(unsigned) * cap));
    c->cap_table = cap;
    return GD_OK;
}

// Refit mode 3 (single queries): B's whole tree is refit into A's frame at
// the start of every launch, into this buffer (grown to B's node count).
gd_status full_refit_tree(gd_ctx* c, const gd_mesh* B, KArgs& a) {
    a.ftree = nullptr;
    if (c->tun.refit_mode != 3) return GD_OK;
    const long long nodes = 2ll << B->L;
    if (nodes > c->cap_ftree) {
        cudaFree(c->ftree);
        c->ftree = nullptr;
        c->cap_ftree = 0;
        GD_CUDA(c, cudaMalloc(&c->ftree, sizeof(float) * 6 * nodes));
        c->cap_ftree = nodes;
        ++c->ws_gen;
    }
    a.ftree = c->ftree;
    return GD_OK;
}

gd_status alloc_queues(gd_ctx* c) {
    free_ws(c);
    GD_CUDA(c, cudaMalloc(&c->front[0], sizeof(Item) * c->cap_front));
    GD_CUDA(c, cudaMalloc(&c->front[1], sizeof(Item) * c->cap_front));
    GD_CUDA(c, cudaMalloc(&c->leafq, sizeof(Item) * c->cap_leaf));
    GD_CUDA(c, cudaMalloc(&c->cand, sizeof(Cand) * c->cap_cand));
    GD_CUDA(c, cudaMalloc(&c->cand_d, sizeof(double) * c->cap_cand));
    GD_CUDA(c, cudaMalloc(&c->cand_pts, sizeof(double) * 6 * c->cap_cand));
    c->cap_slots = std::max(1, c->tun.refit_slots);
    GD_CUDA(c, cudaMalloc(&c->rbox, sizeof(float) * 6 * kRefitBoxes * (size_t)c->cap_slots));
    GD_CUDA(c, cudaMalloc(&c->jobs, sizeof(uint2) * (size_t)c->cap_slots));
    c->ready = true;
    ++c->ws_gen;
    return GD_OK;
}

gd_status ensure_ws(gd_ctx* c, long long nq) {
    if (!c->mb_dev) {
        GD_CUDA(c, cudaMalloc(&c->mb_dev, sizeof(Mailbox)));
        GD_CUDA(c, cudaMemset(c->mb_dev, 0, sizeof(Mailbox)));
        GD_CUDA(c, cudaMallocHost(&c->mb_host, sizeof(Mailbox)));
        GD_CUDA(c, cudaMallocHost(&c->hd, sizeof(HostDone) * (1 + kPipe)));
        std::memset(c->hd, 0, sizeof(HostDone) * (1 + kPipe));
    }
    if (!c->ready) {
        c->cap_front = std::min<long long>(c->tun.front_capacity, 0xffffffffll);
        c->cap_leaf = std::min<long long>(c->tun.leaf_capacity, 0xffffffffll);
        c->cap_cand = std::min<long long>(c->tun.cand_capacity, 0xffffffffll);
        gd_status s = alloc_queues(c);
        if (s != GD_OK) return s;
    }
    if (nq > c->cap_q) {
        long long cap = std::max<long long>(nq, 2 * c->cap_q);
        cudaFree(c->qs); cudaFree(c->qin_dev); cudaFree(c->out_dev); cudaFree(c->done_dev);
        cudaFreeHost(c->qin_host); cudaFreeHost(c->out_host); cudaFreeHost(c->done_host);
        c->qs = nullptr; c->qin_dev = nullptr; c->out_dev = nullptr; c->qin_host = nullptr; c->out_host = nullptr;
        c->done_dev = nullptr; c->done_host = nullptr;
        c->cap_q = 0;
        GD_CUDA(c, cudaMalloc(&c->qs, sizeof(QState) * cap));
        GD_CUDA(c, cudaMalloc(&c->qin_dev, sizeof(QIn) * cap));
        GD_CUDA(c, cudaMalloc(&c->out_dev, sizeof(gd_result) * cap));
        GD_CUDA(c, cudaMalloc(&c->done_dev, sizeof(unsigned long long) * cap));
        GD_CUDA(c, cudaMallocHost(&c->qin_host, sizeof(QIn) * cap));
        GD_CUDA(c, cudaMallocHost(&c->out_host, sizeof(gd_result) * cap));
        GD_CUDA(c, cudaMallocHost(&c->done_host, sizeof(unsigned long long) * cap));
        c->cap_q = cap;
    }
    return GD_OK;
}

// grow every queue by 4x (bounded by max_capacity); false if already at the limit
bool grow(gd_ctx* c) {
    long long lim = std::min<long long>(c->tun.max_capacity, 0xffffffffll);
    long long f = std::min(lim, c->cap_front * 4), l = std::min(lim, c->cap_leaf * 4),
              k = std::min(lim, c->cap_cand * 4);
    if (f == c->cap_front && l == c->cap_leaf && k == c->cap_cand) return false;
    c->cap_front = f; c->cap_leaf = l; c->cap_cand = k;
    return alloc_queues(c) == GD_OK;
}

// Entries one query of an m-query batch may push per level: every query at
// its limit fills a front buffer, or half the leaf queue (the traversal
// empties the leaf queue once it is half full).
// Per-level limits of a batch of m queries: each query's guaranteed share
// (half of an even split of the room for one level's pushes: the front, or
// the half of the leaf queue that a level may fill) and the common pool, the
// rest of that room, from which queries that outgrow their share draw.
void batch_limits(long long cap_front, long long cap_leaf, long long m, unsigned* share, unsigned* pool) {
    *share = 0u;
    *pool = 0u;
    if (m < 2) return;
    const long long room = std::min(cap_front, cap_leaf / 2);
    const long long b = std::max(1ll, std::min(room / m / 2, 0xffffffffll));
    *share = (unsigned)b;
    *pool = (unsigned)std::max(0ll, std::min(room - m * b, 0xffffffffll));
}

// Queues of a batch of m queries: room for share entries per query and
// level, within max_capacity (they only grow).
gd_status size_for_batch(gd_ctx* c, long long m, long long share) {
    if (m < 2) return GD_OK;
    const long long lim = std::min<long long>(c->tun.max_capacity, 0xffffffffll);
    long long want = std::min(lim, 2 * m * std::max<long long>(1, share));
    long long p = 1;
    while (p < want) p <<= 1;
    want = std::min(lim, p);
    if (c->cap_front >= want && c->cap_leaf >= want) return GD_OK;
    c->cap_front = std::max(c->cap_front, want);
    c->cap_leaf = std::max(c->cap_leaf, want);
    gd_status s = alloc_queues(c);
    if (s != GD_OK) {
        // fall back to the configured sizes; the batch then evicts more
        c->ready = false;
        return ensure_ws(c, m);
    }
    return GD_OK;
}

// Whether phase 0 of a single query may push its root pair itself: only when
// the root needs no refit claim (refit off, or B deeper than one refit tree).
int single_fuse_root(const gd_ctx* c, const gd_mesh* B) {
    return (c->tun.refit_mode != 1 || B->L > kRefitH) ? 1 : 0;
}

// CTAs of a single-query launch that run the traversal: the others (one per
// 8 probes, at most 1/8 of the grid) run the greedy probes in the background.
unsigned single_work_ctas(const gd_ctx* c, int grid) {
    if (c->tun.probes <= 1 || grid < 16) return (unsigned)grid;
    const int bg = std::min(grid / 8, (c->tun.probes + 7) / 8);
    return (unsigned)(grid - bg);
}

int grid_blocks(gd_ctx* c, int kind, bool batch = false) {
    int occ = query_max_blocks_per_sm(kind, batch);
    int b = c->tun.blocks_per_sm > 0 ? std::min(c->tun.blocks_per_sm, occ) : occ;
    if (b < 1) b = 1;
    return b * c->sms;
}

// The launch fields that follow from the context's tunables.
void fill_tunables(const gd_ctx* c, KArgs& a) {
    a.work_target = c->tun.work_target;
    a.k_max = c->tun.k_max;
    a.timeout_ns = c->tun.timeout_ns;
    a.refit = c->tun.refit_mode == 1 ? 1 : 0;
    a.conventional = c->tun.bounds_mode == 2 ? 1 : 0;
    a.probes = c->tun.probes;
}

void fill_common(gd_ctx* c, KArgs& a, unsigned* ctr, StatsDev* stats) {
    a.qs = c->qs;
    a.front0 = c->front[0];
    a.front1 = c->front[1];
    a.cap_front = (unsigned)c->cap_front;
    a.leafq = c->leafq;
    a.cap_leaf = (unsigned)c->cap_leaf;
    a.cand = c->cand;
    a.cand_d = c->cand_d;
    a.cand_pts = c->cand_pts;
    a.cap_cand = (unsigned)c->cap_cand;
    a.ctr = ctr;
    a.stats = stats;
    a.rbox = c->rbox;
    a.jobs = c->jobs;
    a.cap_slots = (unsigned)c->cap_slots;
    a.slot_of = c->slot_of;
    fill_tunables(c, a);
    a.n_slot_of = 0;
}

void to_stats(const StatsDev& s, unsigned blocks, unsigned retries, gd_stats* o) {
    std::memset(o, 0, sizeof(*o));
    o->levels = s.levels;
    for (int i = 0; i < 32; ++i) { o->front[i] = s.front[i]; o->slots[i] = s.slots[i]; }
    o->pairs_tested = 0;
    o->alg_bytes = 0;
    o->tri_pairs = 0;
    o->refined = 0;
    for (int i = 0; i < kAccWays; ++i) {
        o->pairs_tested += s.acc_pairs[i];
        o->alg_bytes += s.acc_bytes[i];
        o->tri_pairs += s.acc_tri[i];
        o->refined += s.acc_ref[i];
    }
    o->leaf_pairs = s.leaf_pairs;
    o->candidates = s.candidates;
    o->retries = retries;
    o->blocks = blocks;
    for (int i = 0; i < 32; ++i) o->level_ns[i] = s.level_ns[i];
    for (int i = 0; i < 12; ++i) o->phase_ns[i] = s.phase_ns[i];
    o->probes = s.probes;
    for (int i = 0; i < 32; ++i) o->u_level[i] = s.u_level[i];
    o->u_probe = s.u_probe;
    o->refits = s.refits;
}

gd_status check_pair(gd_ctx* ctx, const gd_mesh* A, const gd_mesh* B) {
    if (!A || !B) return fail(ctx, GD_ERR_INVALID_ARG, "NULL mesh");
    if (A->ctx != ctx || B->ctx != ctx) return fail(ctx, GD_ERR_INVALID_ARG, "mesh belongs to another context");
    if (!A->built || !B->built) return fail(ctx, GD_ERR_NOT_BUILT, "BVH not built (call gd_bvh_build)");
    return GD_OK;
}

// own: the meshes must belong to ctx (a server's private execution context
// runs meshes of the user's context on the same device and passes false)
gd_status run_single(gd_ctx* ctx, const gd_mesh* A, const gd_mesh* B, int kind, const double* xa, const double* xb,
                     gd_result* out, bool own = true) {
    if (!ctx) return GD_ERR_INVALID_ARG;
    if (!out || !xa || !xb) return fail(ctx, GD_ERR_INVALID_ARG, "NULL argument");
    gd_status s = own ? check_pair(ctx, A, B) : GD_OK;
    if (s != GD_OK) return s;
    if (!own && (!A || !B || !A->built || !B->built || A->ctx->device != ctx->device))
        return fail(ctx, GD_ERR_INVALID_ARG, "meshes not built on this device");
    std::string why;
    if (!xform_ok(xa, &why) || !xform_ok(xb, &why)) return fail(ctx, GD_ERR_INVALID_ARG, why);
    s = ensure_ws(ctx, 1);
    if (s != GD_OK) return s;
    const long long tab = table_entries(ctx, B);
    s = ensure_table(ctx, tab);
    if (s != GD_OK) return s;
    unsigned retries = 0;
    for (;;) {
        KArgs a{};
        a.nq = 1;
        a.qin = nullptr;
        a.mA = A->d_desc;
        a.mB = B->d_desc;
        a.xa_src = nullptr;
        a.xb_src = nullptr;
        std::memcpy(a.xa_val, xa, sizeof(a.xa_val));
        std::memcpy(a.xb_val, xb, sizeof(a.xb_val));
        fill_common(ctx, a, ctx->mb_dev->ctr, &ctx->mb_dev->stats);
        a.slot_of = ctx->slot_of;
        a.n_slot_of = (unsigned long long)tab;
        a.out = &ctx->mb_dev->out;
        a.done_ns = ctx->in_batch ? ctx->done_dev : nullptr;
        s = full_refit_tree(ctx, B, a);
        if (s != GD_OK) return s;
        int grid = grid_blocks(ctx, kind);
        a.work_ctas = single_work_ctas(ctx, grid);
        a.fuse_root = single_fuse_root(ctx, B);
        // the launch's last CTA writes the result record to pinned host
        // memory and stamps it with seq: no copy to enqueue and no stream
        // synchronisation on the way back
        const unsigned long long seq = ++ctx->hd_seq;
        a.host_done = ctx->hd;
        a.seq = seq;
        GD_CUDA(ctx, launch_query(kind, a, grid, ctx->stream));
        const volatile unsigned long long* stamp = &ctx->hd->seq;
        bool got = false;
        for (unsigned spin = 1;; ++spin) {
            if (*stamp == seq) { got = true; break; }
            if ((spin & 4095u) == 0u) {
                // a launch that ended (or failed) without the record
                const cudaError_t q = cudaStreamQuery(ctx->stream);
                if (q == cudaSuccess) { got = *stamp == seq; break; }
                if (q != cudaErrorNotReady) return cuda_fail(ctx, q, "query launch");
            }
        }
        std::atomic_thread_fence(std::memory_order_acquire);
        gd_result r;
        unsigned last_abort, bad_index;
        if (got) {
            std::memcpy(&r, (const void*)&ctx->hd->out, sizeof(r));
            last_abort = ctx->hd->last_abort;
            bad_index = ctx->hd->bad_index;
        } else {
            GD_CUDA(ctx, cudaMemcpyAsync(ctx->mb_host, ctx->mb_dev, kResultBytes, cudaMemcpyDeviceToHost, ctx->stream));
            GD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
            r = ctx->mb_host->out;
            last_abort = ctx->mb_host->ctr[kCtrLastAbort];
            bad_index = ctx->mb_host->ctr[kCtrBadIndex];
        }
        ctx->stats_pending = true;
        ctx->last_grid = grid;
        ctx->pending_retries = retries;
        if (last_abort) return fail(ctx, GD_ERR_TIMEOUT, "a device-side wait timed out");
        if (bad_index)
            return fail(ctx, GD_ERR_CUDA, "internal index check failed (sites " + std::to_string(bad_index) + ")");
        if (r.status == GD_ERR_OVERFLOW) {
            if (!grow(ctx)) return fail(ctx, GD_ERR_OVERFLOW, "work queues exceeded max_capacity");
            ++retries;
            continue;
        }
        *out = r;
        if (r.status != GD_OK) return fail(ctx, (gd_status)r.status, "query failed");
        return GD_OK;
    }
}

// One launch over the queries ids (all of one kind); results go to out, the
// queries that ran out of queue space to *redo, the launch's counters add to
// *agg.
gd_status batch_pass(gd_ctx* ctx, const gd_query* q, const std::vector<int64_t>& ids, int kind, gd_result* out,
                     gd_stats* agg, std::vector<int64_t>* redo, long long share) {
    const long long m = (long long)ids.size();
    gd_status s = ensure_ws(ctx, m);
    if (s != GD_OK) return s;
    s = size_for_batch(ctx, m, share);
    if (s != GD_OK) return s;
    long long tab = 0;
    for (long long j = 0; j < m; ++j) {
        const gd_query& Q = q[ids[j]];
        QIn& in = ctx->qin_host[j];
        in.A = Q.a->d_desc;
        in.B = Q.b->d_desc;
        std::memcpy(in.xa, Q.xa, sizeof(in.xa));
        std::memcpy(in.xb, Q.xb, sizeof(in.xb));
        in.slot_base = (unsigned)tab;
        tab += table_entries(ctx, Q.b);
    }
    if (tab > 0xfffffff0ll) return fail(ctx, GD_ERR_INVALID_ARG, "batch too large for the refit tables");
    s = ensure_table(ctx, tab);
    if (s != GD_OK) return s;
    GD_CUDA(ctx, cudaMemcpyAsync(ctx->qin_dev, ctx->qin_host, sizeof(QIn) * m, cudaMemcpyHostToDevice, ctx->stream));
    KArgs a{};
    a.nq = (int)m;
    a.qin = ctx->qin_dev;
    fill_common(ctx, a, ctx->mb_dev->ctr, &ctx->mb_dev->stats);
    a.slot_of = ctx->slot_of;
    a.n_slot_of = (unsigned long long)tab;
    a.out = ctx->out_dev;
    a.done_ns = ctx->done_dev;
    batch_limits(ctx->cap_front, ctx->cap_leaf, m, &a.q_budget, &a.q_pool);
    int grid = grid_blocks(ctx, kind, m > 1);
    GD_CUDA(ctx, launch_query(kind, a, grid, ctx->stream));
    GD_CUDA(ctx, cudaMemcpyAsync(ctx->out_host, ctx->out_dev, sizeof(gd_result) * m, cudaMemcpyDeviceToHost, ctx->stream));
    GD_CUDA(ctx, cudaMemcpyAsync(ctx->done_host, ctx->done_dev, sizeof(unsigned long long) * m,
                                 cudaMemcpyDeviceToHost, ctx->stream));
    GD_CUDA(ctx, cudaMemcpyAsync(ctx->mb_host, ctx->mb_dev, sizeof(Mailbox), cudaMemcpyDeviceToHost, ctx->stream));
    GD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (ctx->batch_t0 == 0) ctx->batch_t0 = ctx->mb_host->stats.t_start;
    gd_stats st;
    to_stats(ctx->mb_host->stats, (unsigned)grid, 0, &st);
    agg->levels = std::max(agg->levels, st.levels);
    agg->pairs_tested += st.pairs_tested;
    agg->leaf_pairs += st.leaf_pairs;
    agg->tri_pairs += st.tri_pairs;
    agg->candidates += st.candidates;
    agg->refined += st.refined;
    agg->alg_bytes += st.alg_bytes;
    agg->blocks = st.blocks;
    for (int i = 0; i < 32; ++i) {
        agg->front[i] += st.front[i];
        agg->slots[i] = std::max(agg->slots[i], st.slots[i]);
    }
    // phase times of CTA 0, summed over the batch's launches
    for (int i = 0; i < 12; ++i) agg->phase_ns[i] += st.phase_ns[i];
    if (ctx->mb_host->ctr[kCtrLastAbort]) return fail(ctx, GD_ERR_TIMEOUT, "a device-side wait timed out");
    if (ctx->mb_host->ctr[kCtrBadIndex])
        return fail(ctx, GD_ERR_CUDA,
                    "internal index check failed (sites " + std::to_string(ctx->mb_host->ctr[kCtrBadIndex]) + ")");
    for (long long j = 0; j < m; ++j) {
        out[ids[j]] = ctx->out_host[j];
        ctx->batch_done[ids[j]] = (long long)(ctx->done_host[j] - ctx->batch_t0);
        if (ctx->out_host[j].status == GD_ERR_OVERFLOW) redo->push_back(ids[j]);
    }
    return GD_OK;
}

}  // namespace

// =========================================================== C ABI

extern "C" {

GD_API gd_status gd_ctx_create(int device, gd_ctx** out) {
    if (!out) return GD_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return GD_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return GD_ERR_CUDA;
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, device);
    if (!coop) return GD_ERR_CUDA;
    gd_ctx* c = new gd_ctx();
    c->device = device;
    cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, device);
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete c;
        return GD_ERR_CUDA;
    }
    c->tun.work_target = 1ll << 17;
    c->tun.k_max = 6;
    c->tun.blocks_per_sm = 0;
    c->tun.front_capacity = 1ll << 24;
    c->tun.leaf_capacity = 1ll << 24;
    c->tun.cand_capacity = 1ll << 22;
    c->tun.max_capacity = 1ll << 30;
    c->tun.timeout_ns = 2000000000ll;
    c->tun.refit_mode = 1;
    c->tun.refit_slots = 1 << 13;
    c->tun.probes = 64;
    c->tun.batch_budget = 1ll << 23;
    c->tun.bounds_mode = 1;
    *out = c;
    return GD_OK;
}

GD_API void gd_ctx_destroy(gd_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    free_ws(c);
    cudaFree(c->mb_dev);
    cudaFreeHost(c->mb_host);
    cudaFreeHost(c->hd);
    cudaFree(c->qs); cudaFree(c->qin_dev); cudaFree(c->out_dev); cudaFree(c->done_dev);
    cudaFreeHost(c->qin_host); cudaFreeHost(c->out_host); cudaFreeHost(c->done_host);
    cudaFree(c->slot_of);
    cudaFree(c->ftree);
    cudaFree(c->naive_ws);
    cudaFree(c->point_ws); cudaFree(c->pts_dev); cudaFree(c->pres_dev);
    cudaFree(c->pkeys[0]); cudaFree(c->pkeys[1]); cudaFree(c->pvals[0]); cudaFree(c->pvals[1]);
    cudaFree(c->phist);
    cudaStreamDestroy(c->stream);
    delete c;
}

GD_API const char* gd_last_error(gd_ctx* c) { return c ? c->err.c_str() : "no context"; }

GD_API void* gd_ctx_stream(gd_ctx* c) { return c ? (void*)c->stream : nullptr; }

GD_API gd_status gd_ctx_set_tunables(gd_ctx* c, const gd_tunables* t) {
    if (!c || !t) return GD_ERR_INVALID_ARG;
    bool realloc = false;
    if (t->work_target > 0) c->tun.work_target = t->work_target;
    if (t->k_max > 0) c->tun.k_max = std::min(t->k_max, 12);
    if (t->blocks_per_sm > 0) c->tun.blocks_per_sm = t->blocks_per_sm;
    if (t->front_capacity > 0) { c->tun.front_capacity = t->front_capacity; realloc = true; }
    if (t->leaf_capacity > 0) { c->tun.leaf_capacity = t->leaf_capacity; realloc = true; }
    if (t->cand_capacity > 0) { c->tun.cand_capacity = t->cand_capacity; realloc = true; }
    if (t->max_capacity > 0) c->tun.max_capacity = t->max_capacity;
    if (t->timeout_ns > 0) c->tun.timeout_ns = t->timeout_ns;
    if (t->refit_mode >= 1 && t->refit_mode <= 3) c->tun.refit_mode = t->refit_mode;
    if (t->refit_slots > 0) { c->tun.refit_slots = t->refit_slots; realloc = true; }
    if (t->probes > 0) c->tun.probes = t->probes;
    if (t->batch_budget > 0) c->tun.batch_budget = t->batch_budget;
    if (t->bounds_mode == 1 || t->bounds_mode == 2) c->tun.bounds_mode = t->bounds_mode;
    ++c->ws_gen;
    if (realloc && c->ready) {
        cudaStreamSynchronize(c->stream);
        free_ws(c);
    }
    return GD_OK;
}

// Autotuner: one coordinate-descent pass over the traversal tunables, each
// setting timed (wall clock of the synchronous call, median of reps after one
// untimed run) on the caller's sample; a value is kept when it is at least 1%
// faster.  The tunables change only the speed, never the results.
GD_API gd_status gd_autotune(gd_ctx* c, const gd_query* sample, int64_t n, int32_t reps, gd_tunables* best) {
    if (!c) return GD_ERR_INVALID_ARG;
    if (!sample || n < 1 || n > (1ll << 20)) return fail(c, GD_ERR_INVALID_ARG, "autotune needs 1..2^20 sample queries");
    reps = reps > 0 ? std::min(reps, 50) : 3;
    std::vector<gd_result> out((size_t)n);
    auto timed = [&](double* ms) -> gd_status {
        std::vector<double> t;
        for (int r = -1; r < reps; ++r) {
            const auto t0 = std::chrono::steady_clock::now();
            gd_status s;
            if (n == 1) {
                const gd_query& q = sample[0];
                s = run_single(c, q.a, q.b, (int)q.kind, q.xa, q.xb, out.data());
            } else {
                s = gd_batch_query(c, sample, n, out.data());
            }
            const auto t1 = std::chrono::steady_clock::now();
            if (s != GD_OK) return s;
            if (r >= 0) t.push_back(std::chrono::duration<double, std::milli>(t1 - t0).count());
        }
        std::sort(t.begin(), t.end());
        *ms = t[t.size() / 2];
        return GD_OK;
    };
    double best_ms = 0.0;
    gd_status s = timed(&best_ms);
    if (s != GD_OK) return s;
    struct Axis {
        int64_t* f64;
        int32_t* f32;
        std::vector<int64_t> values;
    };
    std::vector<Axis> axes = {
        {&c->tun.work_target, nullptr, {1ll << 16, 1ll << 17, 1ll << 18, 1ll << 19, 1ll << 20}},
        {nullptr, &c->tun.k_max, {4, 5, 6, 7}},
        {nullptr, &c->tun.probes, {1, 16, 64, 128}},
        {nullptr, &c->tun.blocks_per_sm, {1, 2}},
    };
    if (n > 1) axes.push_back({&c->tun.batch_budget, nullptr, {1ll << 18, 1ll << 20, 1ll << 22, 1ll << 23, 1ll << 24}});
    for (Axis& ax : axes) {
        const int64_t keep = ax.f64 ? *ax.f64 : *ax.f32;
        int64_t chosen = keep;
        for (int64_t v : ax.values) {
            if (v == keep) continue;
            if (ax.f64) *ax.f64 = v; else *ax.f32 = (int32_t)v;
            double ms = 0.0;
            s = timed(&ms);
            if (s != GD_OK) {
                if (ax.f64) *ax.f64 = keep; else *ax.f32 = (int32_t)keep;
                return s;
            }
            if (ms < 0.99 * best_ms) {
                best_ms = ms;
                chosen = v;
            }
        }
        if (ax.f64) *ax.f64 = chosen; else *ax.f32 = (int32_t)chosen;
    }
    if (best) *best = c->tun;
    return GD_OK;
}

GD_API gd_status gd_batch_times(gd_ctx* c, int64_t n, int64_t* done_ns) {
    if (!c) return GD_ERR_INVALID_ARG;
    if (!done_ns || n != (int64_t)c->batch_done.size())
        return fail(c, GD_ERR_INVALID_ARG, "n must be the query count of the last gd_batch_query");
    for (int64_t i = 0; i < n; ++i) done_ns[i] = c->batch_done[(size_t)i];
    return GD_OK;
}

GD_API gd_status gd_ctx_get_tunables(gd_ctx* c, gd_tunables* t) {
    if (!c || !t) return GD_ERR_INVALID_ARG;
    *t = c->tun;
    return GD_OK;
}

GD_API gd_status gd_get_stats(gd_ctx* c, gd_stats* o) {
    if (!c || !o) return GD_ERR_INVALID_ARG;
    if (c->stats_pending) {
        // a device-resident query ran on a caller's stream: wait for the device
        cudaSetDevice(c->device);
        GD_CUDA(c, cudaDeviceSynchronize());
        GD_CUDA(c, cudaStreamSynchronize(c->stream));  // the launch may still be leaving
        GD_CUDA(c, cudaMemcpy(&c->mb_host->stats, &c->mb_dev->stats, sizeof(StatsDev), cudaMemcpyDeviceToHost));
        to_stats(c->mb_host->stats, (unsigned)c->last_grid, c->pending_retries, &c->last);
        c->stats_pending = false;
    }
    *o = c->last;
    return GD_OK;
}

GD_API gd_status gd_mesh_create(gd_ctx* ctx, const float* verts, int64_t nv, const int32_t* tris, int64_t nt,
                                gd_mesh** out) {
    if (!ctx || !out) return GD_ERR_INVALID_ARG;
    *out = nullptr;
    if (!verts || !tris || nv <= 0 || nt <= 0 || nt > (1ll << 30) || nv > (1ll << 31))
        return fail(ctx, GD_ERR_INVALID_ARG, "bad mesh sizes (need 1 <= nt <= 2^30, nv >= 1)");
    cudaSetDevice(ctx->device);
    gd_mesh* m = new gd_mesh();
    m->ctx = ctx;
    m->nv = nv;
    m->nt = nt;
    cudaError_t e = cudaMalloc(&m->d_verts, sizeof(float) * 3 * nv);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_tris, sizeof(int32_t) * 3 * nt);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->d_verts, verts, sizeof(float) * 3 * nv, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->d_tris, tris, sizeof(int32_t) * 3 * nt, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        gd_mesh_destroy(m);
        return cuda_fail(ctx, e, "gd_mesh_create");
    }
    *out = m;
    return GD_OK;
}

GD_API gd_status gd_bvh_build(gd_mesh* m, const gd_build_opts* opts) {
    if (!m) return GD_ERR_INVALID_ARG;
    gd_ctx* ctx = m->ctx;
    cudaSetDevice(ctx->device);
    int bits = 21;
    if (opts) {
        if (opts->morton_bits < 1 || opts->morton_bits > 21) return fail(ctx, GD_ERR_INVALID_ARG, "morton_bits in 1..21");
        bits = opts->morton_bits;
    }
    int L = 0;
    while ((2ll << L) <= m->nt) ++L;
    cudaFree(m->d_box); cudaFree(m->d_tri); cudaFree(m->d_order); cudaFree(m->d_stris);
    m->d_box = nullptr; m->d_tri = nullptr; m->d_order = nullptr; m->d_stris = nullptr;
    m->built = false;
    m->tree = false;
    BuildBuffers b{};
    b.verts = m->d_verts; b.tris = m->d_tris; b.nv = m->nv; b.nt = m->nt; b.L = L; b.morton_bits = bits;
    std::vector<void*> tmp;
    auto cleanup = [&]() { for (void* p : tmp) cudaFree(p); };
#define GD_ALLOC(ptr, bytes)                                                 \
    do {                                                                     \
        cudaError_t e_ = cudaMalloc((void**)&(ptr), (bytes));                \
        if (e_ != cudaSuccess) { cleanup(); return cuda_fail(ctx, e_, "gd_bvh_build alloc"); } \
        tmp.push_back((void*)(ptr));                                         \
    } while (0)
    GD_ALLOC(b.flags, 64 * sizeof(unsigned));
    GD_ALLOC(b.keys[0], sizeof(unsigned long long) * m->nt);
    GD_ALLOC(b.keys[1], sizeof(unsigned long long) * m->nt);
    GD_ALLOC(b.vals[0], sizeof(unsigned) * m->nt);
    GD_ALLOC(b.vals[1], sizeof(unsigned) * m->nt);
    GD_ALLOC(b.hist, sizeof(unsigned) * build_hist_words(m->nt));
#undef GD_ALLOC
    cudaError_t e = cudaMalloc(&m->d_box, sizeof(float) * 6 * (2ull << L));
    if (e == cudaSuccess) e = cudaMalloc(&m->d_tri, sizeof(float4) * 3 * m->nt);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_order, sizeof(unsigned) * m->nt);
    if (e == cudaSuccess) e = cudaMalloc(&m->d_stris, sizeof(int32_t) * 3 * m->nt);
    if (e != cudaSuccess) { cleanup(); return cuda_fail(ctx, e, "gd_bvh_build alloc"); }
    b.box = m->d_box;
    b.tri = m->d_tri;
    b.order = m->d_order;
    b.stris = m->d_stris;
    unsigned flags[8] = {0};
    // device time of the build's kernels: events around the validation and
    // around the tree build (not the allocations and the flag read-back)
    cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};
    for (cudaEvent_t& x : ev) cudaEventCreate(&x);
    auto drop_events = [&]() { for (cudaEvent_t& x : ev) if (x) cudaEventDestroy(x); };
    cudaEventRecord(ev[0], ctx->stream);
    e = build_validate(b, ctx->stream);
    cudaEventRecord(ev[1], ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(flags, b.flags, sizeof(flags), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) { drop_events(); cleanup(); return cuda_fail(ctx, e, "gd_bvh_build validate"); }
    if (flags[0]) { drop_events(); cleanup(); return fail(ctx, GD_ERR_INVALID_ARG, "triangle index out of range"); }
    if (flags[1]) { drop_events(); cleanup(); return fail(ctx, GD_ERR_INVALID_ARG, "non-finite vertex coordinate"); }
    cudaEventRecord(ev[2], ctx->stream);
    e = build_tree(b, ctx->stream);
    cudaEventRecord(ev[3], ctx->stream);
    float root[6];
    if (e == cudaSuccess) e = cudaMemcpyAsync(root, m->d_box + 6, sizeof(root), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    cleanup();
    if (e == cudaSuccess) {
        float t0 = 0.f, t1 = 0.f;
        cudaEventElapsedTime(&t0, ev[0], ev[1]);
        cudaEventElapsedTime(&t1, ev[2], ev[3]);
        m->build_ms = t0 + t1;
    }
    drop_events();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gd_bvh_build");
    float P = 0.f;
    for (int i = 0; i < 6; ++i) P = std::max(P, std::fabs(root[i]));
    m->L = L;
    m->h_desc.box = m->d_box;
    m->h_desc.tri = m->d_tri;
    m->h_desc.T = m->nt;
    m->h_desc.L = L;
    m->h_desc.P = P;
    if (!m->d_desc) GD_CUDA(ctx, cudaMalloc(&m->d_desc, sizeof(MeshDev)));
    GD_CUDA(ctx, cudaMemcpyAsync(m->d_desc, &m->h_desc, sizeof(MeshDev), cudaMemcpyHostToDevice, ctx->stream));
    GD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    m->built = true;
    m->tree = true;
    return GD_OK;
}

GD_API gd_status gd_mesh_update(gd_mesh* m, const float* verts, int64_t nv) {
    if (!m) return GD_ERR_INVALID_ARG;
    gd_ctx* ctx = m->ctx;
    if (!verts) return fail(ctx, GD_ERR_INVALID_ARG, "NULL vertices");
    if (nv != m->nv) return fail(ctx, GD_ERR_INVALID_ARG, "vertex count differs from the mesh's");
    if (!m->tree) return fail(ctx, GD_ERR_NOT_BUILT, "BVH not built (call gd_bvh_build)");
    cudaSetDevice(ctx->device);
    m->built = false;
    if (!m->d_flags) GD_CUDA(ctx, cudaMalloc(&m->d_flags, 64 * sizeof(unsigned)));
    // host or device source: with unified addressing the copy kind follows the pointer
    GD_CUDA(ctx, cudaMemcpyAsync(m->d_verts, verts, sizeof(float) * 3 * nv, cudaMemcpyDefault, ctx->stream));
    BuildBuffers b{};
    b.verts = m->d_verts; b.tris = m->d_tris; b.nv = m->nv; b.nt = m->nt; b.L = m->L;
    b.box = m->d_box; b.tri = m->d_tri; b.order = m->d_order; b.stris = m->d_stris; b.flags = m->d_flags;
    // the refit writes max |coordinate| straight into the device descriptor
    float* P_dev = reinterpret_cast<float*>(reinterpret_cast<char*>(m->d_desc) + offsetof(MeshDev, P));
    GD_CUDA(ctx, build_refit(b, P_dev, ctx->stream));
    unsigned flags[14];
    GD_CUDA(ctx, cudaMemcpyAsync(flags, b.flags, sizeof(flags), cudaMemcpyDeviceToHost, ctx->stream));
    GD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    if (flags[1]) return fail(ctx, GD_ERR_INVALID_ARG, "non-finite vertex coordinate (mesh left unbuilt)");
    float P = 0.f;
    for (int i = 0; i < 6; ++i) {
        float x;
        std::memcpy(&x, &flags[8 + i], sizeof(float));
        P = std::max(P, std::fabs(x));
    }
    m->h_desc.P = P;
    m->built = true;
    return GD_OK;
}

GD_API void gd_mesh_destroy(gd_mesh* m) {
    if (!m) return;
    if (m->ctx) {
        cudaSetDevice(m->ctx->device);
        cudaStreamSynchronize(m->ctx->stream);
    }
    cudaFree(m->d_verts); cudaFree(m->d_tris); cudaFree(m->d_box); cudaFree(m->d_tri); cudaFree(m->d_desc);
    cudaFree(m->d_order); cudaFree(m->d_stris); cudaFree(m->d_flags);
    delete m;
}

GD_API gd_status gd_mesh_build_time(const gd_mesh* m, double* device_ms) {
    if (!m || !device_ms) return GD_ERR_INVALID_ARG;
    if (!m->tree) return GD_ERR_NOT_BUILT;
    *device_ms = m->build_ms;
    return GD_OK;
}

GD_API gd_status gd_mesh_info(const gd_mesh* m, int32_t* levels, int64_t* triangles) {
    if (!m) return GD_ERR_INVALID_ARG;
    if (levels) *levels = m->L;
    if (triangles) *triangles = m->nt;
    return m->built ? GD_OK : GD_ERR_NOT_BUILT;
}

GD_API gd_status gd_mesh_download(const gd_mesh* m, float* boxes, int32_t* order) {
    if (!m) return GD_ERR_INVALID_ARG;
    if (!m->built) return fail(m->ctx, GD_ERR_NOT_BUILT, "BVH not built");
    gd_ctx* ctx = m->ctx;
    cudaSetDevice(ctx->device);
    if (boxes)
        GD_CUDA(ctx, cudaMemcpy(boxes, m->d_box, sizeof(float) * 6 * (2ull << m->L), cudaMemcpyDeviceToHost));
    if (order) {
        std::vector<float4> t(3 * m->nt);
        GD_CUDA(ctx, cudaMemcpy(t.data(), m->d_tri, sizeof(float4) * 3 * m->nt, cudaMemcpyDeviceToHost));
        for (long long j = 0; j < m->nt; ++j) {
            int id;
            std::memcpy(&id, &t[3 * j + 2].y, sizeof(int));
            order[j] = id;
        }
    }
    return GD_OK;
}

namespace {
constexpr long long kPointSortMin = 1 << 14;  // smaller calls walk the points in the caller's order

bool on_device(const void* p) {
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace

GD_API gd_status gd_point_distance(gd_ctx* ctx, const gd_mesh* M, const double x[12], const double* points,
                                   int64_t n, gd_point_result* out) {
    if (!ctx) return GD_ERR_INVALID_ARG;
    if (!x || n < 0 || (n > 0 && (!points || !out))) return fail(ctx, GD_ERR_INVALID_ARG, "NULL argument or n < 0");
    if (n > (1ll << 31)) return fail(ctx, GD_ERR_INVALID_ARG, "at most 2^31 points per call");
    if (!M) return fail(ctx, GD_ERR_INVALID_ARG, "NULL mesh");
    if (M->ctx != ctx) return fail(ctx, GD_ERR_INVALID_ARG, "mesh belongs to another context");
    if (!M->built) return fail(ctx, GD_ERR_NOT_BUILT, "BVH not built (call gd_bvh_build)");
    std::string why;
    if (!xform_ok(x, &why)) return fail(ctx, GD_ERR_INVALID_ARG, why);
    if (n == 0) return GD_OK;
    cudaSetDevice(ctx->device);
    if (!ctx->point_ws) GD_CUDA(ctx, cudaMalloc(&ctx->point_ws, sizeof(unsigned long long) * kPointWords));
    const bool dev_in = on_device(points), dev_out = on_device(out);
    if ((!dev_in || !dev_out) && n > ctx->cap_pts) {
        cudaFree(ctx->pts_dev); cudaFree(ctx->pres_dev);
        ctx->pts_dev = nullptr; ctx->pres_dev = nullptr; ctx->cap_pts = 0;
        GD_CUDA(ctx, cudaMalloc(&ctx->pts_dev, sizeof(double) * 3 * n));
        GD_CUDA(ctx, cudaMalloc(&ctx->pres_dev, sizeof(gd_point_result) * n));
        ctx->cap_pts = n;
    }
    PointArgs g{};
    g.box = M->d_box; g.tri = M->d_tri; g.T = M->nt; g.L = M->L;
    std::memcpy(g.x, x, sizeof(g.x));
    g.pts = dev_in ? points : ctx->pts_dev;
    g.n = n;
    g.out = dev_out ? out : ctx->pres_dev;
    g.ws = ctx->point_ws;
    g.timeout_ns = ctx->tun.timeout_ns;
    if (!dev_in)
        GD_CUDA(ctx, cudaMemcpyAsync(ctx->pts_dev, points, sizeof(double) * 3 * n, cudaMemcpyHostToDevice, ctx->stream));
    // enough points to fill the GPU: walk them in Morton order (warps of
    // nearby points visit the same nodes)
    if (n >= kPointSortMin) {
        if (n > ctx->cap_psort) {
            for (int k = 0; k < 2; ++k) {
                cudaFree(ctx->pkeys[k]); cudaFree(ctx->pvals[k]);
                ctx->pkeys[k] = nullptr; ctx->pvals[k] = nullptr;
            }
            cudaFree(ctx->phist);
            ctx->phist = nullptr;
            ctx->cap_psort = 0;
            for (int k = 0; k < 2; ++k) {
                GD_CUDA(ctx, cudaMalloc(&ctx->pkeys[k], sizeof(unsigned long long) * n));
                GD_CUDA(ctx, cudaMalloc(&ctx->pvals[k], sizeof(unsigned) * n));
            }
            GD_CUDA(ctx, cudaMalloc(&ctx->phist, sizeof(unsigned) * build_hist_words(n)));
            ctx->cap_psort = n;
        }
        const int cur = sort_points(g, ctx->pkeys, ctx->pvals, ctx->phist, ctx->stream);
        g.order = ctx->pvals[cur];
    }
    GD_CUDA(ctx, launch_point(g, ctx->stream));
    if (!dev_out)
        GD_CUDA(ctx, cudaMemcpyAsync(out, ctx->pres_dev, sizeof(gd_point_result) * n, cudaMemcpyDeviceToHost, ctx->stream));
    unsigned long long w[kPointWords];
    GD_CUDA(ctx, cudaMemcpyAsync(w, ctx->point_ws, sizeof(w), cudaMemcpyDeviceToHost, ctx->stream));
    GD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    ctx->last_point_tests = w[kPointTests];
    ctx->last_point_exact = w[kPointExact];
    if (w[kPointTimeout]) return fail(ctx, GD_ERR_TIMEOUT, "a point query passed the timeout");
    return GD_OK;
}

GD_API gd_status gd_point_stats(gd_ctx* ctx, uint64_t* node_tests, uint64_t* exact_tests) {
    if (!ctx) return GD_ERR_INVALID_ARG;
    if (node_tests) *node_tests = ctx->last_point_tests;
    if (exact_tests) *exact_tests = ctx->last_point_exact;
    return GD_OK;
}

GD_API gd_status gd_naive_query(gd_ctx* ctx, const gd_mesh* A, const gd_mesh* B, gd_kind kind, const double xa[12],
                                const double xb[12], int64_t timeout_ns, gd_naive_result* out) {
    if (!ctx) return GD_ERR_INVALID_ARG;
    if (!out || !xa || !xb) return fail(ctx, GD_ERR_INVALID_ARG, "NULL argument");
    if (kind != GD_MIN && kind != GD_MAX) return fail(ctx, GD_ERR_INVALID_ARG, "kind must be GD_MIN or GD_MAX");
    gd_status s = check_pair(ctx, A, B);
    if (s != GD_OK) return s;
    std::string why;
    if (!xform_ok(xa, &why) || !xform_ok(xb, &why)) return fail(ctx, GD_ERR_INVALID_ARG, why);
    cudaSetDevice(ctx->device);
    if (!ctx->naive_ws) GD_CUDA(ctx, cudaMalloc(&ctx->naive_ws, sizeof(unsigned long long) * kNaiveWords));
    NaiveArgs g{};
    g.triA = A->d_tri; g.TA = A->nt;
    g.boxB = B->d_box; g.triB = B->d_tri; g.TB = B->nt; g.LB = B->L;
    // A-local -> B-local: M = R_B^T R_A, c = R_B^T (t_A - t_B), in float64, then rounded
    double cmax = 0.0;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            double m = 0.0;
            for (int k = 0; k < 3; ++k) m += xb[4 * k + i] * xa[4 * k + j];
            g.R[3 * i + j] = (float)m;
        }
        double c = 0.0;
        for (int k = 0; k < 3; ++k) c += xb[4 * k + i] * (xa[4 * k + 3] - xb[4 * k + 3]);
        g.t[i] = (float)c;
        cmax = std::max(cmax, std::fabs(c));
    }
    // the float32 map is off by a few units in the last place of 3 P_A + |c|
    g.E = (float)std::ldexp(3.0 * (double)A->h_desc.P + cmax, -20);
    g.ws = ctx->naive_ws;
    g.timeout_ns = timeout_ns > 0 ? timeout_ns : ctx->tun.timeout_ns;
    GD_CUDA(ctx, launch_naive(kind, g, ctx->stream));
    unsigned long long w[kNaiveWords];
    GD_CUDA(ctx, cudaMemcpyAsync(w, ctx->naive_ws, sizeof(w), cudaMemcpyDeviceToHost, ctx->stream));
    GD_CUDA(ctx, cudaStreamSynchronize(ctx->stream));
    float u;
    const unsigned ub = (unsigned)(w[kNaiveU] & 0xffffffffull);
    std::memcpy(&u, &ub, sizeof(u));
    out->d = std::sqrt((double)u);
    out->node_tests = w[kNaiveTests];
    out->leaf_tests = w[kNaiveLeaves];
    out->max_thread_tests = w[kNaiveMaxTests];
    out->status = w[kNaiveBad] ? GD_ERR_CUDA : w[kNaiveTimeout] ? GD_ERR_TIMEOUT : GD_OK;
    out->pad = 0;
    if (w[kNaiveBad]) return fail(ctx, GD_ERR_CUDA, "naive walk outgrew its stack");
    if (w[kNaiveTimeout]) return fail(ctx, GD_ERR_TIMEOUT, "naive query passed its deadline");
    return GD_OK;
}

GD_API gd_status gd_min_distance(gd_ctx* ctx, const gd_mesh* A, const gd_mesh* B, const double xa[12],
                                 const double xb[12], gd_result* out) {
    return run_single(ctx, A, B, 0, xa, xb, out);
}

GD_API gd_status gd_max_distance(gd_ctx* ctx, const gd_mesh* A, const gd_mesh* B, const double xa[12],
                                 const double xb[12], gd_result* out) {
    return run_single(ctx, A, B, 1, xa, xb, out);
}

GD_API gd_status gd_query_device(gd_ctx* ctx, const gd_mesh* A, const gd_mesh* B, gd_kind kind, const double* d_xa,
                                 const double* d_xb, gd_result* d_out, void* stream) {
    if (!ctx) return GD_ERR_INVALID_ARG;
    if (!d_xa || !d_xb || !d_out || (kind != GD_MIN && kind != GD_MAX))
        return fail(ctx, GD_ERR_INVALID_ARG, "NULL argument or bad kind");
    gd_status s = check_pair(ctx, A, B);
    if (s != GD_OK) return s;
    if (!ctx->ready || !ctx->mb_dev || ctx->cap_q < 1)
        return fail(ctx, GD_ERR_INVALID_ARG, "work buffers not sized: run one synchronous query first");
    KArgs a{};
    a.nq = 1;
    a.mA = A->d_desc;
    a.mB = B->d_desc;
    a.xa_src = d_xa;
    a.xb_src = d_xb;
    const long long tab = table_entries(ctx, B);
    s = ensure_table(ctx, tab);
    if (s != GD_OK) return s;
    fill_common(ctx, a, ctx->mb_dev->ctr, &ctx->mb_dev->stats);
    a.slot_of = ctx->slot_of;
    a.n_slot_of = (unsigned long long)tab;
    a.out = d_out;
    s = full_refit_tree(ctx, B, a);
    if (s != GD_OK) return s;
    cudaStream_t st = stream ? (cudaStream_t)stream : ctx->stream;
    int grid = grid_blocks(ctx, (int)kind);
    a.work_ctas = single_work_ctas(ctx, grid);
    a.fuse_root = single_fuse_root(ctx, B);
    GD_CUDA(ctx, launch_query((int)kind, a, grid, st));
    ctx->stats_pending = true;
    ctx->last_grid = grid;
    ctx->pending_retries = 0;
    return GD_OK;
}

struct gd_graph {
    gd_ctx* ctx = nullptr;
    const gd_mesh* A = nullptr;
    const gd_mesh* B = nullptr;
    gd_kind kind = GD_MIN;
    const double* d_xa = nullptr;
    const double* d_xb = nullptr;
    gd_result* d_out = nullptr;
    cudaGraphExec_t exec = nullptr;
    unsigned gen = 0;  // work-buffer generation the graph was built for
};

namespace {
gd_status graph_build(gd_graph* g) {
    gd_ctx* ctx = g->ctx;
    KArgs a{};
    a.nq = 1;
    a.mA = g->A->d_desc;
    a.mB = g->B->d_desc;
    a.xa_src = g->d_xa;
    a.xb_src = g->d_xb;
    const long long tab = table_entries(ctx, g->B);
    gd_status s = ensure_table(ctx, tab);
    if (s != GD_OK) return s;
    fill_common(ctx, a, ctx->mb_dev->ctr, &ctx->mb_dev->stats);
    a.slot_of = ctx->slot_of;
    a.n_slot_of = (unsigned long long)tab;
    a.out = g->d_out;
    s = full_refit_tree(ctx, g->B, a);
    if (s != GD_OK) return s;
    const int grid = grid_blocks(ctx, (int)g->kind);
    a.work_ctas = single_work_ctas(ctx, grid);
    a.fuse_root = single_fuse_root(ctx, g->B);
    if (g->exec) {
        cudaGraphExecDestroy(g->exec);
        g->exec = nullptr;
    }
    GD_CUDA(ctx, build_query_graph((int)g->kind, a, grid, &g->exec));
    g->gen = ctx->ws_gen;
    ctx->last_grid = grid;
    return GD_OK;
}
}  // namespace

GD_API gd_status gd_graph_create(gd_ctx* ctx, const gd_mesh* A, const gd_mesh* B, gd_kind kind, const double* d_xa,
                                 const double* d_xb, gd_result* d_out, gd_graph** out) {
    if (!ctx || !out) return GD_ERR_INVALID_ARG;
    *out = nullptr;
    if (!d_xa || !d_xb || !d_out || (kind != GD_MIN && kind != GD_MAX))
        return fail(ctx, GD_ERR_INVALID_ARG, "NULL argument or bad kind");
    gd_status s = check_pair(ctx, A, B);
    if (s != GD_OK) return s;
    if (!ctx->ready || !ctx->mb_dev || ctx->cap_q < 1)
        return fail(ctx, GD_ERR_INVALID_ARG, "work buffers not sized: run one synchronous query first");
    gd_graph* g = new gd_graph();
    g->ctx = ctx;
    g->A = A;
    g->B = B;
    g->kind = kind;
    g->d_xa = d_xa;
    g->d_xb = d_xb;
    g->d_out = d_out;
    s = graph_build(g);
    if (s != GD_OK) {
        delete g;
        return s;
    }
    *out = g;
    return GD_OK;
}

GD_API gd_status gd_graph_launch(gd_graph* g, void* stream) {
    if (!g) return GD_ERR_INVALID_ARG;
    gd_ctx* ctx = g->ctx;
    if (!ctx->ready) return fail(ctx, GD_ERR_INVALID_ARG, "work buffers not sized: run one synchronous query first");
    if (g->gen != ctx->ws_gen) {
        // the context's work buffers moved (grown queues, new tunables): the
        // node's arguments are rebuilt
        gd_status s = graph_build(g);
        if (s != GD_OK) return s;
    }
    GD_CUDA(ctx, cudaGraphLaunch(g->exec, stream ? (cudaStream_t)stream : ctx->stream));
    ctx->stats_pending = true;
    return GD_OK;
}

GD_API gd_status gd_graph_destroy(gd_graph* g) {
    if (!g) return GD_ERR_INVALID_ARG;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    delete g;
    return GD_OK;
}

GD_API gd_status gd_batch_query(gd_ctx* ctx, const gd_query* q, int64_t n, gd_result* out) {
    if (!ctx) return GD_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!q || !out))) return fail(ctx, GD_ERR_INVALID_ARG, "NULL argument");
    if (n == 0) return GD_OK;
    if (n > (1ll << 24)) return fail(ctx, GD_ERR_INVALID_ARG, "batch larger than 2^24 queries");
    std::string why;
    for (int64_t i = 0; i < n; ++i) {
        gd_status s = check_pair(ctx, q[i].a, q[i].b);
        if (s != GD_OK) return s;
        if (q[i].kind != GD_MIN && q[i].kind != GD_MAX) return fail(ctx, GD_ERR_INVALID_ARG, "bad query kind");
        if (!xform_ok(q[i].xa, &why) || !xform_ok(q[i].xb, &why)) return fail(ctx, GD_ERR_INVALID_ARG, why);
    }
    unsigned total_retries = 0;
    gd_stats agg{};
    ctx->batch_done.assign((size_t)n, -1);
    ctx->batch_t0 = 0;
    struct InBatch {
        gd_ctx* c;
        ~InBatch() { c->in_batch = false; }
    } in_batch_guard{ctx};
    ctx->in_batch = true;
    for (int kind = 0; kind < 2; ++kind) {
        std::vector<int64_t> idx;
        for (int64_t i = 0; i < n; ++i)
            if ((int)q[i].kind == kind) idx.push_back(i);
        if (idx.empty()) continue;
        // Rounds: in round r every query may push share_r = batch_budget x
        // 16^r entries per level, so one launch takes a chunk of
        // max_capacity / (2 share_r) queries (the front and the leaf queue
        // then never overflow).  Queries evicted in a round, the few with
        // larger fronts, go to the next round in smaller chunks; a chunk of
        // one runs alone, where the queues grow as far as that query needs.
        const long long lim = std::min<long long>(ctx->tun.max_capacity, 0xffffffffll);
        long long share = std::max<long long>(1, ctx->tun.batch_budget);
        std::vector<int64_t> cur = std::move(idx);
        while (!cur.empty()) {
            const long long chunk = std::max<long long>(1, lim / (2 * share));
            std::vector<int64_t> next;
            for (size_t b = 0; b < cur.size(); b += (size_t)chunk) {
                const size_t e = std::min(cur.size(), b + (size_t)chunk);
                if (e - b == 1) {
                    const int64_t i = cur[b];
                    gd_status r = run_single(ctx, q[i].a, q[i].b, kind, q[i].xa, q[i].xb, &out[i]);
                    total_retries += ctx->pending_retries;
                    if (r != GD_OK && r != GD_ERR_OVERFLOW) return r;
                    // its completion stamp (and, for a batch that starts with
                    // a lone query, the call's first launch start)
                    unsigned long long st[2] = {0ull, 0ull};
                    GD_CUDA(ctx, cudaMemcpy(&st[0], ctx->done_dev, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
                    if (ctx->batch_t0 == 0) {
                        GD_CUDA(ctx, cudaMemcpy(&st[1], &ctx->mb_dev->stats.t_start, sizeof(unsigned long long),
                                                cudaMemcpyDeviceToHost));
                        ctx->batch_t0 = st[1];
                    }
                    ctx->batch_done[i] = (long long)(st[0] - ctx->batch_t0);
                    continue;
                }
                std::vector<int64_t> part(cur.begin() + b, cur.begin() + e);
                gd_status s = batch_pass(ctx, q, part, kind, out, &agg, &next, share);
                if (s != GD_OK) return s;
            }
            total_retries += (unsigned)next.size();
            cur = std::move(next);
            share *= 16;
        }
    }
    agg.retries = total_retries;
    ctx->last = agg;
    ctx->stats_pending = false;
    return GD_OK;
}

}  // extern "C"

// ---- hooks for the serving loop (gd_serve.cu)
namespace gd {

gd_status serve_prepare(gd_ctx* ctx, long long m) {
    cudaSetDevice(ctx->device);
    gd_status s = ensure_ws(ctx, m);
    if (s != GD_OK) return s;
    return ensure_table(ctx, 1 << 16);
}

gd_status serve_single(gd_ctx* ctx, const gd_query& q, gd_result* out) {
    return run_single(ctx, q.a, q.b, (int)q.kind, q.xa, q.xb, out, false);
}

// The server's pipelined single queries: launch one on ctx's stream with its
// result record in pinned slot 1 + slot (stream order keeps launches from
// overlapping, so they share the work buffers), and later collect it.  A
// query that overflowed the buffers, or whose record is missing, is run
// again synchronously (the buffers grow there).
gd_status serve_single_launch(gd_ctx* ctx, const gd_query& q, int slot, unsigned long long* seq) {
    const gd_mesh* A = q.a;
    const gd_mesh* B = q.b;
    const int kind = (int)q.kind;
    if (!A || !B || !A->built || !B->built || A->ctx->device != ctx->device)
        return fail(ctx, GD_ERR_INVALID_ARG, "meshes not built on this device");
    gd_status s = ensure_ws(ctx, 1);
    if (s != GD_OK) return s;
    const long long tab = table_entries(ctx, B);
    s = ensure_table(ctx, tab);
    if (s != GD_OK) return s;
    KArgs a{};
    a.nq = 1;
    a.mA = A->d_desc;
    a.mB = B->d_desc;
    std::memcpy(a.xa_val, q.xa, sizeof(a.xa_val));
    std::memcpy(a.xb_val, q.xb, sizeof(a.xb_val));
    fill_common(ctx, a, ctx->mb_dev->ctr, &ctx->mb_dev->stats);
    a.slot_of = ctx->slot_of;
    a.n_slot_of = (unsigned long long)tab;
    a.out = &ctx->mb_dev->out;
    s = full_refit_tree(ctx, B, a);
    if (s != GD_OK) return s;
    const int grid = grid_blocks(ctx, kind);
    a.work_ctas = single_work_ctas(ctx, grid);
    a.fuse_root = single_fuse_root(ctx, B);
    *seq = ++ctx->hd_seq;
    a.host_done = ctx->hd + 1 + slot;
    a.seq = *seq;
    GD_CUDA(ctx, launch_query(kind, a, grid, ctx->stream));
    ctx->stats_pending = true;
    ctx->last_grid = grid;
    ctx->pending_retries = 0;
    return GD_OK;
}

bool serve_single_ready(gd_ctx* ctx, int slot, unsigned long long seq) {
    return *(const volatile unsigned long long*)&ctx->hd[1 + slot].seq == seq;
}

gd_status serve_single_finish(gd_ctx* ctx, const gd_query& q, int slot, unsigned long long seq, gd_result* out) {
    HostDone* h = ctx->hd + 1 + slot;
    const volatile unsigned long long* stamp = &h->seq;
    bool got = false;
    for (unsigned spin = 1;; ++spin) {
        if (*stamp == seq) { got = true; break; }
        if ((spin & 4095u) == 0u) {
            const cudaError_t e = cudaStreamQuery(ctx->stream);
            if (e == cudaSuccess) { got = *stamp == seq; break; }
            if (e != cudaErrorNotReady) return cuda_fail(ctx, e, "serving launch");
        }
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    if (!got) return fail(ctx, GD_ERR_CUDA, "serving launch ended without its result record");
    if (h->last_abort) return fail(ctx, GD_ERR_TIMEOUT, "a device-side wait timed out");
    if (h->bad_index)
        return fail(ctx, GD_ERR_CUDA, "internal index check failed (sites " + std::to_string(h->bad_index) + ")");
    gd_result r;
    std::memcpy(&r, (const void*)&h->out, sizeof(r));
    if (r.status == GD_ERR_OVERFLOW) return serve_single(ctx, q, out);
    *out = r;
    return r.status == GD_OK ? GD_OK : (gd_status)r.status;
}

// One launch of m queries of one kind on ctx's own buffers, for the server:
// the kernel reads the queries from pinned host memory, and its last CTA
// copies the m result records and its abort and index-check words to pinned
// memory and stamps them, so the host neither copies nor synchronises the
// stream on the way (a lost stamp falls back to the stream's status).
// Queries that outgrew their share of the queues come back with status
// GD_ERR_OVERFLOW; the caller reruns them alone.
gd_status serve_batch(gd_ctx* ctx, const gd_query* qs, long long m, int kind, gd_result* out) {
    gd_status s = ensure_ws(ctx, m);
    if (s != GD_OK) return s;
    long long tab = 0;
    for (long long j = 0; j < m; ++j) {
        QIn& in = ctx->qin_host[j];
        in.A = qs[j].a->d_desc;
        in.B = qs[j].b->d_desc;
        std::memcpy(in.xa, qs[j].xa, sizeof(in.xa));
        std::memcpy(in.xb, qs[j].xb, sizeof(in.xb));
        in.slot_base = (unsigned)tab;
        tab += table_entries(ctx, qs[j].b);
    }
    if (tab > 0xfffffff0ll) return fail(ctx, GD_ERR_INVALID_ARG, "batch too large for the refit tables");
    s = ensure_table(ctx, tab);
    if (s != GD_OK) return s;
    KArgs a{};
    a.nq = (int)m;
    a.qin = ctx->qin_host;  // pinned: read by the kernel's setup
    fill_common(ctx, a, ctx->mb_dev->ctr, &ctx->mb_dev->stats);
    a.slot_of = ctx->slot_of;
    a.n_slot_of = (unsigned long long)tab;
    a.out = ctx->out_dev;
    batch_limits(ctx->cap_front, ctx->cap_leaf, m, &a.q_budget, &a.q_pool);
    const unsigned long long seq = ++ctx->hd_seq;
    a.host_done = ctx->hd;
    a.host_out = ctx->out_host;
    a.seq = seq;
    const int grid = grid_blocks(ctx, kind, m > 1);
    a.work_ctas = m == 1 ? single_work_ctas(ctx, grid) : (unsigned)grid;
    GD_CUDA(ctx, launch_query(kind, a, grid, ctx->stream));
    const volatile unsigned long long* stamp = &ctx->hd->seq;
    bool got = false;
    for (unsigned spin = 1;; ++spin) {
        if (*stamp == seq) { got = true; break; }
        if ((spin & 4095u) == 0u) {
            const cudaError_t q = cudaStreamQuery(ctx->stream);
            if (q == cudaSuccess) { got = *stamp == seq; break; }
            if (q != cudaErrorNotReady) return cuda_fail(ctx, q, "serving batch launch");
        }
    }
    std::atomic_thread_fence(std::memory_order_acquire);
    ctx->stats_pending = true;
    ctx->last_grid = grid;
    ctx->pending_retries = 0;
    if (!got) return fail(ctx, GD_ERR_CUDA, "serving batch ended without its result records");
    if (ctx->hd->last_abort) return fail(ctx, GD_ERR_TIMEOUT, "a device-side wait timed out");
    if (ctx->hd->bad_index)
        return fail(ctx, GD_ERR_CUDA, "internal index check failed (sites " + std::to_string(ctx->hd->bad_index) + ")");
    std::memcpy(out, (const void*)ctx->out_host, sizeof(gd_result) * (size_t)m);
    return GD_OK;
}

int serve_device(gd_ctx* ctx) { return ctx->device; }
int serve_sms(gd_ctx* ctx) { return ctx->sms; }
const gd_tunables& serve_tunables(gd_ctx* ctx) { return ctx->tun; }
bool serve_query_ok(gd_ctx* ctx, const gd_query& q, std::string* why) {
    if (check_pair(ctx, q.a, q.b) != GD_OK) { *why = ctx->err; return false; }
    if (q.kind != GD_MIN && q.kind != GD_MAX) { *why = "bad query kind"; return false; }
    return xform_ok(q.xa, why) && xform_ok(q.xb, why);
}
long long serve_mesh_tris(const gd_mesh* m) { return m ? m->nt : 0; }

// ---- read-only views used by the allocation-free entry point (gd_noalloc.cu)
gd_ctx* mesh_ctx(const gd_mesh* m) { return m ? m->ctx : nullptr; }
const MeshDev* mesh_desc(const gd_mesh* m) { return m && m->built ? m->d_desc : nullptr; }
int mesh_levels(const gd_mesh* m) { return m ? m->L : 0; }

// The launch shape and the tunable-derived fields of a single query on ctx
// against B, exactly as gd_query_device sets them: grid, background probe
// CTAs, the fused root push, bounds and refit modes.  Returns the grid.
int single_launch_fields(gd_ctx* c, const gd_mesh* B, int kind, KArgs& a) {
    fill_tunables(c, a);
    const int grid = grid_blocks(c, kind);
    a.work_ctas = single_work_ctas(c, grid);
    a.fuse_root = single_fuse_root(c, B);
    return grid;
}

}  // namespace gd
