// Persistent BVTT-front traversal for D_min / D_max (Algorithms 1-2, Sections
// 5-7) on GB300: one cooperative launch per query or batch.
//
// Phases (grid-wide barriers between them):
//   0  per-query setup: B-local -> A-local rigid map in float64, its float32
//      copy, and the absolute widening E of every float32 bound;
//   1  the root pair enters the front (Algorithm 1, front initialisation);
//   2  level loop (Algorithm 1's while loop, with the host round trip of the
//      paper removed): the adaptive depth k is chosen on the device from the
//      front length (Section 6), every entry is re-culled against the running
//      bound (Section 7.1), expanded k levels per side and its descendant
//      pairs are evaluated one per thread (Section 7.2: thread t serves entry
//      t >> 2k, its low bits pick the descendants in the implicit tree of
//      Section 7.3); survivors are appended with warp-aggregated atomics and
//      the running bound is lowered with a warp-reduced atomicMin on the float
//      bits (Section 7.4).  When the front first reaches a B subtree of 2^8
//      leaves, that subtree is refit into A's frame (the paper refits B per
//      frame, Section 8; here only the subtrees the front reaches are refit),
//      and right after the first refit, greedy probes seed the bound;
//   3  leaf-pair narrow phase: float32 triangle-triangle bounds, running bound
//      update, candidate list;
//   4  float64 refinement of the candidates in the world frame;
//   5  witness selection (smallest original (tri_a, tri_b) at the extreme);
//   6  witness points and result records.
#include <cfloat>
#include <cstdio>

#include "gd_geom.cuh"
#include "gd_internal.cuh"
#include "gd_launch.h"


namespace gd {

constexpr float kU = 5.9604645e-08f;    // 2^-24, unit roundoff of float32
constexpr float kRelW = 9.5367432e-07f; // 2^-20: world vs working-frame slack
constexpr unsigned kFltMaxBits = 0x7f7fffffu;
constexpr unsigned kNoSlot = 0xffffffffu, kClaimed = 0xfffffffeu;
constexpr unsigned kReprobes = 256;
constexpr int kDryRunDepth = 30;  // L_A + L_B from which background CTAs warm the code of later phases

// ------------------------------------------------------------- thresholds
// All float32 bounds are made rigorous for float64 world distances:
//   lower_world >= (lower_computed (1 - 16u) - E) (1 - 2^-20)
//   upper_world <= (upper_computed (1 + 16u) + E) (1 + 2^-20)
// with E covering the float32 mapping of B into A's frame (Phase 0).

// keep a pair whose squared enclosure gap is s2 while the min bound is U
__device__ __forceinline__ float min_keep_threshold(float U, float E) {
    float x = __fmul_ru(__fadd_ru(U, E), 1.0f + kRelW);
    return __fmul_ru(__fmul_ru(x, x), 1.0f + 16.0f * kU);
}

// keep a pair whose squared max-spread is s2 while the max bound is L
__device__ __forceinline__ float max_keep_threshold(float L, float E) {
    float x = __fsub_rd(L, E);
    if (!(x > 0.f)) return 0.f;
    x = __fmul_rd(x, 1.0f - kRelW);
    return __fmul_rd(__fmul_rd(x, x), 1.0f - 16.0f * kU);
}

__device__ __forceinline__ float upper_from_sq(float s2, float E) {
    float d = __fsqrt_ru(s2);
    return __fmul_ru(__fadd_ru(__fmul_ru(d, 1.0f + 16.0f * kU), E), 1.0f + kRelW);
}

__device__ __forceinline__ float lower_from_dist(float d, float E) {
    float x = __fsub_rd(__fmul_rd(d, 1.0f - 16.0f * kU), E);
    if (!(x > 0.f)) return 0.f;
    return __fmul_rd(x, 1.0f - kRelW);
}

__device__ __forceinline__ float lower_from_sq(float s2, float E) { return lower_from_dist(__fsqrt_rd(s2), E); }

// ------------------------------------------------------------- helpers

__device__ __forceinline__ Box load_box(const float* box, unsigned long long i) {
    const float2* p = reinterpret_cast<const float2*>(box + 6ull * i);
    float2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
    Box r;
    r.lo[0] = a.x; r.lo[1] = a.y; r.lo[2] = b.x;
    r.hi[0] = b.y; r.hi[1] = c.x; r.hi[2] = c.y;
    return r;
}

// refit boxes are written during the launch: read them through L2
__device__ __forceinline__ Box load_box_cg(const float* box, unsigned long long i) {
    const float2* p = reinterpret_cast<const float2*>(box + 6ull * i);
    float2 a = __ldcg(p), b = __ldcg(p + 1), c = __ldcg(p + 2);
    Box r;
    r.lo[0] = a.x; r.lo[1] = a.y; r.lo[2] = b.x;
    r.hi[0] = b.y; r.hi[1] = c.x; r.hi[2] = c.y;
    return r;
}

struct Tri32 {
    V3<float> v[3];
    int id;
};

__device__ __forceinline__ Tri32 load_tri(const float4* tri, unsigned j) {
    float4 p = __ldg(tri + 3ull * j), q = __ldg(tri + 3ull * j + 1), r = __ldg(tri + 3ull * j + 2);
    Tri32 t;
    t.v[0] = mk3(p.x, p.y, p.z);
    t.v[1] = mk3(p.w, q.x, q.y);
    t.v[2] = mk3(q.z, q.w, r.x);
    t.id = __float_as_int(r.y);
    return t;
}

__device__ __forceinline__ unsigned leaf_first(long long T, int L, unsigned leaf) {
    return (unsigned)(((unsigned long long)leaf * (unsigned long long)T) >> L);
}

__device__ __forceinline__ int depth_of(unsigned node) { return 31 - __clz(node); }

// Append v to buf if want (warp-aggregated: one atomic per warp).  Returns
// false for a lane whose entry did not fit.
template <class E>
__device__ __forceinline__ bool warp_push(bool want, const E& v, E* buf, unsigned* cnt, unsigned cap) {
    unsigned m = __ballot_sync(kFull, want);
    if (m == 0) return true;
    int lane = threadIdx.x & 31;
    int leader = __ffs(m) - 1;
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(cnt, (unsigned)__popc(m));
    base = __shfl_sync(kFull, base, leader);
    if (!want) return true;
    unsigned idx = base + __popc(m & lanemask_lt());
    if (idx < cap) {
        __stcg(reinterpret_cast<float4*>(buf + idx), *reinterpret_cast<const float4*>(&v));
        return true;
    }
    return false;
}

// Defensive index checks: a record read back from a work buffer must name a
// query of this launch and nodes / triangles of its meshes.  A failed check
// sets a bit in the counters (the host reports an internal error) and the
// access is skipped, so a bad record can never become an out-of-range load.
enum : unsigned {
    kBadFront = 1u, kBadLeaf = 2u, kBadCand = 4u, kBadJob = 8u, kBadProbe = 16u,
};

__device__ __forceinline__ bool item_ok(const KArgs& A, const Item& it) {
    return it.q < (unsigned)A.nq && it.a >= 1u && it.b >= 1u;
}

__device__ __forceinline__ void flag_bad(const KArgs& A, unsigned bit) { atomicOr(A.ctr + kCtrBadIndex, bit); }

__device__ __forceinline__ void mark_overflow(const KArgs& A, unsigned q) {
    atomicOr(&A.qs[q].status, kStatOverflow);
    atomicOr(A.ctr + kCtrOverflow, 1u);
}

// The launch arguments seen with the launch's mode as a compile-time
// constant (same layout as KArgs): kOne for a launch of one query.  The
// phases take the arguments as a deduced template type, so that every
// single-query / batch branch folds in each kernel instantiation.
template <bool ONE>
struct KArgsT : KArgs {
    static constexpr bool kOne = ONE;
};

// the constants of one query that the traversal reads
struct QConst {
    Rigid32 X;
    float E_box, E_tri;
    const float* boxA;
    const float* boxB;
    const float4* triA;
    const float4* triB;
    long long TA, TB;
    int LA, LB;
    int dR;
    unsigned slot_base;
};

// cached per-thread view of one query's constants
struct QView : QConst {
    unsigned q = 0xffffffffu;
};

// Per-CTA shared copies of global state, refreshed by thread 0 right after
// every grid barrier (the barrier's closing __syncthreads publishes them):
// the counters, and in a single-query launch the query's constants and its
// running bound and status.  Reading these from shared memory instead of
// L2 keeps 2,000+ warps from queueing on the same few words; a CTA's own
// bound improvements lower its copy at once and reach the global bound by one
// atomic each.
struct CtaState {
    QConst v;                 // query 0 (single-query launches)
    float Rl[9], tl[3], E_df; // its double-float map remainders
    unsigned ctr[kCtrReset];  // counters at the last barrier
    unsigned U, stat;         // its running bound (lowered by this CTA) and status
    unsigned cnt[2][2];       // entries this CTA appends in one iteration (by parity, queue)
    unsigned base[2];         // their first index in each queue
    unsigned rem;             // max remaining depth this CTA pushed in this level
    int ready;                // v, Rl, tl, E_df loaded
};

__device__ __forceinline__ CtaState& cta() {
    __shared__ CtaState s;
    return s;
}

__device__ __forceinline__ void load_qconst(const QState& s, QConst& V) {
#pragma unroll
    for (int i = 0; i < 9; ++i) V.X.R[i] = s.R[i];
#pragma unroll
    for (int i = 0; i < 3; ++i) V.X.t[i] = s.t[i];
    V.E_box = s.E_box;
    V.E_tri = s.E_tri;
    const MeshDev* ma = s.A;
    const MeshDev* mb = s.B;
    V.boxA = ma->box; V.boxB = mb->box;
    V.triA = ma->tri; V.triB = mb->tri;
    V.TA = ma->T; V.TB = mb->T;
    V.LA = ma->L; V.LB = mb->L;
    V.dR = s.dR;
    V.slot_base = s.slot_base;
}

// The constant fields of a QState are written once, in phase 0, before the
// first barrier, and no CTA reads them earlier in the launch: plain (L1
// cached) loads are safe for them.  U, status and the other fields written
// during the traversal are always read with relaxed GPU-scope loads.
template <class AT>
__device__ __forceinline__ void view(const AT& A, unsigned q, QView& V) {
    if (V.q == q) return;
    if (AT::kOne) static_cast<QConst&>(V) = cta().v;
    else load_qconst(A.qs[q], V);
    V.q = q;
}

// CTAs that run the traversal; any others run background probes
__device__ __forceinline__ unsigned work_ctas(const KArgs& A) { return A.work_ctas ? A.work_ctas : gridDim.x; }

// Thread 0: the single query's running bound and status, and (once) its
// constants, into the CTA state.
__device__ __forceinline__ void cta_load_query(const KArgs& A) {
    CtaState& c = cta();
    const unsigned long long w = ld_relaxed64(reinterpret_cast<const unsigned long long*>(&A.qs[0].U));
    c.U = (unsigned)w;
    c.stat = (unsigned)(w >> 32);
    if (!c.ready) {
        const QState& s = A.qs[0];
        load_qconst(s, c.v);
#pragma unroll
        for (int i = 0; i < 9; ++i) c.Rl[i] = s.Rl[i];
#pragma unroll
        for (int i = 0; i < 3; ++i) c.tl[i] = s.tl[i];
        c.E_df = s.E_df;
        c.ready = 1;
    }
}

// Thread 0's refresh of the CTA state after a barrier.
template <class AT>
__device__ __forceinline__ void cta_refresh(const AT& A) {
    CtaState& c = cta();
    unsigned v[kCtrReset];
#pragma unroll
    for (int i = 0; i < kCtrReset; ++i) v[i] = ld_relaxed(A.ctr + i);
#pragma unroll
    for (int i = 0; i < kCtrReset; ++i) c.ctr[i] = v[i];
    if (AT::kOne) cta_load_query(A);
    c.cnt[0][0] = c.cnt[0][1] = c.cnt[1][0] = c.cnt[1][1] = 0u;
    c.rem = 0u;
}

template <class AT>
__device__ __forceinline__ bool sync(const AT& A) {
    return grid_sync(A, [&] { cta_refresh(A); });
}

// The running bound U of a query and whether its traversal has stopped
// (D_min = 0 proven, or evicted from a batch), in one relaxed load (U and
// status are adjacent in an 8-byte aligned word).
__device__ __forceinline__ float load_U(const QState& s, bool* stop) {
    const unsigned long long w = ld_relaxed64(reinterpret_cast<const unsigned long long*>(&s.U));
    *stop = ((unsigned)(w >> 32) & kStatStop) != 0u;
    return __uint_as_float((unsigned)w);
}

// The same for query q of this launch: a single-query launch reads the CTA's
// copy (the bound at the last barrier, lowered by this CTA since).
template <class AT>
__device__ __forceinline__ float load_Uq(const AT& A, unsigned q, bool* stop) {
    if (AT::kOne) {
        const volatile CtaState& c = cta();
        *stop = (c.stat & kStatStop) != 0u;
        return __uint_as_float(c.U);
    }
    return load_U(A.qs[q], stop);
}

// Lower (KIND 0) or raise (KIND 1) the running bound of query q by bits v.
// All lanes of the warp call this; lanes with have == false pass nothing.  A
// single-query launch lowers the CTA's copy first and sends the global atomic
// only for a warp value that beats it.
template <int KIND, class AT>
__device__ __forceinline__ void warp_bound_update(const AT& A, bool have, unsigned q, unsigned v) {
    if (AT::kOne) {
        const unsigned r = KIND == 0 ? __reduce_min_sync(kFull, have ? v : 0xffffffffu)
                                     : __reduce_max_sync(kFull, have ? v : 0u);
        if ((threadIdx.x & 31) == 0) {
            volatile unsigned* cu = &cta().U;
            if (KIND == 0 ? r < *cu : r > *cu) {
                if (KIND == 0) {
                    atomicMin(const_cast<unsigned*>(cu), r);
                    atomicMin(&A.qs[0].U, r);
                } else {
                    atomicMax(const_cast<unsigned*>(cu), r);
                    atomicMax(&A.qs[0].U, r);
                }
            }
        }
        return;
    }
    QState* qs = A.qs;
    unsigned q0 = __shfl_sync(kFull, q, 0);
    bool uniform = __all_sync(kFull, q == q0);
    if (uniform) {
        unsigned r = KIND == 0 ? __reduce_min_sync(kFull, have ? v : 0xffffffffu)
                               : __reduce_max_sync(kFull, have ? v : 0u);
        if ((threadIdx.x & 31) == 0) {
            unsigned* U = &qs[q0].U;
            if (KIND == 0) {
                if (r < ld_relaxed(U)) atomicMin(U, r);
            } else {
                if (r > ld_relaxed(U)) atomicMax(U, r);
            }
        }
    } else if (have) {
        unsigned* U = &qs[q].U;
        if (KIND == 0) atomicMin(U, v);
        else atomicMax(U, v);
    }
}

// The CTA's ranges in two queues for the counts its warps added to the
// shared counters of parity p (every thread calls; threads 0 and 32 take one
// global atomic each and clear the other parity for the next iteration).
__device__ __forceinline__ void cta_reserve(int p, unsigned* cnt0, unsigned* cnt1) {
    CtaState& c = cta();
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned n = c.cnt[p][0];
        c.base[0] = n ? atomicAdd(cnt0, n) : 0u;
        c.cnt[p ^ 1][0] = 0u;
    } else if (threadIdx.x == 32) {
        const unsigned n = c.cnt[p][1];
        c.base[1] = n ? atomicAdd(cnt1, n) : 0u;
        c.cnt[p ^ 1][1] = 0u;
    }
    __syncthreads();
}

// Append the entries of one CTA-wide iteration to two queues (want0 -> buf0,
// want1 -> buf1) with one global atomic per queue and CTA: the warps count
// into shared memory, threads 0 and 32 reserve the CTA's ranges.  Every
// thread of the CTA calls it in the same iteration it (its parity picks the
// shared counters, the other parity is cleared for the next iteration).
// Returns false for a lane whose entry did not fit.
template <class E>
__device__ __forceinline__ bool cta_push2(int it, const E& v, bool want0, E* buf0, unsigned* cnt0, unsigned cap0,
                                          bool want1, E* buf1, unsigned* cnt1, unsigned cap1) {
    CtaState& c = cta();
    const int lane = threadIdx.x & 31, p = it & 1;
    const unsigned m0 = __ballot_sync(kFull, want0), m1 = __ballot_sync(kFull, want1);
    unsigned o0 = 0u, o1 = 0u;
    if (lane == 0) {
        if (m0) o0 = atomicAdd(&c.cnt[p][0], (unsigned)__popc(m0));
        if (m1) o1 = atomicAdd(&c.cnt[p][1], (unsigned)__popc(m1));
    }
    o0 = __shfl_sync(kFull, o0, 0);
    o1 = __shfl_sync(kFull, o1, 0);
    cta_reserve(p, cnt0, cnt1);
    const unsigned lt = lanemask_lt();
    bool ok = true;
    if (want0) {
        const unsigned idx = c.base[0] + o0 + __popc(m0 & lt);
        if (idx < cap0) __stcg(reinterpret_cast<float4*>(buf0 + idx), *reinterpret_cast<const float4*>(&v));
        else ok = false;
    }
    if (want1) {
        const unsigned idx = c.base[1] + o1 + __popc(m1 & lt);
        if (idx < cap1) __stcg(reinterpret_cast<float4*>(buf1 + idx), *reinterpret_cast<const float4*>(&v));
        else ok = false;
    }
    return ok;
}

// The same for up to four entries per thread: v[j] for the bits j of m, all
// to buf1 if to1, else all to buf0, in the order of j.  The warp's offsets
// come from the bits of the per-thread counts (three ballots per queue).
template <class E>
__device__ __forceinline__ bool cta_push4(int it, const E* v, unsigned m, bool to1, E* buf0, unsigned* cnt0,
                                          unsigned cap0, E* buf1, unsigned* cnt1, unsigned cap1) {
    CtaState& c = cta();
    const int lane = threadIdx.x & 31, p = it & 1;
    const unsigned k = (unsigned)__popc(m);
    const unsigned k0 = to1 ? 0u : k, k1 = to1 ? k : 0u;
    const unsigned lt = lanemask_lt();
    unsigned pre0 = 0u, tot0 = 0u, pre1 = 0u, tot1 = 0u;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        const unsigned b0 = __ballot_sync(kFull, (k0 >> b) & 1u), b1 = __ballot_sync(kFull, (k1 >> b) & 1u);
        pre0 += (unsigned)__popc(b0 & lt) << b;
        tot0 += (unsigned)__popc(b0) << b;
        pre1 += (unsigned)__popc(b1 & lt) << b;
        tot1 += (unsigned)__popc(b1) << b;
    }
    unsigned o0 = 0u, o1 = 0u;
    if (lane == 0) {
        if (tot0) o0 = atomicAdd(&c.cnt[p][0], tot0);
        if (tot1) o1 = atomicAdd(&c.cnt[p][1], tot1);
    }
    o0 = __shfl_sync(kFull, o0, 0);
    o1 = __shfl_sync(kFull, o1, 0);
    cta_reserve(p, cnt0, cnt1);
    E* buf = to1 ? buf1 : buf0;
    const unsigned cap = to1 ? cap1 : cap0;
    unsigned idx = to1 ? c.base[1] + o1 + pre1 : c.base[0] + o0 + pre0;
    bool ok = true;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        if ((m >> j) & 1u) {
            if (idx < cap) __stcg(reinterpret_cast<float4*>(buf + idx), *reinterpret_cast<const float4*>(&v[j]));
            else ok = false;
            ++idx;
        }
    }
    return ok;
}

// Refit slot holding B node b (depth db >= dR) in A's frame, or kNoSlot.  A
// refit publishes its slot index (after a fence) only once its boxes are
// written, and the refit jobs run beside the next level's expansion (no grid
// barrier between them): the acquire load makes the boxes visible with the
// index; a root still being refit reads as kNoSlot (mapped local boxes).
__device__ __forceinline__ unsigned refit_slot(const KArgs& A, const QView& V, unsigned b, int db) {
    if (V.dR < 0 || db < V.dR) return kNoSlot;
    unsigned root = b >> (db - V.dR);
    unsigned s = ld_acquire(A.slot_of + V.slot_base + (root - (1u << V.dR)));
    return s < A.cap_slots ? s : kNoSlot;
}

__device__ __forceinline__ unsigned long long refit_index(const QView& V, unsigned slot, unsigned b, int db) {
    int rel = db - V.dR;
    unsigned local = (1u << rel) | (b & ((1u << rel) - 1u));
    return (unsigned long long)slot * kRefitBoxes + local;
}

// Claim the refit of root b for query q (first claimer appends the job).
__device__ __forceinline__ void claim_root(const KArgs& A, const QView& V, unsigned q, unsigned b) {
    unsigned* e = A.slot_of + V.slot_base + (b - (1u << V.dR));
    if (ld_relaxed(e) != kNoSlot) return;
    if (atomicCAS(e, kNoSlot, kClaimed) != kNoSlot) return;
    unsigned j = atomicAdd(A.ctr + kCtrJobs, 1u);
    if (j < A.cap_slots) A.jobs[j] = make_uint2(q, b);
    // beyond capacity: the root stays claimed without a slot, and its subtree
    // keeps using the mapped local boxes (valid, only looser)
}

// ------------------------------------------------------------- triangles

// Bounds of one triangle pair (sorted ids ta of A, tb of B), rigorous for the
// float64 world distance: KIND 0 bounds the pair's min distance, KIND 1 its
// max distance.  The min lower bound is the separation of the two triangles
// along the direction between their float32 closest points (any direction
// gives a valid separation; this one is nearly optimal).
// Bounds on local float32 coordinates Al (triangle of A) and Bl (triangle of
// B) whose distances err by at most E: KIND 0 bounds the pair's min distance
// (upper: the best feature pair; lower: the separation of the two triangles
// along the direction between those closest points, valid for any
// direction and nearly tight for this one), KIND 1 its max distance.
template <int KIND>
__device__ __forceinline__ void tri_bounds_core(const V3<float>* Al, const V3<float>* Bl, float E, float* lo,
                                                float* up) {
    if (KIND == 0) {
        // the 21 feature pairs one after another (not unrolled): this code
        // runs once or a few times per CTA and query, and a compact loop is
        // fetched once where the unrolled form is fetched instruction by
        // instruction from L2
        V3<float> P = Al[0], Q = Bl[0];
        float d2 = INFINITY;
#pragma unroll 1
        for (int f = 0; f < 21; ++f) {
            V3<float> p, q;
            float e2;
            bool h;
            tri_feature(f, Al, Bl, &p, &q, &e2, &h);
            if (h) {
                P = p; Q = p; d2 = 0.f;
                break;
            }
            if (e2 < d2) { d2 = e2; P = p; Q = q; }
        }
        *up = upper_from_sq(d2, E);
        float l = 0.f;
        V3<float> nrm = P - Q;
        float nn = dot(nrm, nrm);
        if (nn > 0.f) {
            float amin = FLT_MAX, bmax = -FLT_MAX;
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                amin = fminf(amin, dot(nrm, Al[k]));
                bmax = fmaxf(bmax, dot(nrm, Bl[k]));
            }
            float sep = amin - bmax;
            if (sep > 0.f) l = lower_from_dist(sep / sqrtf(nn), E);
        }
        *lo = l;
    } else {
        V3<float> P, Q;
        float d2;
        tri_tri_max(Al, Bl, &P, &Q, &d2);
        *lo = lower_from_sq(d2, E);
        *up = upper_from_sq(d2, E);
    }
}

__device__ __forceinline__ float max_abs3(V3<float> v) { return fmaxf(fmaxf(fabsf(v.x), fabsf(v.y)), fabsf(v.z)); }

// Bounds of one triangle pair (sorted ids ta of A, tb of B), rigorous for the
// float64 world distance, from B's float32 map into A's frame.  The pair is
// moved to A's first vertex first: a difference of two float32 values is
// rounded relative to the (small) result, so every later rounding error
// scales with the pair's local extent X, not with the scene's coordinates;
// E_box covers the mapping of B's vertices.
template <int KIND>
__device__ __forceinline__ void tri_pair_bounds(const QView& V, unsigned ta, unsigned tb, float* lo, float* up) {
    Tri32 TA = load_tri(V.triA, ta), TB = load_tri(V.triB, tb);
    const V3<float> o = TA.v[0];
    V3<float> Al[3], Bl[3];
    float X = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        Al[k] = TA.v[k] - o;
        Bl[k] = map32(V.X, TB.v[k].x, TB.v[k].y, TB.v[k].z) - o;
        X = fmaxf(X, fmaxf(max_abs3(Al[k]), max_abs3(Bl[k])));
    }
    tri_bounds_core<KIND>(Al, Bl, __fadd_ru(V.E_box, __fmul_ru(256.0f * kU * 1.001f, X)), lo, up);
}

// The same bounds, tight: B's vertices mapped into A's frame in double-float
// (R + Rl, t + tl, ~48 bits) and moved to A's first vertex before rounding to
// float32, so that neither the map nor the magnitude of the coordinates
// leaves more than ~u times the pair's local extent (plus E_df) of error.
// Used for pairs that pass the float32 test, so that only near-ties reach the
// float64 refinement; it stays on the float32 pipe (float64 is slow here).
template <int KIND, class AT>
__device__ __forceinline__ void tri_pair_bounds_tight(const AT& A, unsigned q, const QView& V, const Tri32& TA,
                                                      const Tri32& TB, float* lo, float* up) {
    float Rl[9], tl[3], Edf;
    if (AT::kOne) {
        const CtaState& c = cta();
#pragma unroll
        for (int i = 0; i < 9; ++i) Rl[i] = c.Rl[i];
#pragma unroll
        for (int i = 0; i < 3; ++i) tl[i] = c.tl[i];
        Edf = c.E_df;
    } else {
        const QState& s = A.qs[q];
#pragma unroll
        for (int i = 0; i < 9; ++i) Rl[i] = s.Rl[i];
#pragma unroll
        for (int i = 0; i < 3; ++i) tl[i] = s.tl[i];
        Edf = s.E_df;
    }
    const V3<float> o = TA.v[0];
    const float oc[3] = {o.x, o.y, o.z};
    V3<float> Al[3], Bl[3];
    float X = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        Al[k] = mk3(__fsub_rn(TA.v[k].x, o.x), __fsub_rn(TA.v[k].y, o.y), __fsub_rn(TA.v[k].z, o.z));
        const float p[3] = {TB.v[k].x, TB.v[k].y, TB.v[k].z};
        float c[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            DF acc = two_sum(V.X.t[i], -oc[i]);
            acc = df_add(acc, DF{tl[i], 0.f});
#pragma unroll
            for (int j = 0; j < 3; ++j) acc = df_add(acc, df_mul_f(DF{V.X.R[3 * i + j], Rl[3 * i + j]}, p[j]));
            c[i] = __fadd_rn(acc.hi, acc.lo);
        }
        Bl[k] = mk3(c[0], c[1], c[2]);
        X = fmaxf(X, fmaxf(max_abs3(Al[k]), max_abs3(Bl[k])));
    }
    tri_bounds_core<KIND>(Al, Bl, __fadd_ru(Edf, __fmul_ru(256.0f * kU * 1.001f, X)), lo, up);
}

// Whether the plane of triangle P separates it from triangle Q by more than
// the running bound U: the separation of the two along P's normal (any axis
// gives a lower bound of their distance), widened as in tri_bounds_core.
__device__ __forceinline__ bool plane_apart(const V3<float>* P, const V3<float>* Q, float E, float U) {
    const V3<float> n = cross(P[1] - P[0], P[2] - P[0]);
    const float nn = dot(n, n);
    if (!(nn > 0.f)) return false;
    float pmin = FLT_MAX, pmax = -FLT_MAX, qmin = FLT_MAX, qmax = -FLT_MAX;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float p = dot(n, P[k]), q = dot(n, Q[k]);
        pmin = fminf(pmin, p);
        pmax = fmaxf(pmax, p);
        qmin = fminf(qmin, q);
        qmax = fmaxf(qmax, q);
    }
    const float sep = fmaxf(qmin - pmax, pmin - qmax);
    return sep > 0.f && lower_from_dist(sep / sqrtf(nn), E) > U;
}

// Cheap float32 test run before the tight bounds of a leaf's triangle pair:
// false only if the pair cannot hold the extreme.  Min kind: the separation
// of the two triangles along the line between their centroids, or (planes)
// along the normal of either one's plane (along any direction a valid lower
// bound of their distance, widened as in tri_bounds_core), exceeds the
// running bound U.  Max kind: the largest float32 vertex-pair distance, widened upward, is
// below the running bound.  Triangles with long thin shapes have boxes far
// larger than themselves, so most leaf pairs that pass the box test fail
// this one at a tenth of the cost of the tight bounds.
// Bw: B's three vertices already mapped into A's frame.
template <int KIND>
__device__ __forceinline__ bool tri_pair_may_hold_mapped(float E_box, const Tri32& TA, const V3<float>* Bw, float U,
                                                         bool planes) {
    const V3<float> o = TA.v[0];
    V3<float> Al[3], Bl[3];
    float X = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        Al[k] = TA.v[k] - o;
        Bl[k] = Bw[k] - o;
        X = fmaxf(X, fmaxf(max_abs3(Al[k]), max_abs3(Bl[k])));
    }
    const float E = __fadd_ru(E_box, __fmul_ru(256.0f * kU * 1.001f, X));
    if (KIND == 0) {
        const V3<float> n = (Al[0] + Al[1] + Al[2]) - (Bl[0] + Bl[1] + Bl[2]);
        const float nn = dot(n, n);
        if (!(nn > 0.f)) return true;
        float amin = FLT_MAX, bmax = -FLT_MAX;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            amin = fminf(amin, dot(n, Al[k]));
            bmax = fmaxf(bmax, dot(n, Bl[k]));
        }
        const float sep = amin - bmax;
        if (sep > 0.f && lower_from_dist(sep / sqrtf(nn), E) > U) return false;
        // the pairs left: the planes of A and of B as the separating axes
        return !(planes && (plane_apart(Al, Bl, E, U) || plane_apart(Bl, Al, E, U)));
    } else {
        float m2 = 0.f;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                const V3<float> d = Al[i] - Bl[j];
                m2 = fmaxf(m2, dot(d, d));
            }
        return upper_from_sq(m2, E) >= U;
    }
}

// The same test with B's triangle as stored (mapped into A's frame here).
template <int KIND>
__device__ __forceinline__ bool tri_pair_may_hold(const QConst& V, const Tri32& TA, const Tri32& TB, float U,
                                                  bool planes) {
    V3<float> Bw[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) Bw[k] = map32(V.X, TB.v[k].x, TB.v[k].y, TB.v[k].z);
    return tri_pair_may_hold_mapped<KIND>(V.E_box, TA, Bw, U, planes);
}

// ------------------------------------------------------------- pair bounds

// Bounds of node pair (ia of A, ib of B at depth db).  Returns the stored
// culling value (KIND 0: squared lower bound of the min; KIND 1: squared upper
// bound of the max) and whether the pair survives against Ucur; for a
// survivor, *newU is its enhanced bound (Eq. 10 / Eq. 11) for the running
// bound and *key orders survivors by it.
template <int KIND, bool FULL = false>
__device__ __forceinline__ float pair_bounds(const KArgs& A, const QView& V, unsigned ia, unsigned ib, int db,
                                             float Ucur, bool* survive, unsigned* newU, unsigned* key) {
    Box ba = load_box(V.boxA, ia);
    // FULL: B's whole tree was refit into A's frame at the start of the launch
    const unsigned slot = FULL ? 0u : refit_slot(A, V, ib, db);
    float bound;
    *key = 0xffffffffu;
    if (slot != kNoSlot) {
        // B's box already in A's frame (refit): plain AABB-AABB bounds
        Box bb = FULL ? load_box_cg(A.ftree, ib) : load_box_cg(A.rbox, refit_index(V, slot, ib, db));
        if (KIND == 0) {
            bound = lower_min_sq(ba, bb.lo, bb.hi);
            *survive = bound <= min_keep_threshold(Ucur, V.E_box);
            if (*survive) {
                float u2 = A.conventional ? upper_max_sq(ba, bb.lo, bb.hi) : upper_min_sq_enhanced<true>(V.X, ba, bb);
                *newU = __float_as_uint(upper_from_sq(u2, V.E_box));
                *key = __float_as_uint(u2);
            }
        } else {
            bound = upper_max_sq(ba, bb.lo, bb.hi);
            *survive = bound >= max_keep_threshold(Ucur, V.E_box);
            if (*survive) {
                float l2 = A.conventional ? lower_min_sq(ba, bb.lo, bb.hi) : lower_max_sq_enhanced<true>(V.X, ba, bb);
                *newU = __float_as_uint(lower_from_sq(l2, V.E_box));
                *key = ~__float_as_uint(l2);
            }
        }
    } else {
        Box bb = load_box(V.boxB, ib);
        float elo[3], ehi[3];
        enclose(V.X, bb, elo, ehi);
        if (KIND == 0) {
            bound = lower_min_sq(ba, elo, ehi);
            *survive = bound <= min_keep_threshold(Ucur, V.E_box);
            if (*survive) {
                float u2 = A.conventional ? upper_max_sq(ba, elo, ehi) : upper_min_sq_enhanced<false>(V.X, ba, bb);
                *newU = __float_as_uint(upper_from_sq(u2, V.E_box));
                *key = __float_as_uint(u2);
            }
        } else {
            bound = upper_max_sq(ba, elo, ehi);
            *survive = bound >= max_keep_threshold(Ucur, V.E_box);
            if (*survive) {
                float l2 = A.conventional ? lower_min_sq(ba, elo, ehi) : lower_max_sq_enhanced<false>(V.X, ba, bb);
                *newU = __float_as_uint(lower_from_sq(l2, V.E_box));
                *key = ~__float_as_uint(l2);
            }
        }
    }
    return bound;
}

// ------------------------------------------------------------- refit

// One shared-memory buffer for the refit of a subtree (lazy or full) and the
// full refit's upper levels: one declaration, so the three uses do not each
// add 12 KB of static shared memory to the CTA (2 CTAs per SM must fit).
__device__ __forceinline__ float* refit_smem() {
    __shared__ float sb[kRefitBoxes * 6];
    return sb;
}

// Refit the B subtree below root (depth dR, 2^h leaves, h <= kRefitH) into
// A's frame: one thread per leaf maps its one or two triangles with the
// query's float32 map, the CTA reduces the h levels in shared memory, and the
// 2^(h+1) - 1 boxes go to the slot in heap order (local root 1).  Every box is
// the exact bound of float32-mapped vertices, each within e_c of its exact
// image, so the widening E_box keeps every bound on it valid.
template <class AT>
__device__ void refit_subtree(const AT& A, unsigned q, unsigned root, unsigned slot) {
    float* sb = refit_smem();
    QView V;
    view(A, q, V);
    const int h = V.LB - V.dR;
    const unsigned nleaf = 1u << h;
    for (unsigned i = threadIdx.x; i < nleaf; i += blockDim.x) {
        unsigned leaf = ((root << h) | i) - (1u << V.LB);
        unsigned t0 = leaf_first(V.TB, V.LB, leaf), t1 = leaf_first(V.TB, V.LB, leaf + 1);
        float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
        for (unsigned t = t0; t < t1; ++t) {
            Tri32 T = load_tri(V.triB, t);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                V3<float> p = map32(V.X, T.v[k].x, T.v[k].y, T.v[k].z);
                lo[0] = fminf(lo[0], p.x); lo[1] = fminf(lo[1], p.y); lo[2] = fminf(lo[2], p.z);
                hi[0] = fmaxf(hi[0], p.x); hi[1] = fmaxf(hi[1], p.y); hi[2] = fmaxf(hi[2], p.z);
            }
        }
        float* o = sb + 6 * (nleaf + i);
        o[0] = lo[0]; o[1] = lo[1]; o[2] = lo[2]; o[3] = hi[0]; o[4] = hi[1]; o[5] = hi[2];
    }
    __syncthreads();
    for (int lev = h - 1; lev >= 0; --lev) {
        for (unsigned j = threadIdx.x; j < (1u << lev); j += blockDim.x) {
            unsigned k = (1u << lev) + j;
            const float* l = sb + 12 * k;
            float* o = sb + 6 * k;
            o[0] = fminf(l[0], l[6]); o[1] = fminf(l[1], l[7]); o[2] = fminf(l[2], l[8]);
            o[3] = fmaxf(l[3], l[9]); o[4] = fmaxf(l[4], l[10]); o[5] = fmaxf(l[5], l[11]);
        }
        __syncthreads();
    }
    float* dst = A.rbox + (unsigned long long)slot * kRefitBoxes * 6;
    for (unsigned i = 6 + threadIdx.x; i < 6u * (2u << h); i += blockDim.x) __stcg(dst + i, sb[i]);
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        A.slot_of[V.slot_base + (root - (1u << V.dR))] = slot;
    }
}

// Full refit of B into A's frame (refit mode 3: the paper refits B's tree for
// every frame of a rigid motion, Section 8).  Pass 1: CTA job j refits the
// subtree of 2^h leaves below node 2^dF + j exactly as refit_subtree does
// (float32-mapped vertices, exact bounds, h levels reduced in shared memory)
// and writes its boxes at their heap positions of A.ftree.  Pass 2 (after a
// grid barrier): the levels above, 8 at a time, one CTA per 2^8 nodes.
__device__ void full_refit_leaves(const KArgs& A, const QConst& V, unsigned root, int h) {
    float* sb = refit_smem();
    const unsigned nleaf = 1u << h;
    for (unsigned i = threadIdx.x; i < nleaf; i += blockDim.x) {
        const unsigned leaf = ((root << h) | i) - (1u << V.LB);
        const unsigned t0 = leaf_first(V.TB, V.LB, leaf), t1 = leaf_first(V.TB, V.LB, leaf + 1);
        float lo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, hi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
        for (unsigned t = t0; t < t1; ++t) {
            const Tri32 T = load_tri(V.triB, t);
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const V3<float> p = map32(V.X, T.v[k].x, T.v[k].y, T.v[k].z);
                lo[0] = fminf(lo[0], p.x); lo[1] = fminf(lo[1], p.y); lo[2] = fminf(lo[2], p.z);
                hi[0] = fmaxf(hi[0], p.x); hi[1] = fmaxf(hi[1], p.y); hi[2] = fmaxf(hi[2], p.z);
            }
        }
        float* o = sb + 6 * (nleaf + i);
        o[0] = lo[0]; o[1] = lo[1]; o[2] = lo[2]; o[3] = hi[0]; o[4] = hi[1]; o[5] = hi[2];
    }
    __syncthreads();
    for (int lev = h - 1; lev >= 0; --lev) {
        for (unsigned j = threadIdx.x; j < (1u << lev); j += blockDim.x) {
            const unsigned k = (1u << lev) + j;
            const float* l = sb + 12 * k;
            float* o = sb + 6 * k;
            o[0] = fminf(l[0], l[6]); o[1] = fminf(l[1], l[7]); o[2] = fminf(l[2], l[8]);
            o[3] = fmaxf(l[3], l[9]); o[4] = fmaxf(l[4], l[10]); o[5] = fmaxf(l[5], l[11]);
        }
        __syncthreads();
    }
    // local node k (level rel = depth of k) is node (root << rel) | (k - 2^rel)
    for (unsigned k = 1 + threadIdx.x; k < (2u << h); k += blockDim.x) {
        const int rel = 31 - __clz(k);
        const unsigned long long node = ((unsigned long long)root << rel) | (k - (1u << rel));
        float* dst = A.ftree + 6ull * node;
#pragma unroll
        for (int c = 0; c < 6; ++c) __stcg(dst + c, sb[6 * k + c]);
    }
    __syncthreads();
}

// lv levels above depth d for the 2^lv nodes of depth d from first: their
// parents up to depth d - lv, reduced in shared memory
__device__ void full_refit_up(const KArgs& A, unsigned long long first, int lv) {
    float* sb = refit_smem();
    const unsigned n = 1u << lv;
    for (unsigned i = threadIdx.x; i < n; i += blockDim.x) {
        const float* b = A.ftree + 6ull * (first + i);
#pragma unroll
        for (int c = 0; c < 6; ++c) sb[6 * (n + i) + c] = __ldcg(b + c);
    }
    __syncthreads();
    for (int lev = lv - 1; lev >= 0; --lev) {
        for (unsigned j = threadIdx.x; j < (1u << lev); j += blockDim.x) {
            const unsigned k = (1u << lev) + j;
            const float* l = sb + 12 * k;
            float* o = sb + 6 * k;
            o[0] = fminf(l[0], l[6]); o[1] = fminf(l[1], l[7]); o[2] = fminf(l[2], l[8]);
            o[3] = fmaxf(l[3], l[9]); o[4] = fmaxf(l[4], l[10]); o[5] = fmaxf(l[5], l[11]);
            const int rel = lev;
            const unsigned long long node = ((first >> lv) << rel) | j;
            float* dst = A.ftree + 6ull * node;
#pragma unroll
            for (int c = 0; c < 6; ++c) __stcg(dst + c, o[c]);
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------- probes

// One compiled copy (not inlined): every caller (the refinement's grid and
// tail paths, the D = 0 proof) gets bit-identical float64 results for a pair,
// whatever multiply-adds the compiler would contract into FMAs in an inlined
// copy.
template <int KIND>
__device__ __noinline__ double refine_pair_warp(const QState& s, unsigned ta, unsigned tb, V3<double>* P,
                                                V3<double>* Q, int* ida, int* idb);
template <int KIND>
__device__ __noinline__ double refine_pair_cta(const QState& s, const float4* triA, const float4* triB, unsigned ta,
                                               unsigned tb, V3<double>* P, V3<double>* Q, int* ida, int* idb);
template <int KIND, class AT>
__device__ __noinline__ void leaf_tight(const AT& A, const uint4* list, unsigned n, int& pit, unsigned& tripairs,
                                        unsigned long long& bytes, bool dry);

// Proof of D_min = 0 (min kind), run by a whole warp on one pair (ta, tb) of
// query q whose float32 lower bound is 0: the float64 distance of the pair,
// computed exactly as the refinement does.  If it is exactly 0 the query is
// done: no pair can be closer, so kStatZero stops its traversal, and the pair
// enters the candidates with bound -1, the only mark the refinement keeps once
// kStatZero is set.  A query starts at most kCertMax checks per launch, so
// touching but disjoint pairs cannot make the proof attempts dominate.
template <class AT>
__device__ __noinline__ void certify_zero(const AT& A, unsigned q, unsigned ta, unsigned tb) {
    QState& s = A.qs[q];
    const int lane = threadIdx.x & 31;
    unsigned go = 0;
    if (lane == 0) go = !(ld_relaxed(&s.status) & kStatZero) && atomicAdd(&s.cert, 1u) < kCertMax;
    if (!__shfl_sync(kFull, go, 0)) return;
    V3<double> P, Q;
    int ia, ib;
    const double d = refine_pair_warp<0>(s, ta, tb, &P, &Q, &ia, &ib);
    if (d == 0.0 && lane == 0) {
        if (AT::kOne) atomicOr(&cta().stat, kStatZero);
        if (!(atomicOr(&s.status, kStatZero) & kStatZero)) {
            unsigned i = atomicAdd(A.ctr + kCtrCand, 1u);
            if (i < A.cap_cand) A.cand[i] = Cand{ta, tb, -1.f, q};
            else mark_overflow(A, q);
        }
    }
}

// Greedy descent from one front entry by one warp: at each step up to 32
// descendant pairs (5 levels split between the two trees) are bounded, the
// running bound takes their enhanced bounds (Eq. 10 / Eq. 11), and the walk
// follows the pair with the best enhanced bound until both nodes are leaves,
// whose triangle pairs then tighten the bound further.  Probes only move the
// running bound by valid bounds; they add no front entries or candidates, so
// the traversal's result does not depend on them.  They exist to reach a
// near-final bound before the breadth-first levels widen (the sequential
// depth-first behaviour Section 6 contrasts with).
template <int KIND, class AT>
__device__ void probe(const AT& A, Item it, const QView& V) {
    const int lane = threadIdx.x & 31;
    unsigned a = it.a, b = it.b;
    const unsigned q = it.q;
    for (int step = 0; step < 64; ++step) {
        const int remA = V.LA - depth_of(a), remB = V.LB - depth_of(b);
        if (remA == 0 && remB == 0) break;
        int kA = min(remA, 3);
        const int kB = min(remB, 5 - kA);
        kA = min(remA, 5 - kB);
        const bool valid = lane < (1 << (kA + kB));
        const unsigned ia = (a << kA) | ((unsigned)lane >> kB);
        const unsigned ib = (b << kB) | ((unsigned)lane & ((1u << kB) - 1u));
        bool stop;
        // a background probe CTA meets no barrier: it reads the global bound
        const float Ucur = blockIdx.x >= work_ctas(A) ? load_U(A.qs[q], &stop) : load_Uq(A, q, &stop);
        if (__any_sync(kFull, stop)) return;
        bool ok = false;
        unsigned newU = KIND == 0 ? 0xffffffffu : 0u, key = 0xffffffffu;
        if (valid) pair_bounds<KIND>(A, V, ia, ib, depth_of(b) + kB, Ucur, &ok, &newU, &key);
        warp_bound_update<KIND>(A, ok, q, newU);
        const unsigned best = __reduce_min_sync(kFull, ok ? key : 0xffffffffu);
        const unsigned m = __ballot_sync(kFull, ok && key == best);
        if (m == 0) return;
        const int src = __ffs(m) - 1;
        a = __shfl_sync(kFull, ia, src);
        b = __shfl_sync(kFull, ib, src);
    }
    const unsigned la = a - (1u << V.LA), lb = b - (1u << V.LB);
    const unsigned a0 = leaf_first(V.TA, V.LA, la), a1 = leaf_first(V.TA, V.LA, la + 1);
    const unsigned b0 = leaf_first(V.TB, V.LB, lb), b1 = leaf_first(V.TB, V.LB, lb + 1);
    const unsigned ta = a0 + ((unsigned)lane >> 1), tb = b0 + ((unsigned)lane & 1u);
    const bool valid = lane < 4 && ta < a1 && tb < b1;
    float lo = 0.f, up = 0.f;
    if (valid) tri_pair_bounds<KIND>(V, ta, tb, &lo, &up);
    warp_bound_update<KIND>(A, valid, q, __float_as_uint(KIND == 0 ? up : lo));
    if (KIND == 0) {
        const unsigned m = __ballot_sync(kFull, valid && lo <= 0.f);
        if (m) {
            const int src = __ffs(m) - 1;
            certify_zero(A, q, __shfl_sync(kFull, ta, src), __shfl_sync(kFull, tb, src));
        }
    }
}

// A probe that starts at the root pair.  Its first two steps take the
// descendant pair of rank w mod 32 and then (w / 32) mod 32 among the
// survivors (ordered by their enhanced bound), so that the walks of different
// warps start in different subtree pairs; then it walks greedily as probe().
template <int KIND, class AT>
__device__ void probe_root(const AT& A, unsigned w, const QView& V) {
    const int lane = threadIdx.x & 31;
    unsigned a = 1u, b = 1u;
    for (int step = 0; step < 2; ++step) {
        const int remA = V.LA - depth_of(a), remB = V.LB - depth_of(b);
        if (remA == 0 && remB == 0) break;
        int kA = min(remA, 3);
        const int kB = min(remB, 5 - kA);
        kA = min(remA, 5 - kB);
        const bool valid = lane < (1 << (kA + kB));
        const unsigned ia = (a << kA) | ((unsigned)lane >> kB);
        const unsigned ib = (b << kB) | ((unsigned)lane & ((1u << kB) - 1u));
        bool stop;
        const float Ucur = load_U(A.qs[0], &stop);
        if (__any_sync(kFull, stop)) return;
        bool ok = false;
        unsigned newU = KIND == 0 ? 0xffffffffu : 0u, key = 0xffffffffu;
        if (valid) pair_bounds<KIND>(A, V, ia, ib, depth_of(b) + kB, Ucur, &ok, &newU, &key);
        warp_bound_update<KIND>(A, ok, 0u, newU);
        const unsigned okm = __ballot_sync(kFull, ok);
        const unsigned nsurv = __popc(okm);
        if (nsurv == 0) return;
        unsigned rank = 0;
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const unsigned kj = __shfl_sync(kFull, key, j);
            rank += ((okm >> j) & 1u) && (kj < key || (kj == key && j < lane));
        }
        const unsigned want = (step == 0 ? w : w / 32u) % nsurv;
        const unsigned m = __ballot_sync(kFull, ok && rank == want);
        const int src = m ? __ffs(m) - 1 : __ffs(okm) - 1;
        a = __shfl_sync(kFull, ia, src);
        b = __shfl_sync(kFull, ib, src);
    }
    probe<KIND>(A, Item{a, b, 0.f, 0u}, V);
}

// A background probe CTA of a single-query launch: it waits (bounded) until
// the query's setup is published, then every warp walks one probe_root from
// the root while the traversal CTAs run their levels; the probes only lower
// the global running bound (and may prove D_min = 0), which the traversal
// reads at its next barrier.  The probes do not use refit boxes: those are
// being written while the probes run.
template <int KIND, class AT>
__device__ void bg_probe_cta(const AT& A) {
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned long long t0 = globaltimer();
        while (!ld_acquire(A.ctr + kCtrSetupDone)) {
            if (ld_relaxed(A.ctr + kCtrAbort)) { ok = 0; break; }
            if ((long long)(globaltimer() - t0) > A.timeout_ns) {
                raise_abort(A);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        if (ok) {
            cta().ready = 0;
            cta_load_query(A);
        }
        s_ok = ok;
    }
    __syncthreads();
    if (!s_ok) return;
    QView V;
    view(A, 0u, V);
    V.dR = -1;
    const unsigned w = (blockIdx.x - work_ctas(A)) * (blockDim.x >> 5) + (threadIdx.x >> 5);
    probe_root<KIND>(A, w, V);
    if (threadIdx.x == 0) atomicAdd(&A.stats->probes, blockDim.x >> 5);
    // Dry runs of the tight leaf bounds and the float64 refinement on
    // triangle pair (0, 0): they only compute, but fetching their code puts it
    // in L2, where the traversal CTAs find it when their leaf and refinement
    // phases start (a cold start from HBM cost those phases ~15 us per query).
    // Small queries skip them: their traversal may end before the dry runs do.
    if (V.LA + V.LB < kDryRunDepth) return;
    __shared__ uint4 dry_list[1];
    if (threadIdx.x == 0) {
        dry_list[0] = make_uint4(0u, 0u, 0u, 0u);
        // the CTA-wide push of the dry run must find nothing to append
        CtaState& c = cta();
        c.cnt[0][0] = c.cnt[0][1] = c.cnt[1][0] = c.cnt[1][1] = 0u;
    }
    __syncthreads();
    int pit = 0;
    unsigned tp = 0;
    unsigned long long by = 0;
    leaf_tight<KIND>(A, dry_list, 1u, pit, tp, by, true);
    V3<double> P, Q;
    int ia, ib;
    const double d = refine_pair_cta<KIND>(A.qs[0], A.qs[0].A->tri, A.qs[0].B->tri, 0u, 0u, &P, &Q, &ia, &ib);
    if (by == 7ull && d == -1.0) atomicAdd(&A.stats->probes, 0u);  // keeps the dry runs live
}

// ------------------------------------------------------------- phase 0

// Widening of a query's float32 map: every mapped coordinate is within
// e_c = gamma_10 (sqrt(3) P_B + |t|_inf) of its exact value; E_box =
// sqrt(3) e_c; the triangle narrow phase adds 256 u X for its own
// arithmetic on coordinates of magnitude <= X; the double-float map
// (including the shift to A's vertex) makes about a dozen roundings of
// relative size 2^-46 on terms of magnitude <= P_A + sqrt(3) P_B + |t|, plus
// the float64 relative map itself.  The inputs are floats, the constants are
// rounded up and every operation rounds up, so each result bounds its
// real-valued expression from above (the 1.000001 factors are margin).
__device__ __forceinline__ void setup_widening(QState& s, float PA, float PB0, float tinf) {
    constexpr float kSqrt3Up = 1.7320509f;        // > sqrt(3)
    constexpr float kGamma10Up = 5.9604682e-07f;  // > 10 u / (1 - 10 u), u = 2^-24
    constexpr float kMarginUp = 1.0000011f;       // > 1.000001
    const float PB = __fmul_ru(PB0, kMarginUp);
    const float reach = __fadd_ru(__fmul_ru(kSqrt3Up, PB), tinf);  // sqrt(3) P_B + |t|_inf
    const float Eb = __fmul_ru(__fmul_ru(kSqrt3Up, __fmul_ru(kGamma10Up, reach)), kMarginUp);
    const float Xm = __fadd_ru(__fmul_ru(fmaxf(PA, reach), kMarginUp), Eb);
    s.E_box = Eb;
    s.E_tri = __fadd_ru(Eb, __fmul_ru(256.f * kU, Xm));
    s.E_df = __fmul_ru(1.0000001e-12f, __fadd_ru(__fadd_ru(PA, reach), 1.f));
}

// The fields of a query's state that the traversal changes, at their
// starting values.
__device__ __forceinline__ void setup_state(QState& s, int kind, unsigned slot_base, int LB, bool refit) {
    s.U = kind == 0 ? kFltMaxBits : 0u;
    s.status = 0u;
    s.best_d = kind == 0 ? 0x7ff0000000000000ull : 0ull;  // +inf / +0
    s.best_key = 0xffffffffffffffffull;
    s.slot_base = slot_base;
    s.dR = refit ? max(0, LB - kRefitH) : -1;
    s.cert = 0u;
    s.pushed[0] = s.pushed[1] = 0u;
}

// The setup of a launch's only query by one warp (every lane calls it).  The
// nine entries of B's rotation in A's frame and the three of its translation
// are independent three-term dot products of A's inverted 3x3 part with B's
// transform, so lanes 0-8 compute one rotation entry each (row lane / 3,
// column lane % 3) and lanes 9-11 one translation entry each.  A float64
// instruction costs the same for one active lane as for a whole warp, and the
// single thread of setup_query evaluating all twelve in turn spent
// microseconds on them.  Lanes 0-8 also hold one entry of the adjugate each;
// the determinant takes the first column from lanes 0, 3 and 6.
__device__ void setup_query_warp(const KArgs& A, int kind) {
    const int lane = threadIdx.x & 31;
    QState& s = A.qs[0];
    const MeshDev* ma;
    const MeshDev* mb;
    const double* xa;
    const double* xb;
    unsigned slot_base = 0;
    if (A.qin) {
        ma = A.qin[0].A; mb = A.qin[0].B;
        xa = A.qin[0].xa; xb = A.qin[0].xb;
        slot_base = A.qin[0].slot_base;
    } else {
        ma = A.mA; mb = A.mB;
        xa = A.xa_src ? A.xa_src : A.xa_val;
        xb = A.xb_src ? A.xb_src : A.xb_val;
    }
    const bool rot = lane < 9, tra = lane >= 9 && lane < 12;
    const int i = rot ? lane / 3 : (tra ? lane - 9 : 0);  // row of A's inverse
    const int j = rot ? lane - 3 * (lane / 3) : 0;        // column (rotation lanes)
    // adjugate entry (i, j) of A's 3x3 part a[r][c] = xa[4 r + c]
    const int r1 = j == 2 ? 0 : j + 1, r2 = j == 0 ? 2 : j - 1;
    const int c1 = i == 2 ? 0 : i + 1, c2 = i == 0 ? 2 : i - 1;
    const double adj = xa[4 * r1 + c1] * xa[4 * r2 + c2] - xa[4 * r1 + c2] * xa[4 * r2 + c1];
    const double det = xa[0] * __shfl_sync(kFull, adj, 0) + xa[1] * __shfl_sync(kFull, adj, 3) +
                       xa[2] * __shfl_sync(kFull, adj, 6);
    const double ai = adj * (1.0 / det);  // entry (i, j) of A's inverse (lanes 0-8)
    const double i0 = __shfl_sync(kFull, ai, 3 * i), i1 = __shfl_sync(kFull, ai, 3 * i + 1),
                 i2 = __shfl_sync(kFull, ai, 3 * i + 2);
    // rotation lanes: column j of B's 3x3 part; translation lanes: t_B - t_A
    const double v0 = tra ? xb[3] - xa[3] : xb[j];
    const double v1 = tra ? xb[7] - xa[7] : xb[4 + j];
    const double v2 = tra ? xb[11] - xa[11] : xb[8 + j];
    const double r = i0 * v0 + i1 * v1 + i2 * v2;
    const float h = (float)r;
    const float lo = (float)(r - (double)h);
    if (rot) {
        s.R[lane] = h;
        s.Rl[lane] = lo;
    } else if (tra) {
        s.t[i] = h;
        s.tl[i] = lo;
    }
    if (lane < 12) {
        s.xa[lane] = xa[lane];
        s.xb[lane] = xb[lane];
    }
    const float tinf = fmaxf(fabsf(__shfl_sync(kFull, h, 9)), fmaxf(fabsf(__shfl_sync(kFull, h, 10)),
                                                                   fabsf(__shfl_sync(kFull, h, 11))));
    if (lane == 0) {
        setup_widening(s, ma->P, mb->P, tinf);
        s.A = ma;
        s.B = mb;
        setup_state(s, kind, slot_base, mb->L, A.refit);
    }
    // every lane's fields are published before the CTA's barrier that
    // precedes the setup flag or the grid barrier
    __threadfence();
    __syncwarp();
}

__device__ void setup_query(const KArgs& A, int q, int kind) {
    QState& s = A.qs[q];
    const MeshDev* ma;
    const MeshDev* mb;
    const double* xa;
    const double* xb;
    unsigned slot_base = 0;
    if (A.qin) {
        ma = A.qin[q].A; mb = A.qin[q].B;
        xa = A.qin[q].xa; xb = A.qin[q].xb;
        slot_base = A.qin[q].slot_base;
    } else {
        ma = A.mA; mb = A.mB;
        xa = A.xa_src ? A.xa_src : A.xa_val;
        xb = A.xb_src ? A.xb_src : A.xb_val;
    }
    double Xa[12], Xb[12];
    for (int i = 0; i < 12; ++i) { Xa[i] = xa[i]; Xb[i] = xb[i]; }
    // inverse of A's 3x3 part (adjugate / determinant)
    double a00 = Xa[0], a01 = Xa[1], a02 = Xa[2], a10 = Xa[4], a11 = Xa[5], a12 = Xa[6];
    double a20 = Xa[8], a21 = Xa[9], a22 = Xa[10];
    double c00 = a11 * a22 - a12 * a21, c01 = a02 * a21 - a01 * a22, c02 = a01 * a12 - a02 * a11;
    double c10 = a12 * a20 - a10 * a22, c11 = a00 * a22 - a02 * a20, c12 = a02 * a10 - a00 * a12;
    double c20 = a10 * a21 - a11 * a20, c21 = a01 * a20 - a00 * a21, c22 = a00 * a11 - a01 * a10;
    double det = a00 * c00 + a01 * c10 + a02 * c20;
    double id = 1.0 / det;
    double Ai[9] = {c00 * id, c01 * id, c02 * id, c10 * id, c11 * id, c12 * id, c20 * id, c21 * id, c22 * id};
    // R = Ai Rb, t = Ai (tb - ta)
    double dt[3] = {Xb[3] - Xa[3], Xb[7] - Xa[7], Xb[11] - Xa[11]};
    float tinf = 0.f;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j) {
            double r = Ai[3 * i] * Xb[j] + Ai[3 * i + 1] * Xb[4 + j] + Ai[3 * i + 2] * Xb[8 + j];
            float h = (float)r;
            s.R[3 * i + j] = h;
            s.Rl[3 * i + j] = (float)(r - (double)h);
        }
        double tt = Ai[3 * i] * dt[0] + Ai[3 * i + 1] * dt[1] + Ai[3 * i + 2] * dt[2];
        float h = (float)tt;
        s.t[i] = h;
        s.tl[i] = (float)(tt - (double)h);
        tinf = fmaxf(tinf, fabsf(h));
    }
    setup_widening(s, ma->P, mb->P, tinf);
    s.A = ma;
    s.B = mb;
    for (int i = 0; i < 12; ++i) { s.xa[i] = Xa[i]; s.xb[i] = Xb[i]; }
    setup_state(s, kind, slot_base, mb->L, A.refit);
}

// ------------------------------------------------------------- phase 2

__device__ __forceinline__ int adaptive_k(unsigned n, long long C, int kmax) {
    int k = 1;
    while (k < kmax && (long long)n << (2 * (k + 1)) < C) ++k;
    return k;
}

template <int KIND, bool FULL, class AT>
__device__ void expand_level(const AT& A, int level, unsigned n, int s, unsigned long long& pairs,
                             unsigned long long& bytes) {
    const Item* in = (level & 1) ? A.front1 : A.front0;
    Item* out = (level & 1) ? A.front0 : A.front1;
    unsigned* out_cnt = A.ctr + kCtrCnt + (level + 1) % 3;
    unsigned* out_rem = A.ctr + kCtrRem + (level + 1) % 3;
    unsigned* leaf_cnt = A.ctr + kCtrLeaf;
    const unsigned long long total = (unsigned long long)n << s;
    const unsigned long long gstride = (unsigned long long)work_ctas(A) * blockDim.x;
    const unsigned long long mask = (1ull << s) - 1;
    const int lane = threadIdx.x & 31;
    QView V;
    // CTA-uniform loop: every thread of a CTA runs the same iterations, so
    // that the appends can be counted per CTA (cta_push2)
    int iter = 0;
    for (unsigned long long cbase = (unsigned long long)blockIdx.x * blockDim.x; cbase < total;
         cbase += gstride, ++iter) {
        unsigned long long vt = cbase + threadIdx.x;
        bool valid = vt < total;
        Item it = {1u, 1u, 0.f, 0u};
        if (valid) {
            float4 raw = __ldcg(reinterpret_cast<const float4*>(in + (vt >> s)));
            it = *reinterpret_cast<Item*>(&raw);
            if (!item_ok(A, it)) {
                flag_bad(A, kBadFront);
                it = Item{1u, 1u, 0.f, 0u};
                valid = false;
            }
        }
        unsigned q = it.q;
        view(A, q, V);
        const int dA = depth_of(it.a), dB = depth_of(it.b);
        int remA = V.LA - dA, remB = V.LB - dB;
        if (remA < 0 || remB < 0) {
            if (valid) flag_bad(A, kBadFront);
            valid = false;
            remA = max(remA, 0);
            remB = max(remB, 0);
        }
        int kA = min((s + 1) >> 1, remA);
        int kB = min(s - kA, remB);
        if (V.dR >= 0 && dB < V.dR) kB = min(kB, V.dR - dB);  // stop on the refit roots
        kA = min(s - kB, remA);
        unsigned local = (unsigned)(vt & mask);
        valid = valid && local < (1u << (kA + kB));
        bool stop;
        float Ucur = load_Uq(A, q, &stop);
        valid = valid && !stop;
        if (KIND == 0) valid = valid && it.bound <= min_keep_threshold(Ucur, V.E_box);
        else valid = valid && it.bound >= max_keep_threshold(Ucur, V.E_box);
        if (valid && local == 0) bytes += 16ull + 24ull * ((1ull << kA) + (1ull << kB));
        unsigned ia = (it.a << kA) | (local >> kB);
        unsigned ib = (it.b << kB) | (local & ((1u << kB) - 1u));
        const int dBc = dB + kB;
        bool leafpair = (kA == remA) && (kB == remB);
        bool survive = false;
        float bound = 0.f;
        unsigned newU = KIND == 0 ? 0xffffffffu : 0u, key;
        if (valid) {
            ++pairs;
            bound = pair_bounds<KIND, FULL>(A, V, ia, ib, dBc, Ucur, &survive, &newU, &key);
        }
        warp_bound_update<KIND>(A, survive, q, newU);
        if (A.q_budget) {
            // a batch query that pushes more than its share of the queues in
            // this level takes the excess from the launch's common pool; when
            // that is spent it leaves the batch (kStatEvict) and runs later
            // with a larger share, so that a few very large queries cannot
            // crowd out the rest (shares plus pool never exceed the queues)
            const unsigned peers = __match_any_sync(kFull, survive ? q : 0xffffffffu);
            const int leader = __ffs(peers) - 1;
            unsigned over = 0u;
            if (survive && lane == leader) {
                const unsigned cnt = __popc(peers);
                const unsigned old = atomicAdd(&A.qs[q].pushed[(level + 1) & 1], cnt);
                if (old + cnt > A.q_budget) {
                    const unsigned pold = atomicAdd(A.ctr + (((level + 1) & 1) ? kCtrPool1 : kCtrPool0), cnt);
                    if (pold + cnt > A.q_pool) {
                        over = 1u;
                        atomicOr(&A.qs[q].status, kStatEvict);
                    }
                }
            }
            if (__shfl_sync(kFull, over, leader)) survive = false;
        }
        Item o = {ia, ib, bound, q};
        if (!cta_push2(iter, o, survive && !leafpair, out, out_cnt, A.cap_front, survive && leafpair, A.leafq,
                       leaf_cnt, A.cap_leaf))
            mark_overflow(A, q);
        if (survive) bytes += 16ull;
        if (survive && !leafpair && dBc == V.dR) claim_root(A, V, q, ib);
        // remaining depth of the entries pushed to the next front
        unsigned rem = (survive && !leafpair) ? (unsigned)(remA - kA + remB - kB) : 0u;
        rem = __reduce_max_sync(kFull, rem);
        if (lane == 0 && rem > 0) atomicMax(&cta().rem, rem);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned r = cta().rem;
        if (r > 0) atomicMax(out_rem, r);
    }
}

// A batch level of one tree level each (s = 2) whose front outgrows the
// grid: one thread per front entry and its (up to) four child pairs, so that
// the entry's load, its query's view and running bound, and the warp's
// collective steps (bound update, queue shares, CTA append) run once per
// entry instead of once per child pair.  Same bounds, survivors and queue
// contents (up to order) as expand_level.
template <int KIND, class AT>
__device__ void expand_level_entries(const AT& A, int level, unsigned n, unsigned long long& pairs,
                                     unsigned long long& bytes) {
    constexpr int s = 2;
    const Item* in = (level & 1) ? A.front1 : A.front0;
    Item* out = (level & 1) ? A.front0 : A.front1;
    unsigned* out_cnt = A.ctr + kCtrCnt + (level + 1) % 3;
    unsigned* out_rem = A.ctr + kCtrRem + (level + 1) % 3;
    unsigned* leaf_cnt = A.ctr + kCtrLeaf;
    const unsigned long long gstride = (unsigned long long)work_ctas(A) * blockDim.x;
    const int lane = threadIdx.x & 31;
    QView V;
    int iter = 0;
    for (unsigned long long cbase = (unsigned long long)blockIdx.x * blockDim.x; cbase < n;
         cbase += gstride, ++iter) {
        const unsigned long long vt = cbase + threadIdx.x;
        bool valid = vt < n;
        Item it = {1u, 1u, 0.f, 0u};
        if (valid) {
            float4 raw = __ldcg(reinterpret_cast<const float4*>(in + vt));
            it = *reinterpret_cast<Item*>(&raw);
            if (!item_ok(A, it)) {
                flag_bad(A, kBadFront);
                it = Item{1u, 1u, 0.f, 0u};
                valid = false;
            }
        }
        const unsigned q = it.q;
        view(A, q, V);
        const int dA = depth_of(it.a), dB = depth_of(it.b);
        int remA = V.LA - dA, remB = V.LB - dB;
        if (remA < 0 || remB < 0) {
            if (valid) flag_bad(A, kBadFront);
            valid = false;
            remA = max(remA, 0);
            remB = max(remB, 0);
        }
        int kA = min((s + 1) >> 1, remA);
        int kB = min(s - kA, remB);
        if (V.dR >= 0 && dB < V.dR) kB = min(kB, V.dR - dB);  // stop on the refit roots
        kA = min(s - kB, remA);
        bool stop;
        const float Ucur = load_Uq(A, q, &stop);
        valid = valid && !stop;
        if (KIND == 0) valid = valid && it.bound <= min_keep_threshold(Ucur, V.E_box);
        else valid = valid && it.bound >= max_keep_threshold(Ucur, V.E_box);
        if (valid) bytes += 16ull + 24ull * ((1ull << kA) + (1ull << kB));
        const int dBc = dB + kB;
        const bool leafpair = (kA == remA) && (kB == remB);
        const unsigned nchild = valid ? 1u << (kA + kB) : 0u;
        // the children (child c: A's child c >> kB, B's child c & (2^kB - 1)),
        // their survivors (bit c of sm) and the best enhanced bound among them
        Item o[4];
        unsigned sm = 0u;
        unsigned best = KIND == 0 ? 0xffffffffu : 0u;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const unsigned ia = (it.a << kA) | ((unsigned)c >> kB);
            const unsigned ib = (it.b << kB) | ((unsigned)c & ((1u << kB) - 1u));
            o[c] = Item{ia, ib, 0.f, q};
            if ((unsigned)c < nchild) {
                ++pairs;
                bool survive = false;
                unsigned newU = KIND == 0 ? 0xffffffffu : 0u, key;
                o[c].bound = pair_bounds<KIND, false>(A, V, ia, ib, dBc, Ucur, &survive, &newU, &key);
                if (survive) {
                    sm |= 1u << c;
                    best = KIND == 0 ? min(best, newU) : max(best, newU);
                }
            }
        }
        warp_bound_update<KIND>(A, sm != 0u, q, best);
        if (A.q_budget) {
            // the queue shares (as in expand_level), one atomic per query
            // among the warp's lanes with survivors
            bool pend = sm != 0u;
            for (;;) {
                const unsigned pm = __ballot_sync(kFull, pend);
                if (!pm) break;
                const int leader = __ffs(pm) - 1;
                const unsigned lq = __shfl_sync(kFull, q, leader);
                const bool mine = pend && q == lq;
                const unsigned tot = __reduce_add_sync(kFull, mine ? (unsigned)__popc(sm) : 0u);
                unsigned over = 0u;
                if (lane == leader) {
                    const unsigned old = atomicAdd(&A.qs[lq].pushed[(level + 1) & 1], tot);
                    if (old + tot > A.q_budget) {
                        const unsigned pold = atomicAdd(A.ctr + (((level + 1) & 1) ? kCtrPool1 : kCtrPool0), tot);
                        if (pold + tot > A.q_pool) {
                            over = 1u;
                            atomicOr(&A.qs[lq].status, kStatEvict);
                        }
                    }
                }
                over = __shfl_sync(kFull, over, leader);
                if (mine) {
                    pend = false;
                    if (over) sm = 0u;
                }
            }
        }
        if (!cta_push4(iter, o, sm, leafpair, out, out_cnt, A.cap_front, A.leafq, leaf_cnt, A.cap_leaf))
            mark_overflow(A, q);
        bytes += 16ull * (unsigned)__popc(sm);
        if (!leafpair && dBc == V.dR) {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if ((sm >> c) & 1u) claim_root(A, V, q, o[c].b);
        }
        // remaining depth of the entries pushed to the next front
        unsigned rem = (sm != 0u && !leafpair) ? (unsigned)(remA - kA + remB - kB) : 0u;
        rem = __reduce_max_sync(kFull, rem);
        if (lane == 0 && rem > 0) atomicMax(&cta().rem, rem);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned r = cta().rem;
        if (r > 0) atomicMax(out_rem, r);
    }
}

// ------------------------------------------------------------- phase 3

// Single-query launches: merge the global running bound and status word
// (read earlier into w by thread 0) into the CTA's copy.  The leaf phase has
// no grid barrier to refresh that copy, so without this a CTA would not see
// the other CTAs' bounds, nor a D = 0 proof, until the phase ended.
template <int KIND>
__device__ __forceinline__ void cta_merge_bound(unsigned long long w) {
    CtaState& c = cta();
    if (KIND == 0) atomicMin(&c.U, (unsigned)w);
    else atomicMax(&c.U, (unsigned)w);
    const unsigned st = (unsigned)(w >> 32) & kStatStop;
    if (st) atomicOr(&c.stat, st);
}

// Tight bounds of the triangle pairs queued in the CTA's list (thread i takes
// entry i < n; every thread calls, for the CTA-wide push): running-bound
// update, candidates, and the D = 0 check of a pair that may touch.  One
// compiled copy (not inlined), so that a dry run (dry: bounds only, no side
// effect) by a background CTA early in the launch brings its code into L2
// before the leaf phase needs it.  It keeps a query view of its own: a view
// passed in by reference would live in local memory in the caller, whose
// slot loop re-fills it for every query change of a batch.
template <int KIND, class AT>
__device__ __noinline__ void leaf_tight(const AT& A, const uint4* list, unsigned n, int& pit, unsigned& tripairs,
                                        unsigned long long& bytes, bool dry) {
    QView V;
    bool have = false, emit = false;
    float cb = 0.f;
    unsigned newU = KIND == 0 ? 0xffffffffu : 0u;
    unsigned ta = 0u, tb = 0u, q = 0u;
    if (threadIdx.x < n) {
        const uint4 e = list[threadIdx.x];
        ta = e.x; tb = e.y; q = e.z;
        view(A, q, V);
        bool stop;
        const float Ucur = load_Uq(A, q, &stop);
        if (!stop) {
            const Tri32 TA = load_tri(V.triA, ta), TB = load_tri(V.triB, tb);
            // the bound may have moved since the pair was queued: test again
            if (dry || tri_pair_may_hold<KIND>(V, TA, TB, Ucur, !AT::kOne)) {
                ++tripairs;
                float lo, up;
                tri_pair_bounds_tight<KIND>(A, q, V, TA, TB, &lo, &up);
                have = true;
                if (KIND == 0) {
                    newU = __float_as_uint(up);
                    cb = lo;
                    emit = lo <= fminf(Ucur, up);
                } else {
                    newU = __float_as_uint(lo);
                    cb = up;
                    emit = up >= fmaxf(Ucur, lo);
                }
            }
        }
    }
    if (dry) {
        // keep the result live so that the bounds are computed, then run the
        // rest with nothing to publish (no bound, no candidate, no D = 0 check)
        if (have && cb == 1.2345678e-30f) bytes += 1ull;
        have = false;
        emit = false;
    }
    warp_bound_update<KIND>(A, have, q, newU);
    Cand c = {ta, tb, cb, q};
    if (!cta_push2(pit++, c, emit, A.cand, A.ctr + kCtrCand, A.cap_cand, false, (Cand*)nullptr, (unsigned*)nullptr,
                   0u))
        mark_overflow(A, q);
    if (emit) bytes += 16ull;
    if (KIND == 0) {
        // a pair that may touch: try to prove D_min = 0 with it
        const unsigned m = __ballot_sync(kFull, emit && cb <= 0.f);
        if (m) {
            const int src = __ffs(m) - 1;
            certify_zero(A, __shfl_sync(kFull, q, src), __shfl_sync(kFull, ta, src), __shfl_sync(kFull, tb, src));
        }
    }
}

// The CTA's list of triangle pairs waiting for their tight bounds (both
// forms of the leaf phase use it; it holds 3 kBlock entries).
__device__ __forceinline__ uint4* leaf_list() {
    __shared__ uint4 l[3 * kBlock];
    return l;
}

__device__ __forceinline__ unsigned& leaf_list_n() {
    __shared__ unsigned n;
    return n;
}

// The leaf pairs' triangle pairs, 4 slots per leaf pair (<= 2 x 2 triangles),
// in two stages per CTA: every thread takes one slot, loads its two
// triangles and runs the cheap float32 test; the pairs that pass go to a
// list in shared memory, and whenever it holds a CTA's worth (and at the
// end) every thread takes one listed pair for the tight bounds.  Only a few
// per cent of the pairs pass the cheap test, so bounding them densely keeps
// whole warps on the expensive part instead of one lane in each.
template <int KIND, class AT>
__device__ void leaf_phase_slots(const AT& A, unsigned nleaf, unsigned& tripairs, unsigned long long& bytes) {
    // slots per thread and iteration (two, measured for single queries: the
    // leaf phase took 17.2 -> 18.3 us on the rings; one kept)
    constexpr int U = 1;
    uint4* list = leaf_list();
    unsigned& list_n = leaf_list_n();
    const unsigned long long total = (unsigned long long)nleaf * 4ull;
    const unsigned long long gstride = (unsigned long long)work_ctas(A) * blockDim.x;
    const bool pull = AT::kOne && threadIdx.x == 0;
    const int lane = threadIdx.x & 31;
    // the plane axes of the cheap test pay off on queues longer than one pass
    // (a rings query, one pass, lost 1.8 us of leaf phase with them)
    const bool planes = total > gstride;
    // the query's constants: a single query reads the CTA's shared copy where
    // it uses them (no per-thread copy held through the slot loop); a batch
    // keeps a per-thread view of the last query it met
    QView Vb;
    int pit = 0;
    if (threadIdx.x == 0) list_n = 0u;
    for (unsigned long long cbase = (unsigned long long)blockIdx.x * blockDim.x; cbase < total; cbase += U * gstride) {
        // a single query whose traversal stopped (D = 0 proven) skips the rest
        // (this barrier also publishes list_n)
        if (__syncthreads_or(AT::kOne && (((volatile CtaState&)cta()).stat & kStatStop) != 0u)) break;
        // issued now, merged at the end of the iteration (the load's latency
        // hides behind this iteration's work)
        unsigned long long gw = 0;
        if (pull) gw = ld_relaxed64(reinterpret_cast<const unsigned long long*>(&A.qs[0].U));
        // the slots' queue entries first (independent loads), then their tests
        Item it[U];
        bool valid[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const unsigned long long vt = cbase + (unsigned long long)u * gstride + threadIdx.x;
            valid[u] = vt < total;
            it[u] = Item{1u, 1u, 0.f, 0u};
            if (valid[u]) {
                float4 raw = __ldcg(reinterpret_cast<const float4*>(A.leafq + (vt >> 2)));
                it[u] = *reinterpret_cast<Item*>(&raw);
            }
        }
        unsigned ta[U], tb[U], q[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const unsigned long long vt = cbase + (unsigned long long)u * gstride + threadIdx.x;
            if (valid[u] && !item_ok(A, it[u])) {
                flag_bad(A, kBadLeaf);
                it[u] = Item{1u, 1u, 0.f, 0u};
                valid[u] = false;
            }
            q[u] = it[u].q;
            if (!AT::kOne) view(A, q[u], Vb);
            const QConst& V = AT::kOne ? static_cast<const QConst&>(cta().v) : static_cast<const QConst&>(Vb);
            if (valid[u] && (depth_of(it[u].a) != V.LA || depth_of(it[u].b) != V.LB)) {
                flag_bad(A, kBadLeaf);
                valid[u] = false;
            }
            const unsigned sub = (unsigned)(vt & 3);
            const unsigned la = it[u].a - (1u << V.LA), lb = it[u].b - (1u << V.LB);
            const unsigned a0 = leaf_first(V.TA, V.LA, la), a1 = leaf_first(V.TA, V.LA, la + 1);
            const unsigned b0 = leaf_first(V.TB, V.LB, lb), b1 = leaf_first(V.TB, V.LB, lb + 1);
            ta[u] = a0 + (sub >> 1);
            tb[u] = b0 + (sub & 1);
            valid[u] = valid[u] && ta[u] < a1 && tb[u] < b1;
            bool stop;
            const float Ucur = load_Uq(A, q[u], &stop);
            valid[u] = valid[u] && !stop;
            if (KIND == 0) valid[u] = valid[u] && it[u].bound <= min_keep_threshold(Ucur, V.E_box);
            else valid[u] = valid[u] && it[u].bound >= max_keep_threshold(Ucur, V.E_box);
            if (valid[u] && sub == 0) bytes += 16ull + 36ull * ((a1 - a0) + (b1 - b0));
            if (valid[u]) {
                const Tri32 TA = load_tri(V.triA, ta[u]), TB = load_tri(V.triB, tb[u]);
                valid[u] = tri_pair_may_hold<KIND>(V, TA, TB, Ucur, planes);
            }
        }
        // queue the pairs that passed (one shared atomic per warp and slot);
        // the list holds < kBlock entries between iterations, so it never
        // overflows
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const unsigned m = __ballot_sync(kFull, valid[u]);
            unsigned base = 0u;
            if (lane == 0 && m) base = atomicAdd(&list_n, (unsigned)__popc(m));
            base = __shfl_sync(kFull, base, 0);
            if (valid[u]) list[base + __popc(m & lanemask_lt())] = make_uint4(ta[u], tb[u], q[u], 0u);
        }
        __syncthreads();
        unsigned n = list_n;
        while (n >= (unsigned)kBlock) {
            leaf_tight<KIND>(A, list + (n - kBlock), kBlock, pit, tripairs, bytes, false);
            __syncthreads();
            n -= kBlock;
            if (threadIdx.x == 0) list_n = n;
        }
        if (pull) cta_merge_bound<KIND>(gw);
    }
    __syncthreads();
    const unsigned n = list_n;
    if (n > 0u) leaf_tight<KIND>(A, list, n, pit, tripairs, bytes, false);
    __syncthreads();
}

// The same two stages with one thread per leaf pair: it loads the pair's
// (up to) 2 + 2 triangles, maps each of B's into A's frame once, and runs the
// cheap test on its (up to) four triangle pairs.  The passing pairs reach the
// list in two pushes of two between CTA barriers, so that it holds fewer
// than kBlock + 2 kBlock entries before a drain.
template <int KIND, class AT>
__device__ void leaf_phase_pairs(const AT& A, unsigned nleaf, unsigned& tripairs, unsigned long long& bytes) {
    uint4* list = leaf_list();
    unsigned& list_n = leaf_list_n();
    const unsigned long long gstride = (unsigned long long)work_ctas(A) * blockDim.x;
    const bool pull = AT::kOne && threadIdx.x == 0;
    const int lane = threadIdx.x & 31;
    QView Vb;
    int pit = 0;
    if (threadIdx.x == 0) list_n = 0u;
    for (unsigned long long cbase = (unsigned long long)blockIdx.x * blockDim.x; cbase < nleaf; cbase += gstride) {
        if (__syncthreads_or(AT::kOne && (((volatile CtaState&)cta()).stat & kStatStop) != 0u)) break;
        unsigned long long gw = 0;
        if (pull) gw = ld_relaxed64(reinterpret_cast<const unsigned long long*>(&A.qs[0].U));
        const unsigned long long vt = cbase + threadIdx.x;
        bool valid = vt < nleaf;
        Item it = Item{1u, 1u, 0.f, 0u};
        if (valid) {
            float4 raw = __ldcg(reinterpret_cast<const float4*>(A.leafq + vt));
            it = *reinterpret_cast<Item*>(&raw);
            if (!item_ok(A, it)) {
                flag_bad(A, kBadLeaf);
                it = Item{1u, 1u, 0.f, 0u};
                valid = false;
            }
        }
        const unsigned q = it.q;
        if (!AT::kOne) view(A, q, Vb);
        const QConst& V = AT::kOne ? static_cast<const QConst&>(cta().v) : static_cast<const QConst&>(Vb);
        if (valid && (depth_of(it.a) != V.LA || depth_of(it.b) != V.LB)) {
            flag_bad(A, kBadLeaf);
            valid = false;
        }
        const unsigned la = it.a - (1u << V.LA), lb = it.b - (1u << V.LB);
        const unsigned a0 = leaf_first(V.TA, V.LA, la), a1 = leaf_first(V.TA, V.LA, la + 1);
        const unsigned b0 = leaf_first(V.TB, V.LB, lb), b1 = leaf_first(V.TB, V.LB, lb + 1);
        valid = valid && a0 < a1 && b0 < b1;
        bool stop;
        const float Ucur = load_Uq(A, q, &stop);
        valid = valid && !stop;
        if (KIND == 0) valid = valid && it.bound <= min_keep_threshold(Ucur, V.E_box);
        else valid = valid && it.bound >= max_keep_threshold(Ucur, V.E_box);
        // bit 2i + j: triangle pair (a0 + i, b0 + j) passed the cheap test
        unsigned m = 0u;
        if (valid) {
            bytes += 16ull + 36ull * ((a1 - a0) + (b1 - b0));
            const bool a2 = a1 - a0 >= 2u, b2 = b1 - b0 >= 2u;
            const Tri32 TA0 = load_tri(V.triA, a0), TA1 = load_tri(V.triA, a2 ? a0 + 1u : a0);
            const Tri32 TB0 = load_tri(V.triB, b0), TB1 = load_tri(V.triB, b2 ? b0 + 1u : b0);
            // B's triangles mapped once each, one at a time
            V3<float> Bw[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) Bw[k] = map32(V.X, TB0.v[k].x, TB0.v[k].y, TB0.v[k].z);
            if (tri_pair_may_hold_mapped<KIND>(V.E_box, TA0, Bw, Ucur, true)) m |= 1u;
            if (a2 && tri_pair_may_hold_mapped<KIND>(V.E_box, TA1, Bw, Ucur, true)) m |= 4u;
            if (b2) {
#pragma unroll
                for (int k = 0; k < 3; ++k) Bw[k] = map32(V.X, TB1.v[k].x, TB1.v[k].y, TB1.v[k].z);
                if (tri_pair_may_hold_mapped<KIND>(V.E_box, TA0, Bw, Ucur, true)) m |= 2u;
                if (a2 && tri_pair_may_hold_mapped<KIND>(V.E_box, TA1, Bw, Ucur, true)) m |= 8u;
            }
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
#pragma unroll
            for (int r = 2 * h; r < 2 * h + 2; ++r) {
                const bool p = (m >> r) & 1u;
                const unsigned mb = __ballot_sync(kFull, p);
                unsigned base = 0u;
                if (lane == 0 && mb) base = atomicAdd(&list_n, (unsigned)__popc(mb));
                base = __shfl_sync(kFull, base, 0);
                if (p) list[base + __popc(mb & lanemask_lt())] = make_uint4(a0 + (r >> 1), b0 + (r & 1), q, 0u);
            }
            __syncthreads();
            unsigned n = list_n;
            if (n >= (unsigned)kBlock) {
                while (n >= (unsigned)kBlock) {
                    leaf_tight<KIND>(A, list + (n - kBlock), kBlock, pit, tripairs, bytes, false);
                    __syncthreads();
                    n -= kBlock;
                }
                if (threadIdx.x == 0) list_n = n;
            }
            // every thread has read list_n before the next push changes it
            __syncthreads();
        }
        if (pull) cta_merge_bound<KIND>(gw);
    }
    __syncthreads();
    const unsigned n = list_n;
    if (n > 0u) leaf_tight<KIND>(A, list, n, pit, tripairs, bytes, false);
    __syncthreads();
}

// The leaf phase.  A batch whose queue needs more than one pass of slots (4
// slots per leaf pair, one per thread) runs the form with a thread per leaf
// pair, which loads each triangle and maps each of B's once instead of twice
// (gear batch of 512 queries: 94 -> 75 ms).  A single query keeps the slot
// form, the shortest chain per thread: the per-pair form in its kernel, even
// out of line and taken only for long queues, cost the rings and icosphere
// queries 2-4 % (registers of the rest of the kernel) for 3 % on the gears'
// plain calls.
template <int KIND, class AT>
__device__ void leaf_phase(const AT& A, unsigned nleaf, unsigned& tripairs, unsigned long long& bytes) {
    const unsigned long long threads = (unsigned long long)work_ctas(A) * blockDim.x;
    if (!AT::kOne && 4ull * nleaf > threads) leaf_phase_pairs<KIND>(A, nleaf, tripairs, bytes);
    else leaf_phase_slots<KIND>(A, nleaf, tripairs, bytes);
}

// ------------------------------------------------------------- phases 4-6

// float64 distance of one triangle pair in the world frame, computed by a whole
// warp.  Min kind: lane f owns feature pair f of tri_feature (21 lanes).  A
// float32 pass on local coordinates first bounds every feature from both
// sides (upper: its closest pair; lower: separation of its two point sets,
// or the plane gap for an edge that does not cross the other plane); only
// features whose lower bound does not exceed the best upper bound can hold
// the minimum, and only those run in float64.  Max kind: lane v < 9 owns one
// vertex pair.  Every lane returns the warp's result; P, Q are a closest
// (farthest) pair, *ida, *idb the original triangle indices.
template <int KIND>
__device__ __noinline__ double refine_pair_warp(const QState& s, unsigned ta, unsigned tb, V3<double>* P,
                                                V3<double>* Q, int* ida, int* idb) {
    const int lane = threadIdx.x & 31;
    Tri32 TA = load_tri(s.A->tri, ta), TB = load_tri(s.B->tri, tb);
    *ida = TA.id;
    *idb = TB.id;
    // lanes 0..5 map one vertex each, then share them
    V3<double> w = mk3(0.0, 0.0, 0.0);
    if (lane < 3) w = map64(s.xa, (double)TA.v[lane].x, (double)TA.v[lane].y, (double)TA.v[lane].z);
    else if (lane < 6)
        w = map64(s.xb, (double)TB.v[lane - 3].x, (double)TB.v[lane - 3].y, (double)TB.v[lane - 3].z);
    V3<double> Aw[3], Bw[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        Aw[k] = mk3(__shfl_sync(kFull, w.x, k), __shfl_sync(kFull, w.y, k), __shfl_sync(kFull, w.z, k));
        Bw[k] = mk3(__shfl_sync(kFull, w.x, 3 + k), __shfl_sync(kFull, w.y, 3 + k), __shfl_sync(kFull, w.z, 3 + k));
    }
    V3<double> p = Aw[0], qq = Bw[0];
    double d2 = INFINITY;
    bool hit = false;
    if (KIND == 0) {
        // float32 pre-pass on coordinates local to A's first vertex
        V3<float> Al[3], Bl[3];
        float X = 0.f;
        double W = 0.0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            V3<double> a = Aw[k] - Aw[0], b = Bw[k] - Aw[0];
            Al[k] = mk3((float)a.x, (float)a.y, (float)a.z);
            Bl[k] = mk3((float)b.x, (float)b.y, (float)b.z);
            X = fmaxf(X, fmaxf(max_abs3(Al[k]), max_abs3(Bl[k])));
            W = fmax(W, fmax(fmax(fabs(Aw[k].x), fabs(Aw[k].y)), fabs(Aw[k].z)));
            W = fmax(W, fmax(fmax(fabs(Bw[k].x), fabs(Bw[k].y)), fabs(Bw[k].z)));
        }
        const float E = __fadd_ru(__double2float_ru(1e-15 * (W + 1.0)), __fmul_ru(256.0f * kU * 1.001f, X));
        float upf = INFINITY, lof = INFINITY;
        if (lane < 21) {
            V3<float> p32, q32;
            float d32;
            bool h32;
            tri_feature(lane, Al, Bl, &p32, &q32, &d32, &h32);
            V3<float> FA[3], FB[3];
            feature_points(lane, Al, Bl, FA, FB);
            if (d32 < INFINITY) {
                upf = upper_from_sq(d32, E);
                lof = 0.f;
                V3<float> n = p32 - q32;
                float nn = dot(n, n);
                if (!h32 && nn > 0.f) {
                    float amin = FLT_MAX, bmax = -FLT_MAX;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        amin = fminf(amin, dot(n, FA[k]));
                        bmax = fmaxf(bmax, dot(n, FB[k]));
                    }
                    if (amin - bmax > 0.f) lof = lower_from_dist((amin - bmax) / sqrtf(nn), E);
                }
            } else {
                // an edge that does not cross the other triangle's plane: the
                // plane keeps it at least its nearer endpoint's plane distance away
                const bool ea = lane < 18;
                const V3<float>* F = ea ? Bl : Al;
                const V3<float>* Ed = ea ? FA : FB;
                V3<float> n = cross(F[1] - F[0], F[2] - F[0]);
                float nn = dot(n, n);
                lof = 0.f;
                if (nn > 0.f) {
                    float s0 = dot(n, Ed[0] - F[0]), s1 = dot(n, Ed[1] - F[0]);
                    if ((s0 > 0.f && s1 > 0.f) || (s0 < 0.f && s1 < 0.f))
                        lof = lower_from_dist(fminf(fabsf(s0), fabsf(s1)) / sqrtf(nn), E);
                }
            }
        }
        // non-negative floats order like their bit patterns
        const float minUp = __uint_as_float(__reduce_min_sync(kFull, __float_as_uint(upf)));
        if (lane < 21 && lof <= minUp) tri_feature(lane, Aw, Bw, &p, &qq, &d2, &hit);
    } else {
        if (lane < 9) {
            p = Aw[lane / 3];
            qq = Bw[lane % 3];
            V3<double> d = p - qq;
            d2 = -dot(d, d);  // reduce with min
        }
    }
    const unsigned hits = __ballot_sync(kFull, hit);
    int win;
    double best;
    if (hits) {
        win = __ffs(hits) - 1;
        best = 0.0;
    } else {
        // (d2, lane) lexicographic minimum over the warp
        best = d2;
        win = lane;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            double ob = __shfl_xor_sync(kFull, best, o);
            int ow = __shfl_xor_sync(kFull, win, o);
            if (ob < best || (ob == best && ow < win)) { best = ob; win = ow; }
        }
    }
    P->x = __shfl_sync(kFull, p.x, win); P->y = __shfl_sync(kFull, p.y, win); P->z = __shfl_sync(kFull, p.z, win);
    Q->x = __shfl_sync(kFull, qq.x, win); Q->y = __shfl_sync(kFull, qq.y, win); Q->z = __shfl_sync(kFull, qq.z, win);
    if (KIND == 0) return hits ? 0.0 : sqrt(best);
    return sqrt(-best);
}

// float64 refinement, one warp per candidate (warps first_warp, +wstride, ...)
// float64 distance of one triangle pair computed by three warps of a CTA, one
// per kind of feature pair: warp 0 the 9 edge-edge pairs, warp 1 the 6
// vertex-face pairs, warp 2 the 6 edge-plane crossings (max kind: warp 0, the
// 9 vertex pairs).  All features run in float64 at once, so the three kinds
// do not wait for one another as they do in one warp, and no float32 pass is
// needed.  The per-feature arithmetic is the explicitly rounded float64 of
// tri_feature and the winner is the same (hit first, else the smallest
// (d2, feature)), so the result equals refine_pair_warp's bit for bit.  Every
// thread of the CTA calls it; the result (return value, P, Q) is valid in
// warp 0, *ida and *idb on every thread.
template <int KIND>
__device__ __noinline__ double refine_pair_cta(const QState& s, const float4* triA, const float4* triB, unsigned ta,
                                               unsigned tb, V3<double>* P, V3<double>* Q, int* ida, int* idb) {
    __shared__ double s_d2[3];
    __shared__ int s_f[3];
    __shared__ double s_pq[3][6];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Tri32 TA = load_tri(triA, ta), TB = load_tri(triB, tb);
    *ida = TA.id;
    *idb = TB.id;
    __syncthreads();  // the shared results of a previous pair have been read
    if (warp < 3) {
        V3<double> w = mk3(0.0, 0.0, 0.0);
        if (lane < 3) w = map64(s.xa, (double)TA.v[lane].x, (double)TA.v[lane].y, (double)TA.v[lane].z);
        else if (lane < 6)
            w = map64(s.xb, (double)TB.v[lane - 3].x, (double)TB.v[lane - 3].y, (double)TB.v[lane - 3].z);
        V3<double> Aw[3], Bw[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            Aw[k] = mk3(__shfl_sync(kFull, w.x, k), __shfl_sync(kFull, w.y, k), __shfl_sync(kFull, w.z, k));
            Bw[k] = mk3(__shfl_sync(kFull, w.x, 3 + k), __shfl_sync(kFull, w.y, 3 + k),
                        __shfl_sync(kFull, w.z, 3 + k));
        }
        V3<double> p = Aw[0], qq = Bw[0];
        double d2 = INFINITY;
        bool hit = false;
        int f = 99;
        if (KIND == 0) {
            const bool on = warp == 0 ? lane < 9 : lane < 6;
            f = warp == 0 ? lane : (warp == 1 ? 9 + lane : 15 + lane);
            if (on) tri_feature(f, Aw, Bw, &p, &qq, &d2, &hit);
            else f = 99;
        } else if (warp == 0 && lane < 9) {
            p = Aw[lane / 3];
            qq = Bw[lane % 3];
            const V3<double> d = p - qq;
            d2 = -dot(d, d);  // reduce with min
            f = lane;
        }
        const unsigned hits = __ballot_sync(kFull, hit);
        double best;
        int win;
        if (hits) {
            win = __ffs(hits) - 1;
            best = -1.0;  // marks a hit
        } else if (KIND == 0) {
            // the values are non-negative (or +inf): their bit patterns order
            // like them, so the (d2, lane) minimum takes integer compares
            // (float64 compares issue on the float64 pipe)
            unsigned long long key = (unsigned long long)__double_as_longlong(d2);
            win = lane;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long ok = __shfl_xor_sync(kFull, key, o);
                const int ow = __shfl_xor_sync(kFull, win, o);
                if (ok < key || (ok == key && ow < win)) { key = ok; win = ow; }
            }
            best = __longlong_as_double((long long)key);
        } else {
            best = d2;
            win = lane;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double ob = __shfl_xor_sync(kFull, best, o);
                const int ow = __shfl_xor_sync(kFull, win, o);
                if (ob < best || (ob == best && ow < win)) { best = ob; win = ow; }
            }
        }
        const double px = __shfl_sync(kFull, p.x, win), py = __shfl_sync(kFull, p.y, win),
                     pz = __shfl_sync(kFull, p.z, win), qx = __shfl_sync(kFull, qq.x, win),
                     qy = __shfl_sync(kFull, qq.y, win), qz = __shfl_sync(kFull, qq.z, win);
        const int fw = __shfl_sync(kFull, f, win);
        if (lane == 0) {
            s_d2[warp] = (KIND == 0 && hits) ? -1.0 : best;
            s_f[warp] = fw;
            s_pq[warp][0] = px; s_pq[warp][1] = py; s_pq[warp][2] = pz;
            s_pq[warp][3] = qx; s_pq[warp][4] = qy; s_pq[warp][5] = qz;
        }
    }
    __syncthreads();
    // the result is taken from thread 0: the other warps leave the float64
    // selection and square root to warp 0 (a float64 instruction occupies
    // its SM sub-partition's float64 pipe as long for one warp as for any
    // other, so eight warps computing it would queue on those pipes)
    if (warp != 0) return 0.0;
    // min kind: a hit (-1) wins, the smallest feature index first; otherwise
    // the smallest (d2, feature).  Max kind: the values are -d2.
    int bw = 0;
    for (int k = 1; k < 3; ++k) {
        const bool better = s_d2[k] < s_d2[bw] || (s_d2[k] == s_d2[bw] && s_f[k] < s_f[bw]);
        if (better) bw = k;
    }
    const double best = s_d2[bw];
    P->x = s_pq[bw][0]; P->y = s_pq[bw][1]; P->z = s_pq[bw][2];
    Q->x = s_pq[bw][3]; Q->y = s_pq[bw][4]; Q->z = s_pq[bw][5];
    if (KIND == 0) return best < 0.0 ? 0.0 : sqrt(best);
    return sqrt(-best);
}

// The refinement by CTAs: thread t of CTA c tests candidate c + t W (+ 256 W
// per round) against the running bound, the kept ones are listed in shared
// memory, and the CTA refines them one after another with refine_pair_cta.
// Every candidate's float64 distance (NaN when not kept) and points are
// stored, the per-query extreme is raised or lowered, and the refined
// candidates are listed for the selection.
template <int KIND, class AT>
__device__ void refine_phase_cta(const AT& A, unsigned ncand, unsigned& refined, unsigned long long& bytes) {
    __shared__ unsigned s_list[kBlock];
    __shared__ unsigned s_n;
    const unsigned long long W = work_ctas(A);
    for (unsigned long long base = blockIdx.x; base < ncand; base += W * blockDim.x) {
        if (threadIdx.x == 0) s_n = 0u;
        __syncthreads();
        const unsigned long long i = base + (unsigned long long)threadIdx.x * W;
        if (i < ncand) {
            float4 raw = __ldcg(reinterpret_cast<const float4*>(A.cand + i));
            const Cand c = *reinterpret_cast<Cand*>(&raw);
            bool keep = false;
            // a single query checks against the CTA's copies of its constants
            // and status (refreshed at the barrier before this phase), not
            // through dependent global loads
            const bool bad = AT::kOne ? (c.q != 0u || c.ta >= (unsigned long long)cta().v.TA ||
                                         c.tb >= (unsigned long long)cta().v.TB)
                                      : (c.q >= (unsigned)A.nq ||
                                         c.ta >= (unsigned)A.qs[c.q < (unsigned)A.nq ? c.q : 0].A->T ||
                                         c.tb >= (unsigned)A.qs[c.q < (unsigned)A.nq ? c.q : 0].B->T);
            if (bad) {
                flag_bad(A, kBadCand);
            } else {
                bool stop;
                const float U = load_Uq(A, c.q, &stop);
                const unsigned st = AT::kOne ? ((volatile CtaState&)cta()).stat : ld_relaxed(&A.qs[c.q].status);
                // once D_min = 0 is proven only the proving pair (bound -1) is
                // refined; an evicted query is answered by its own launch later
                keep = KIND == 0 ? (stop ? (st & kStatZero) && c.bound < 0.f : c.bound <= U)
                                 : (!stop && c.bound >= U);
            }
            if (keep) s_list[atomicAdd(&s_n, 1u)] = (unsigned)i;
            else A.cand_d[i] = __longlong_as_double(-1ll);  // NaN: never selected
        }
        __syncthreads();
        const unsigned n = s_n;
        for (unsigned k = 0; k < n; ++k) {
            const unsigned ci = s_list[k];
            float4 raw = __ldcg(reinterpret_cast<const float4*>(A.cand + ci));
            const Cand c = *reinterpret_cast<Cand*>(&raw);
            QState& s = A.qs[c.q];
            V3<double> P, Q;
            int ia, ib;
            // (a single query's triangle arrays from the CTA's copy: two
            // dependent loads fewer before the triangles)
            const float4* tA = AT::kOne ? cta().v.triA : s.A->tri;
            const float4* tB = AT::kOne ? cta().v.triB : s.B->tri;
            const double d = refine_pair_cta<KIND>(s, tA, tB, c.ta, c.tb, &P, &Q, &ia, &ib);
            if (threadIdx.x == 0) {
                double* w = A.cand_pts + 6ull * ci;
                w[0] = P.x; w[1] = P.y; w[2] = P.z; w[3] = Q.x; w[4] = Q.y; w[5] = Q.z;
                const unsigned r = atomicAdd(A.ctr + kCtrRefined, 1u);
                if (r < 4ull * A.cap_leaf) reinterpret_cast<unsigned*>(A.leafq)[r] = ci;
                const unsigned long long bits = (unsigned long long)__double_as_longlong(d);
                if (KIND == 0) atomicMin(&s.best_d, bits);
                else atomicMax(&s.best_d, bits);
                A.cand_d[ci] = d;
                ++refined;
                bytes += 16ull + 72ull;
            }
        }
        __syncthreads();
    }
}

// The candidates to scan after the refinement: the list of refined ones when
// it is complete, else all ncand.
struct RefinedSet {
    const unsigned* list;
    unsigned n;
    __device__ __forceinline__ unsigned at(unsigned k) const { return list ? __ldcg(list + k) : k; }
};

__device__ __forceinline__ RefinedSet refined_set(const KArgs& A, unsigned nrefined, unsigned ncand) {
    if ((unsigned long long)nrefined <= 4ull * A.cap_leaf)
        return RefinedSet{reinterpret_cast<const unsigned*>(A.leafq), nrefined};
    return RefinedSet{nullptr, ncand};
}

__device__ void select_phase(const KArgs& A, RefinedSet R, unsigned long long first, unsigned long long gstride) {
    for (unsigned long long k = first; k < R.n; k += gstride) {
        const unsigned i = R.at((unsigned)k);
        if (i >= A.cap_cand) continue;
        double d = __ldcg(A.cand_d + i);
        float4 raw = __ldcg(reinterpret_cast<const float4*>(A.cand + i));
        Cand c = *reinterpret_cast<Cand*>(&raw);
        if (c.q >= (unsigned)A.nq) continue;  // flagged by the refinement
        QState& s = A.qs[c.q];
        if ((unsigned long long)__double_as_longlong(d) == ld_relaxed64(&s.best_d)) {
            unsigned ia = (unsigned)__float_as_int(__ldg(s.A->tri + 3ull * c.ta + 2).y);
            unsigned ib = (unsigned)__float_as_int(__ldg(s.B->tri + 3ull * c.tb + 2).y);
            atomicMin(&s.best_key, ((unsigned long long)ia << 32) | ib);
        }
    }
}

// the witness record of each query: the candidate at the extreme with the
// smallest original (tri_a, tri_b); its points were stored by the refinement
__device__ void finalize_phase(const KArgs& A, RefinedSet R, unsigned long long first, unsigned long long gstride) {
    for (unsigned long long k = first; k < R.n; k += gstride) {
        const unsigned i = R.at((unsigned)k);
        if (i >= A.cap_cand) continue;
        double d = __ldcg(A.cand_d + i);
        float4 raw = __ldcg(reinterpret_cast<const float4*>(A.cand + i));
        Cand c = *reinterpret_cast<Cand*>(&raw);
        if (c.q >= (unsigned)A.nq) continue;  // flagged by the refinement
        QState& s = A.qs[c.q];
        if ((unsigned long long)__double_as_longlong(d) != ld_relaxed64(&s.best_d)) continue;
        unsigned ia = (unsigned)__float_as_int(__ldg(s.A->tri + 3ull * c.ta + 2).y);
        unsigned ib = (unsigned)__float_as_int(__ldg(s.B->tri + 3ull * c.tb + 2).y);
        if ((((unsigned long long)ia << 32) | ib) != ld_relaxed64(&s.best_key)) continue;
        const double* w = A.cand_pts + 6ull * i;
        gd_result& r = A.out[c.q];
        r.d = d;
        r.tri_a = ia;
        r.tri_b = ib;
        r.pa[0] = __ldcg(w); r.pa[1] = __ldcg(w + 1); r.pa[2] = __ldcg(w + 2);
        r.pb[0] = __ldcg(w + 3); r.pb[1] = __ldcg(w + 4); r.pb[2] = __ldcg(w + 5);
    }
}

// Single query, CTA 0 alone: the witness selection and the result record in
// one pass (select_phase then finalize_phase load every refined candidate
// twice, each through a chain of dependent loads): every thread keeps its
// least original (tri_a, tri_b) at the extreme, the CTA takes the least, and
// the thread that holds it writes the record.  The triangle arrays come from
// the CTA's copy of the query's constants.
__device__ void select_finalize_single(const KArgs& A, RefinedSet R) {
    __shared__ unsigned long long s_key;
    if (threadIdx.x == 0) s_key = 0xffffffffffffffffull;
    __syncthreads();
    QState& s = A.qs[0];
    const unsigned long long best = ld_relaxed64(&s.best_d);
    const float4* triA = cta().v.triA;
    const float4* triB = cta().v.triB;
    unsigned long long mykey = 0xffffffffffffffffull;
    unsigned myi = 0;
    for (unsigned k = threadIdx.x; k < R.n; k += blockDim.x) {
        const unsigned i = R.at(k);
        if (i >= A.cap_cand) continue;
        if ((unsigned long long)__double_as_longlong(__ldcg(A.cand_d + i)) != best) continue;
        float4 raw = __ldcg(reinterpret_cast<const float4*>(A.cand + i));
        const Cand c = *reinterpret_cast<Cand*>(&raw);
        if (c.q != 0u) continue;  // flagged by the refinement
        const unsigned ia = (unsigned)__float_as_int(__ldg(triA + 3ull * c.ta + 2).y);
        const unsigned ib = (unsigned)__float_as_int(__ldg(triB + 3ull * c.tb + 2).y);
        const unsigned long long key = ((unsigned long long)ia << 32) | ib;
        if (key < mykey) { mykey = key; myi = i; }
    }
    if (mykey != 0xffffffffffffffffull) atomicMin(&s_key, mykey);
    __syncthreads();
    if (mykey != 0xffffffffffffffffull && mykey == s_key) {
        // ties hold the same pair: equal records
        const double* w = A.cand_pts + 6ull * myi;
        gd_result& r = A.out[0];
        r.d = __longlong_as_double((long long)best);
        r.tri_a = (long long)(mykey >> 32);
        r.tri_b = (long long)(mykey & 0xffffffffull);
        r.pa[0] = __ldcg(w); r.pa[1] = __ldcg(w + 1); r.pa[2] = __ldcg(w + 2);
        r.pb[0] = __ldcg(w + 3); r.pb[1] = __ldcg(w + 4); r.pb[2] = __ldcg(w + 5);
        s.best_key = mykey;
    }
    __syncthreads();
}

__device__ void status_phase(const KArgs& A, unsigned long long first, unsigned long long gstride) {
    for (unsigned long long q = first; q < (unsigned)A.nq; q += gstride) {
        QState& s = A.qs[q];
        unsigned st = ld_relaxed(&s.status);
        if (ld_relaxed64(&s.best_key) == 0xffffffffffffffffull) st |= kStatNoResult;
        gd_result& r = A.out[q];
        unsigned code = GD_OK;
        // a proven D_min = 0 stands even if some entries were lost to full
        // queues or the query was evicted from its batch
        if (st & kStatEvict) st |= kStatOverflow;
        if ((st & kStatZero) && !(st & kStatNoResult)) st &= ~kStatOverflow;
        if (st & kStatOverflow) code = GD_ERR_OVERFLOW;
        else if (st & kStatTimeout) code = GD_ERR_TIMEOUT;
        else if (st & kStatNoResult) code = GD_ERR_CUDA;
        r.status = code;
        r.flags = (code == GD_OK && __ldcg(&r.d) == 0.0) ? 1u : 0u;
        if (code == GD_OK && (st & kStatZero)) r.flags |= 2u;
        if (code != GD_OK) {
            r.d = __longlong_as_double(0x7ff8000000000000ll);
            r.tri_a = r.tri_b = -1;
        }
        if (A.done_ns) A.done_ns[q] = globaltimer();
    }
}

// Run the refit jobs appended since the last call (one job per CTA at a time);
// returns false if the grid barrier after them failed; *ran tells whether
// there were any.
template <class AT>
__device__ bool refit_jobs(const AT& A, bool lead, unsigned& refits, bool* ran) {
    unsigned jobs = cta().ctr[kCtrJobs], done = cta().ctr[kCtrJobsDone];
    if (jobs > A.cap_slots) jobs = A.cap_slots;
    *ran = jobs > done;
    if (jobs <= done) return true;
    for (unsigned j = done + blockIdx.x; j < jobs; j += work_ctas(A)) {
        uint2 job = __ldcg(A.jobs + j);
        bool ok = job.x < (unsigned)A.nq && job.y >= 1u;
        if (ok) {
            const QState& qsj = A.qs[job.x];
            ok = qsj.dR >= 0 && depth_of(job.y) == qsj.dR && qsj.B->L >= qsj.dR;
        }
        if (ok) refit_subtree(A, job.x, job.y, j);
        else if (threadIdx.x == 0) flag_bad(A, kBadJob);
    }
    // no grid barrier: every CTA goes on to the level with its own job done;
    // the others' refits become visible root by root (refit_slot).  The
    // counter is read again only after the level's barrier.
    if (lead) {
        A.ctr[kCtrJobsDone] = jobs;
        refits = jobs;
    }
    return true;
}

// ------------------------------------------------------------- kernel

// FULL: the single query's B is refit whole into A's frame first (refit mode
// 3, the paper's per-frame refit); a separate instantiation, so that the
// default kernel's level loop is compiled without it.  ONE: a launch of one
// query (nq == 1) or a batch; with the query count known at compile time
// every single-query / batch branch of the inlined phases folds, so each
// instantiation carries only its own code and register pressure.
#ifndef GD_BATCH_CTAS
#define GD_BATCH_CTAS 4
#endif
template <int KIND, bool FULL, bool ONE>
__global__ void __launch_bounds__(kBlock, ONE ? 2 : GD_BATCH_CTAS) k_query(KArgs Aparam) {
    using AT = KArgsT<ONE>;
    const AT& A = static_cast<const AT&>(Aparam);
    unsigned long long pairs = 0, bytes = 0;
    unsigned tripairs = 0, refined = 0, refits = 0;
    unsigned leaf_flushed = 0;
    bool probed = false;  // set below once the first probes ran (or run in the background)
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;
    const unsigned long long gfirst = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned W = work_ctas(A);
    const unsigned long long gstride = (unsigned long long)W * blockDim.x;
    unsigned long long t_start = globaltimer(), t_mark = t_start, t_levels = 0;
    auto lap = [&](int slot) {
        if (lead) {
            unsigned long long now = globaltimer();
            if (slot >= 0) A.stats->phase_ns[slot] += (unsigned)(now - t_mark);
            t_mark = now;
        }
    };

    if (blockIdx.x >= W) {
        bg_probe_cta<KIND>(A);
        goto done;
    }

    // phase 0
    if (threadIdx.x == 0) cta().ready = 0;
    if (blockIdx.x == 0) {
        for (int i = threadIdx.x; i < kCtrReset; i += blockDim.x) A.ctr[i] = 0u;
        if (A.fuse_root) __syncthreads();  // cleared before the root is pushed below
    }
    if (AT::kOne) {
        if (gfirst < 32) setup_query_warp(A, KIND);
    } else {
        for (int q = (int)gfirst; q < A.nq; q += (int)gstride) setup_query(A, q, KIND);
    }
    if (A.fuse_root && gfirst == 0) {
        // one query whose root needs no refit claim: the thread that set it up
        // pushes its root pair now, and phase 1 with its barrier is skipped
        const QState& s = A.qs[0];
        const int LA = s.A->L, LB = s.B->L;
        const Item it = {1u, 1u, KIND == 0 ? 0.f : FLT_MAX, 0u};
        if (LA == 0 && LB == 0) {
            A.leafq[0] = it;
            A.ctr[kCtrLeaf] = 1u;
        } else {
            A.front0[0] = it;
            A.ctr[kCtrCnt] = 1u;
            A.ctr[kCtrRem] = (unsigned)(LA + LB);
        }
    }
    for (unsigned long long i = gfirst; i < A.n_slot_of; i += gstride) A.slot_of[i] = kNoSlot;
    if (lead) {
        StatsDev* S = A.stats;
        S->levels = 0;
        for (int i = 0; i < kAccWays; ++i) {
            S->acc_pairs[i] = 0;
            S->acc_bytes[i] = 0;
            S->acc_tri[i] = 0;
            S->acc_ref[i] = 0;
        }
        S->leaf_pairs = S->candidates = 0;
        S->probes = 0;
        S->refits = 0;
        S->t_start = t_start;
        S->u_probe = 0.f;
        for (int i = 0; i < 12; ++i) S->phase_ns[i] = 0;
        for (int i = 0; i < 32; ++i) { S->level_ns[i] = 0; S->u_level[i] = 0.f; }
    }
    if (W < gridDim.x && blockIdx.x == 0) {
        // publish the (single) query's setup to the background probe CTAs
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicExch(A.ctr + kCtrSetupDone, 1u);
        }
    }
    if (!sync(A)) goto done;

    if (FULL) {
        // full refit of B into A's frame (single query): subtrees of 2^h
        // leaves, then the levels above 8 at a time
        const QConst& V = cta().v;
        const int h = min(V.LB, kRefitH);
        const int dF = V.LB - h;
        for (unsigned j = blockIdx.x; j < (1u << dF); j += W) full_refit_leaves(A, V, (1u << dF) + j, h);
        if (!sync(A)) goto done;
        for (int d = dF; d > 0;) {
            const int lv = min(d, kRefitH);
            for (unsigned j = blockIdx.x; j < (1u << (d - lv)); j += W)
                full_refit_up(A, (1ull << d) + ((unsigned long long)j << lv), lv);
            if (!sync(A)) goto done;
            d -= lv;
        }
        lap(1);
    }

    // phase 1: root pairs
    if (A.fuse_root) goto levels;
    for (int q = (int)gfirst; q < A.nq; q += (int)gstride) {
        const QState& s = A.qs[q];
        int LA = s.A->L, LB = s.B->L;
        Item it = {1u, 1u, KIND == 0 ? 0.f : FLT_MAX, (unsigned)q};
        if (LA == 0 && LB == 0) {
            unsigned i = atomicAdd(A.ctr + kCtrLeaf, 1u);
            if (i < A.cap_leaf) A.leafq[i] = it; else mark_overflow(A, q);
        } else {
            unsigned i = atomicAdd(A.ctr + kCtrCnt, 1u);
            if (i < A.cap_front) A.front0[i] = it; else mark_overflow(A, q);
            atomicMax(A.ctr + kCtrRem, (unsigned)(LA + LB));
            if (s.dR == 0) {
                QView V;
                view(A, q, V);
                claim_root(A, V, q, 1u);
            }
        }
    }
    if (!sync(A)) goto done;
levels:
    lap(0);

    // phase 2: BVTT levels
    if (W < gridDim.x) probed = true;
    for (int level = 0;; ++level) {
        unsigned n = cta().ctr[kCtrCnt + level % 3];
        if (n > A.cap_front) n = A.cap_front;
        if (n == 0) break;
        if (level >= kMaxLevels) {
            if (lead) atomicOr(A.ctr + kCtrOverflow, 2u);
            break;
        }
        bool ran = false;
        if (!refit_jobs(A, lead, refits, &ran)) goto done;
        if (ran) lap(1);
        // probes start where B's boxes are first exact in A's frame (or at
        // level 1 without refit), so that their greedy choices follow tight
        // boxes; the min kind probes again on every level whose front has
        // outgrown 4x the work target, where the descents to leaves may also
        // prove D_min = 0 and so stop the growth
        const bool reprobe = KIND == 0 && probed && (long long)n >= 4 * A.work_target;
        if (reprobe || (!probed && (A.refit ? ran : level == 1))) {
            probed = true;
            // greedy probes from entries spread evenly over the front: every
            // warp takes one (at least one per query when the grid allows)
            const unsigned nwarps = W * (blockDim.x >> 5);
            const unsigned wid = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
            // (a min query's repeated probes on large fronts use at least
            // kReprobes walks, enough to meet an intersection if there is one)
            const unsigned want = max((unsigned)A.nq, reprobe ? max((unsigned)A.probes, kReprobes) : (unsigned)A.probes);
            const unsigned P = min(n, min(nwarps, want));
            const Item* in = (level & 1) ? A.front1 : A.front0;
            QView V;
            for (unsigned p = wid; p < P; p += nwarps) {
                unsigned idx = (unsigned)(((unsigned long long)p * n) / P);
                float4 raw = __ldcg(reinterpret_cast<const float4*>(in + idx));
                Item it = *reinterpret_cast<Item*>(&raw);
                if (!item_ok(A, it)) {
                    if ((threadIdx.x & 31) == 0) flag_bad(A, kBadProbe);
                    continue;
                }
                view(A, it.q, V);
                if (depth_of(it.a) > V.LA || depth_of(it.b) > V.LB) {
                    if ((threadIdx.x & 31) == 0) flag_bad(A, kBadProbe);
                    continue;
                }
                probe<KIND>(A, it, V);
            }
            if (lead) A.stats->probes += P;
            if (!sync(A)) goto done;
            if (lead && !reprobe) A.stats->u_probe = AT::kOne ? __uint_as_float(cta().U) : 0.f;
            lap(2);
        }
        unsigned rmax = cta().ctr[kCtrRem + level % 3];
        int k = adaptive_k(n, A.work_target, A.k_max);
        int s = min(2 * k, (int)rmax);
        if (s < 1) s = 1;
        if (lead) {
            A.ctr[kCtrCnt + (level + 2) % 3] = 0u;
            A.ctr[kCtrRem + (level + 2) % 3] = 0u;
            A.ctr[(level & 1) ? kCtrPool1 : kCtrPool0] = 0u;  // the pool of level + 1's pushes
            if (level < 32) {
                A.stats->front[level] = n;
                A.stats->slots[level] = (unsigned)s;
                // query 0's bound as this CTA knows it (no global round trip
                // on the lead's way into the level)
                A.stats->u_level[level] = AT::kOne ? __uint_as_float(cta().U) : 0.f;
            }
            A.stats->levels = level + 1;
        }
        if (A.q_budget)  // the counters of this level's pushes are those of level + 2
            for (int q = (int)gfirst; q < A.nq; q += (int)gstride) A.qs[q].pushed[level & 1] = 0u;
        // a batch front of more than twice the grid's threads at one tree
        // level each: a thread per entry
        if (!AT::kOne && s == 2 && (unsigned long long)n > 2ull * gstride)
            expand_level_entries<KIND>(A, level, n, pairs, bytes);
        else
            expand_level<KIND, FULL>(A, level, n, s, pairs, bytes);
        if (!sync(A)) goto done;
        if (lead) {
            unsigned long long now = globaltimer();
            if (level < 32) A.stats->level_ns[level] = (unsigned)(now - t_mark);
            t_levels += now - t_mark;
            t_mark = now;
        }
        // a leaf queue at half its capacity is emptied through the leaf phase
        // now (every CTA reads the same count: no push happens between the
        // barrier above and the next level), so that the queue never has to
        // hold the leaf pairs of all levels at once
        unsigned nl = cta().ctr[kCtrLeaf];
        if (nl >= A.cap_leaf / 2) {
            if (nl > A.cap_leaf) nl = A.cap_leaf;
            leaf_phase<KIND>(A, nl, tripairs, bytes);
            if (!sync(A)) goto done;
            if (lead) {
                A.ctr[kCtrLeaf] = 0u;
                leaf_flushed += nl;
            }
            if (!sync(A)) goto done;
            lap(4);
        }
    }
    if (lead) A.stats->phase_ns[3] = (unsigned)t_levels;

    // phase 3
    {
        unsigned nleaf = cta().ctr[kCtrLeaf];
        if (nleaf > A.cap_leaf) nleaf = A.cap_leaf;
        if (lead) A.stats->leaf_pairs = leaf_flushed + nleaf;
        leaf_phase<KIND>(A, nleaf, tripairs, bytes);
    }
    if (!sync(A)) goto done;
    lap(4);
    {
        unsigned nc = cta().ctr[kCtrCand];
        if (nc > A.cap_cand) nc = A.cap_cand;
        if (lead) A.stats->candidates = nc;
        if (nc <= W) {
            // few candidates: one per CTA (its warp 0), spread over the SMs'
            // float64 pipes; CTA 0 waits for the others (bounded) and then
            // selects the witness alone, so no grid-wide barrier is needed
            refine_phase_cta<KIND>(A, nc, refined, bytes);
            __syncthreads();
            lap(5);
            if (threadIdx.x == 0 && blockIdx.x < nc) {
                __threadfence();
                atomicAdd(A.ctr + kCtrTailDone, 1u);
            }
            if (blockIdx.x == 0) {
                __shared__ int s_go;
                if (threadIdx.x == 0) {
                    int go = 1;
                    unsigned long long t0 = globaltimer();
                    while (ld_acquire(A.ctr + kCtrTailDone) < nc) {
                        if (ld_relaxed(A.ctr + kCtrAbort)) { go = 0; break; }
                        if ((long long)(globaltimer() - t0) > A.timeout_ns) {
                            raise_abort(A);
                            go = 0;
                            break;
                        }
                        __nanosleep(32);
                    }
                    __threadfence();
                    s_go = go;
                }
                __syncthreads();
                if (s_go) {
                    lap(6);
                    const RefinedSet R{nullptr, nc};
                    if (AT::kOne) {
                        select_finalize_single(A, R);
                        lap(7);
                    } else {
                        select_phase(A, R, threadIdx.x, blockDim.x);
                        __syncthreads();
                        lap(7);
                        finalize_phase(A, R, threadIdx.x, blockDim.x);
                        __syncthreads();
                    }
                    status_phase(A, threadIdx.x, blockDim.x);
                    __syncthreads();
                    lap(8);
                }
            }
            goto done;
        }
        refine_phase_cta<KIND>(A, nc, refined, bytes);
        if (!sync(A)) goto done;
        lap(5);
        const RefinedSet R = refined_set(A, cta().ctr[kCtrRefined], nc);
        if (AT::kOne) {
            // one query: CTA 0 selects and writes the witness alone (the refined
            // candidates are few), no further grid barrier
            if (blockIdx.x == 0) {
                select_finalize_single(A, R);
                lap(7);
                status_phase(A, threadIdx.x, blockDim.x);
                lap(8);
            }
            goto done;
        }
        select_phase(A, R, gfirst, gstride);
        if (!sync(A)) goto done;
        lap(7);
        finalize_phase(A, R, gfirst, gstride);
        if (!sync(A)) goto done;
        status_phase(A, gfirst, gstride);
        lap(8);
    }

done:
    if (lead) {
        A.stats->phase_ns[9] = (unsigned)(globaltimer() - t_start);
        A.stats->refits = refits;
    }
    // per-CTA statistics
    {
        __shared__ unsigned long long s_pairs, s_bytes;
        __shared__ unsigned s_tri, s_ref;
        if (threadIdx.x == 0) { s_pairs = 0; s_bytes = 0; s_tri = 0; s_ref = 0; }
        __syncthreads();
        // warp sums first, then one shared atomic per warp
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            pairs += __shfl_xor_sync(kFull, pairs, o);
            bytes += __shfl_xor_sync(kFull, bytes, o);
        }
        tripairs = __reduce_add_sync(kFull, tripairs);
        refined = __reduce_add_sync(kFull, refined);
        if ((threadIdx.x & 31) == 0) {
            atomicAdd(&s_pairs, pairs);
            atomicAdd(&s_bytes, bytes);
            atomicAdd(&s_tri, tripairs);
            atomicAdd(&s_ref, refined);
        }
        __shared__ unsigned s_last_ab;
        __shared__ int s_last;
        __syncthreads();
        if (threadIdx.x == 0) {
            const int w = blockIdx.x % kAccWays;
            if (s_pairs) atomicAdd(&A.stats->acc_pairs[w], s_pairs);
            if (s_bytes) atomicAdd(&A.stats->acc_bytes[w], s_bytes);
            if (s_tri) atomicAdd(&A.stats->acc_tri[w], s_tri);
            if (s_ref) atomicAdd(&A.stats->acc_ref[w], s_ref);
            // the last CTA out leaves the barrier and abort words clean for the
            // next launch and publishes this launch's abort flag
            __threadfence();
            unsigned e = atomicAdd(A.ctr + kCtrExit, 1u);
            s_last = e == gridDim.x - 1;
            if (s_last) {
                unsigned ab = atomicExch(A.ctr + kCtrAbort, 0u);
                atomicExch(A.ctr + kCtrLastAbort, ab);
                atomicExch(A.ctr + kCtrBarCount, 0u);
                atomicExch(A.ctr + kCtrSetupDone, 0u);
                atomicExch(A.ctr + kCtrExit, 0u);
                __threadfence();
                s_last_ab = ab;
            }
        }
        __syncthreads();
        if (s_last && A.host_done) {
            // every other CTA has left (their writes, the result records among
            // them, were fenced before their exit count): the records go to
            // the host's pinned memory, then the stamp
            HostDone* h = A.host_done;
            static_assert(sizeof(gd_result) % 8 == 0, "result record copied in 8-byte words");
            constexpr int kW = (int)(sizeof(gd_result) / 8);
            const unsigned long long* src = reinterpret_cast<const unsigned long long*>(A.out);
            if (A.host_out) {
                unsigned long long* dst = reinterpret_cast<unsigned long long*>(A.host_out);
                for (long long k = threadIdx.x; k < (long long)A.nq * kW; k += blockDim.x) dst[k] = __ldcg(src + k);
            } else if (threadIdx.x < kW) {
                reinterpret_cast<unsigned long long*>(&h->out)[threadIdx.x] = __ldcg(src + threadIdx.x);
            }
            __threadfence_system();
            __syncthreads();
            if (threadIdx.x == 0) {
                h->last_abort = s_last_ab;
                h->bad_index = ld_relaxed(A.ctr + kCtrBadIndex);
                __threadfence_system();
                *reinterpret_cast<volatile unsigned long long*>(&h->seq) = A.seq;
            }
        }
    }
}

// ------------------------------------------------------------- host side

// Both kinds get the same shared-memory carveout, so that CTAs of a min and a
// max launch can share an SM (an SM holds CTAs of one carveout at a time).
// The instantiations of one kind: batch, single query, single query with the
// full refit.
template <int KIND>
static const void* kind_kernel(int i) {
    return i == 0 ? (const void*)k_query<KIND, false, false>
                  : (i == 1 ? (const void*)k_query<KIND, false, true> : (const void*)k_query<KIND, true, true>);
}

template <int KIND>
static int occupancy_blocks(bool batch) {
    static bool configured = false;
    if (!configured) {
        // a single query's CTAs need 2 x 22 KB of shared memory per SM; a
        // batch's may take more CTAs per SM
        for (int i = 0; i < 3; ++i)
            cudaFuncSetAttribute(kind_kernel<KIND>(i), cudaFuncAttributePreferredSharedMemoryCarveout, i == 0 ? 50 : 25);
        configured = true;
    }
    // a batch launch runs instantiation 0; a single query 1 or 2, which use
    // the same registers and shared memory per CTA (the smaller occupancy of
    // the two so that either fits)
    int nb = 1 << 30;
    for (int i = batch ? 0 : 1; i < (batch ? 1 : 3); ++i) {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kind_kernel<KIND>(i), kBlock, 0);
        nb = n < nb ? n : nb;
    }
    return nb;
}

int query_max_blocks_per_sm(int kind, bool batch) {
    return kind == 0 ? occupancy_blocks<0>(batch) : occupancy_blocks<1>(batch);
}

static const void* query_kernel(int kind, const KArgs& args) {
    const int i = args.nq != 1 ? 0 : (args.ftree ? 2 : 1);
    return kind == 0 ? kind_kernel<0>(i) : kind_kernel<1>(i);
}

cudaError_t launch_query(int kind, const KArgs& args, int grid, cudaStream_t stream) {
    void* params[] = {const_cast<KArgs*>(&args)};
    return cudaLaunchCooperativeKernel(query_kernel(kind, args), dim3(grid), dim3(kBlock), params, 0, stream);
}

// A graph with the query kernel as its one cooperative kernel node (the
// arguments are copied into the node).
cudaError_t build_query_graph(int kind, const KArgs& args, int grid, cudaGraphExec_t* exec) {
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaGraphCreate(&g, 0);
    if (e != cudaSuccess) return e;
    void* params[] = {const_cast<KArgs*>(&args)};
    cudaKernelNodeParams p{};
    p.func = const_cast<void*>(query_kernel(kind, args));
    p.gridDim = dim3(grid);
    p.blockDim = dim3(kBlock);
    p.sharedMemBytes = 0;
    p.kernelParams = params;
    cudaGraphNode_t node = nullptr;
    e = cudaGraphAddKernelNode(&node, g, nullptr, 0, &p);
    if (e == cudaSuccess) {
        cudaLaunchAttributeValue v{};
        v.cooperative = 1;
        e = cudaGraphKernelNodeSetAttribute(node, cudaLaunchAttributeCooperative, &v);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    return e;
}

}  // namespace gd
