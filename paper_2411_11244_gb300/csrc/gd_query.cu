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
//      bits (Section 7.4);
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

constexpr float kU = 5.9604645e-08f;   // 2^-24, unit roundoff of float32
constexpr float kRelW = 9.5367432e-07f; // 2^-20: world vs working-frame slack
constexpr unsigned kFltMaxBits = 0x7f7fffffu;

template <int KIND>
struct Kind;

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

__device__ __forceinline__ Box load_box(const float* box, unsigned i) {
    const float2* p = reinterpret_cast<const float2*>(box + 6ull * i);
    float2 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
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

// Lower (KIND 0) or raise (KIND 1) the running bound of query q by bits v.
// All lanes of the warp call this; lanes with have == false pass nothing.
template <int KIND>
__device__ __forceinline__ void warp_bound_update(bool have, unsigned q, unsigned v, QState* qs) {
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

__device__ __forceinline__ void mark_overflow(const KArgs& A, unsigned q) {
    atomicOr(&A.qs[q].status, kStatOverflow);
    atomicOr(A.ctr + kCtrOverflow, 1u);
}

// cached per-thread view of one query's constants
struct QView {
    unsigned q = 0xffffffffu;
    Rigid32 X;
    float E_box, E_tri;
    const float* boxA;
    const float* boxB;
    const float4* triA;
    const float4* triB;
    long long TA, TB;
    int LA, LB;
};

__device__ __forceinline__ void view(const KArgs& A, unsigned q, QView& V) {
    if (V.q == q) return;
    const QState& s = A.qs[q];
#pragma unroll
    for (int i = 0; i < 9; ++i) V.X.R[i] = __ldcg(&s.R[i]);
#pragma unroll
    for (int i = 0; i < 3; ++i) V.X.t[i] = __ldcg(&s.t[i]);
    V.E_box = __ldcg(&s.E_box);
    V.E_tri = __ldcg(&s.E_tri);
    const MeshDev* ma = s.A;
    const MeshDev* mb = s.B;
    V.boxA = ma->box; V.boxB = mb->box;
    V.triA = ma->tri; V.triB = mb->tri;
    V.TA = ma->T; V.TB = mb->T;
    V.LA = ma->L; V.LB = mb->L;
    V.q = q;
}

// ------------------------------------------------------------- phase 0

__device__ void setup_query(const KArgs& A, int q, int kind) {
    QState& s = A.qs[q];
    const MeshDev* ma;
    const MeshDev* mb;
    const double* xa;
    const double* xb;
    if (A.qin) {
        ma = A.qin[q].A; mb = A.qin[q].B;
        xa = A.qin[q].xa; xb = A.qin[q].xb;
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
            s.R[3 * i + j] = (float)r;
        }
        double tt = Ai[3 * i] * dt[0] + Ai[3 * i + 1] * dt[1] + Ai[3 * i + 2] * dt[2];
        s.t[i] = (float)tt;
        tinf = fmaxf(tinf, fabsf((float)tt));
    }
    // widening: every mapped coordinate is within e_c of its exact value,
    // e_c = gamma_10 (sqrt(3) P_B + |t|_inf); E_box = sqrt(3) e_c; the
    // triangle narrow phase adds 256 u X for its own arithmetic on
    // coordinates of magnitude <= X.
    const double u = 5.9604644775390625e-08;
    const double g10 = 10.0 * u / (1.0 - 10.0 * u);
    double PB = (double)mb->P * 1.000001, PA = (double)ma->P;
    double ec = g10 * (1.7320508075688772 * PB + (double)tinf);
    double Eb = 1.7320508075688772 * ec * 1.000001;
    double Xm = fmax(PA, 1.7320508075688772 * PB + (double)tinf) * 1.000001 + Eb;
    double Et = Eb + 256.0 * u * Xm;
    s.E_box = __double2float_ru(Eb);
    s.E_tri = __double2float_ru(Et);
    s.A = ma;
    s.B = mb;
    for (int i = 0; i < 12; ++i) { s.xa[i] = Xa[i]; s.xb[i] = Xb[i]; }
    s.U = kind == 0 ? kFltMaxBits : 0u;
    s.status = 0u;
    s.best_d = kind == 0 ? 0x7ff0000000000000ull : 0ull;  // +inf / +0
    s.best_key = 0xffffffffffffffffull;
}

// ------------------------------------------------------------- phase 2

__device__ __forceinline__ int adaptive_k(unsigned n, long long C, int kmax) {
    int k = 1;
    while (k < kmax && (long long)n << (2 * (k + 1)) < C) ++k;
    return k;
}

template <int KIND>
__device__ void expand_level(const KArgs& A, int level, unsigned n, int s, unsigned long long& pairs,
                             unsigned long long& bytes) {
    const Item* in = (level & 1) ? A.front1 : A.front0;
    Item* out = (level & 1) ? A.front0 : A.front1;
    unsigned* out_cnt = A.ctr + kCtrCnt + (level + 1) % 3;
    unsigned* out_rem = A.ctr + kCtrRem + (level + 1) % 3;
    unsigned* leaf_cnt = A.ctr + kCtrLeaf;
    const unsigned long long total = (unsigned long long)n << s;
    const unsigned long long gstride = (unsigned long long)gridDim.x * blockDim.x;
    const unsigned long long mask = (1ull << s) - 1;
    const int lane = threadIdx.x & 31;
    QView V;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
         base < total; base += gstride) {
        unsigned long long vt = base + lane;
        bool valid = vt < total;
        Item it = {1u, 1u, 0.f, 0u};
        if (valid) {
            float4 raw = __ldcg(reinterpret_cast<const float4*>(in + (vt >> s)));
            it = *reinterpret_cast<Item*>(&raw);
        }
        unsigned q = it.q;
        view(A, q, V);
        const int dA = 31 - __clz(it.a), dB = 31 - __clz(it.b);
        const int remA = V.LA - dA, remB = V.LB - dB;
        int kA = min((s + 1) >> 1, remA);
        int kB = min(s - kA, remB);
        kA = min(s - kB, remA);
        unsigned local = (unsigned)(vt & mask);
        valid = valid && local < (1u << (kA + kB));
        float Ucur = __uint_as_float(ld_relaxed(&A.qs[q].U));
        if (KIND == 0) valid = valid && it.bound <= min_keep_threshold(Ucur, V.E_box);
        else valid = valid && it.bound >= max_keep_threshold(Ucur, V.E_box);
        if (valid && local == 0) bytes += 16ull + 24ull * ((1ull << kA) + (1ull << kB));
        unsigned ia = (it.a << kA) | (local >> kB);
        unsigned ib = (it.b << kB) | (local & ((1u << kB) - 1u));
        bool leafpair = (kA == remA) && (kB == remB);
        bool survive = false;
        float bound = 0.f;
        unsigned newU = KIND == 0 ? 0xffffffffu : 0u;
        if (valid) {
            ++pairs;
            Box ba = load_box(V.boxA, ia);
            Box bb = load_box(V.boxB, ib);
            float elo[3], ehi[3];
            enclose(V.X, bb, elo, ehi);
            if (KIND == 0) {
                bound = lower_min_sq(ba, elo, ehi);
                survive = bound <= min_keep_threshold(Ucur, V.E_box);
                if (survive) newU = __float_as_uint(upper_from_sq(upper_min_sq_enhanced(V.X, ba, bb), V.E_box));
            } else {
                bound = upper_max_sq(ba, elo, ehi);
                survive = bound >= max_keep_threshold(Ucur, V.E_box);
                if (survive) newU = __float_as_uint(lower_from_sq(lower_max_sq_enhanced(V.X, ba, bb), V.E_box));
            }
        }
        warp_bound_update<KIND>(survive, q, newU, A.qs);
        Item o = {ia, ib, bound, q};
        bool ok1 = warp_push(survive && !leafpair, o, out, out_cnt, A.cap_front);
        bool ok2 = warp_push(survive && leafpair, o, A.leafq, leaf_cnt, A.cap_leaf);
        if (!ok1 || !ok2) mark_overflow(A, q);
        if (survive) bytes += 16ull;
        // remaining depth of the entries pushed to the next front
        unsigned rem = (survive && !leafpair) ? (unsigned)(remA - kA + remB - kB) : 0u;
        rem = __reduce_max_sync(kFull, rem);
        if (lane == 0 && rem > 0 && rem > ld_relaxed(out_rem)) atomicMax(out_rem, rem);
    }
}

// ------------------------------------------------------------- phase 3

template <int KIND>
__device__ void leaf_phase(const KArgs& A, unsigned nleaf, unsigned& tripairs, unsigned long long& bytes) {
    const unsigned long long total = (unsigned long long)nleaf * 4ull;
    const unsigned long long gstride = (unsigned long long)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    unsigned* cand_cnt = A.ctr + kCtrCand;
    QView V;
    for (unsigned long long base = (unsigned long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
         base < total; base += gstride) {
        unsigned long long vt = base + lane;
        bool valid = vt < total;
        Item it = {1u, 1u, 0.f, 0u};
        if (valid) {
            float4 raw = __ldcg(reinterpret_cast<const float4*>(A.leafq + (vt >> 2)));
            it = *reinterpret_cast<Item*>(&raw);
        }
        unsigned q = it.q;
        view(A, q, V);
        unsigned sub = (unsigned)(vt & 3);
        unsigned la = it.a - (1u << V.LA), lb = it.b - (1u << V.LB);
        unsigned a0 = leaf_first(V.TA, V.LA, la), a1 = leaf_first(V.TA, V.LA, la + 1);
        unsigned b0 = leaf_first(V.TB, V.LB, lb), b1 = leaf_first(V.TB, V.LB, lb + 1);
        unsigned ta = a0 + (sub >> 1), tb = b0 + (sub & 1);
        valid = valid && ta < a1 && tb < b1;
        float Ucur = __uint_as_float(ld_relaxed(&A.qs[q].U));
        if (KIND == 0) valid = valid && it.bound <= min_keep_threshold(Ucur, V.E_box);
        else valid = valid && it.bound >= max_keep_threshold(Ucur, V.E_box);
        if (valid && sub == 0) bytes += 16ull + 36ull * ((a1 - a0) + (b1 - b0));
        bool emit = false;
        float cb = 0.f;
        unsigned newU = KIND == 0 ? 0xffffffffu : 0u;
        bool have = false;
        if (valid) {
            ++tripairs;
            Tri32 TA = load_tri(V.triA, ta), TB = load_tri(V.triB, tb);
            V3<float> Bw[3];
#pragma unroll
            for (int k = 0; k < 3; ++k) Bw[k] = map32(V.X, TB.v[k].x, TB.v[k].y, TB.v[k].z);
            if (KIND == 0) {
                V3<float> P, Q;
                float d2;
                bool hit;
                tri_tri_min(TA.v, Bw, &P, &Q, &d2, &hit);
                float up = upper_from_sq(d2, V.E_tri);
                // lower bound: separation of the two triangles along P - Q
                float lo = 0.f;
                V3<float> nrm = P - Q;
                float nn = dot(nrm, nrm);
                if (nn > 0.f) {
                    float amin = FLT_MAX, bmax = -FLT_MAX;
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        amin = fminf(amin, dot(nrm, TA.v[k]));
                        bmax = fmaxf(bmax, dot(nrm, Bw[k]));
                    }
                    float sep = amin - bmax;
                    if (sep > 0.f) lo = lower_from_dist(sep / sqrtf(nn), V.E_tri);
                }
                have = true;
                newU = __float_as_uint(up);
                cb = lo;
                emit = lo <= fminf(Ucur, up);
            } else {
                V3<float> P, Q;
                float d2;
                tri_tri_max(TA.v, Bw, &P, &Q, &d2);
                float lo = lower_from_sq(d2, V.E_tri);
                float up = upper_from_sq(d2, V.E_tri);
                have = true;
                newU = __float_as_uint(lo);
                cb = up;
                emit = up >= fmaxf(Ucur, lo);
            }
        }
        warp_bound_update<KIND>(have, q, newU, A.qs);
        Cand c = {ta, tb, cb, q};
        if (!warp_push(emit, c, A.cand, cand_cnt, A.cap_cand)) mark_overflow(A, q);
        if (emit) bytes += 16ull;
    }
}

// ------------------------------------------------------------- phases 4-6

__device__ __forceinline__ void world_tri(const float4* tri, unsigned j, const double* X, V3<double>* W, int* id) {
    Tri32 t = load_tri(tri, j);
#pragma unroll
    for (int k = 0; k < 3; ++k) W[k] = map64(X, (double)t.v[k].x, (double)t.v[k].y, (double)t.v[k].z);
    *id = t.id;
}

template <int KIND>
__device__ __forceinline__ double refine_pair(const QState& s, unsigned ta, unsigned tb, V3<double>* P,
                                              V3<double>* Q, int* ida, int* idb) {
    V3<double> Aw[3], Bw[3];
    world_tri(s.A->tri, ta, s.xa, Aw, ida);
    world_tri(s.B->tri, tb, s.xb, Bw, idb);
    double d2;
    if (KIND == 0) {
        bool hit;
        tri_tri_min(Aw, Bw, P, Q, &d2, &hit);
        if (hit) return 0.0;
    } else {
        tri_tri_max(Aw, Bw, P, Q, &d2);
    }
    return sqrt(d2);
}

template <int KIND>
__device__ void refine_phase(const KArgs& A, unsigned ncand, unsigned& refined, unsigned long long& bytes) {
    const unsigned long long gstride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < ncand; i += gstride) {
        float4 raw = __ldcg(reinterpret_cast<const float4*>(A.cand + i));
        Cand c = *reinterpret_cast<Cand*>(&raw);
        QState& s = A.qs[c.q];
        float U = __uint_as_float(ld_relaxed(&s.U));
        bool keep = KIND == 0 ? (c.bound <= U) : (c.bound >= U);
        double d = __longlong_as_double(-1ll);  // NaN: never selected
        if (keep) {
            V3<double> P, Q;
            int ia, ib;
            d = refine_pair<KIND>(s, c.ta, c.tb, &P, &Q, &ia, &ib);
            unsigned long long bits = (unsigned long long)__double_as_longlong(d);
            if (KIND == 0) atomicMin(&s.best_d, bits);
            else atomicMax(&s.best_d, bits);
            ++refined;
            bytes += 16ull + 72ull;
        }
        A.cand_d[i] = d;
    }
}

__device__ void select_phase(const KArgs& A, unsigned ncand) {
    const unsigned long long gstride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < ncand; i += gstride) {
        double d = __ldcg(A.cand_d + i);
        float4 raw = __ldcg(reinterpret_cast<const float4*>(A.cand + i));
        Cand c = *reinterpret_cast<Cand*>(&raw);
        QState& s = A.qs[c.q];
        if ((unsigned long long)__double_as_longlong(d) == ld_relaxed64(&s.best_d)) {
            unsigned ia = (unsigned)__float_as_int(__ldg(s.A->tri + 3ull * c.ta + 2).y);
            unsigned ib = (unsigned)__float_as_int(__ldg(s.B->tri + 3ull * c.tb + 2).y);
            atomicMin(&s.best_key, ((unsigned long long)ia << 32) | ib);
        }
    }
}

template <int KIND>
__device__ void finalize_phase(const KArgs& A, unsigned ncand) {
    const unsigned long long gstride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < ncand; i += gstride) {
        double d = __ldcg(A.cand_d + i);
        float4 raw = __ldcg(reinterpret_cast<const float4*>(A.cand + i));
        Cand c = *reinterpret_cast<Cand*>(&raw);
        QState& s = A.qs[c.q];
        if ((unsigned long long)__double_as_longlong(d) != ld_relaxed64(&s.best_d)) continue;
        unsigned ia = (unsigned)__float_as_int(__ldg(s.A->tri + 3ull * c.ta + 2).y);
        unsigned ib = (unsigned)__float_as_int(__ldg(s.B->tri + 3ull * c.tb + 2).y);
        if ((((unsigned long long)ia << 32) | ib) != ld_relaxed64(&s.best_key)) continue;
        V3<double> P, Q;
        int da, db;
        double dd = refine_pair<KIND>(s, c.ta, c.tb, &P, &Q, &da, &db);
        gd_result& r = A.out[c.q];
        r.d = dd;
        r.tri_a = ia;
        r.tri_b = ib;
        r.pa[0] = P.x; r.pa[1] = P.y; r.pa[2] = P.z;
        r.pb[0] = Q.x; r.pb[1] = Q.y; r.pb[2] = Q.z;
    }
}

__device__ void status_phase(const KArgs& A) {
    const unsigned long long gstride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long q = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; q < (unsigned)A.nq;
         q += gstride) {
        QState& s = A.qs[q];
        unsigned st = s.status;
        if (s.best_key == 0xffffffffffffffffull) st |= kStatNoResult;
        gd_result& r = A.out[q];
        unsigned code = GD_OK;
        if (st & kStatOverflow) code = GD_ERR_OVERFLOW;
        else if (st & kStatTimeout) code = GD_ERR_TIMEOUT;
        else if (st & kStatNoResult) code = GD_ERR_CUDA;
        r.status = code;
        r.flags = (code == GD_OK && __ldcg(&r.d) == 0.0) ? 1u : 0u;
        if (code != GD_OK) {
            r.d = __longlong_as_double(0x7ff8000000000000ll);
            r.tri_a = r.tri_b = -1;
        }
    }
}

// ------------------------------------------------------------- kernel

template <int KIND>
__global__ void __launch_bounds__(kBlock, 2) k_query(KArgs A) {
    unsigned long long pairs = 0, bytes = 0;
    unsigned tripairs = 0, refined = 0;
    const bool lead = blockIdx.x == 0 && threadIdx.x == 0;

    // phase 0
    if (blockIdx.x == 0)
        for (int i = threadIdx.x; i < kCtrReset; i += blockDim.x) A.ctr[i] = 0u;
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < A.nq; q += gridDim.x * blockDim.x)
        setup_query(A, q, KIND);
    if (lead) {
        StatsDev* S = A.stats;
        S->levels = 0;
        S->pairs_tested = 0;
        S->leaf_pairs = S->tri_pairs = S->candidates = S->refined = 0;
        S->alg_bytes = 0;
    }
    if (!grid_sync(A)) goto done;

    // phase 1: root pairs
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < A.nq; q += gridDim.x * blockDim.x) {
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
        }
    }
    if (!grid_sync(A)) goto done;

    // phase 2: BVTT levels
    for (int level = 0;; ++level) {
        unsigned n = ld_relaxed(A.ctr + kCtrCnt + level % 3);
        if (n > A.cap_front) n = A.cap_front;
        if (n == 0) break;
        if (level >= kMaxLevels) {
            if (lead) atomicOr(A.ctr + kCtrOverflow, 2u);
            break;
        }
        unsigned rmax = ld_relaxed(A.ctr + kCtrRem + level % 3);
        int k = adaptive_k(n, A.work_target, A.k_max);
        int s = min(2 * k, (int)rmax);
        if (s < 1) s = 1;
        if (lead) {
            A.ctr[kCtrCnt + (level + 2) % 3] = 0u;
            A.ctr[kCtrRem + (level + 2) % 3] = 0u;
            if (level < 32) { A.stats->front[level] = n; A.stats->slots[level] = (unsigned)s; }
            A.stats->levels = level + 1;
        }
        expand_level<KIND>(A, level, n, s, pairs, bytes);
        if (!grid_sync(A)) goto done;
    }

    // phase 3
    {
        unsigned nleaf = ld_relaxed(A.ctr + kCtrLeaf);
        if (nleaf > A.cap_leaf) nleaf = A.cap_leaf;
        if (lead) A.stats->leaf_pairs = nleaf;
        leaf_phase<KIND>(A, nleaf, tripairs, bytes);
    }
    if (!grid_sync(A)) goto done;
    // phase 4
    {
        unsigned nc = ld_relaxed(A.ctr + kCtrCand);
        if (nc > A.cap_cand) nc = A.cap_cand;
        if (lead) A.stats->candidates = nc;
        refine_phase<KIND>(A, nc, refined, bytes);
    }
    if (!grid_sync(A)) goto done;
    {
        unsigned nc = ld_relaxed(A.ctr + kCtrCand);
        if (nc > A.cap_cand) nc = A.cap_cand;
        select_phase(A, nc);
    }
    if (!grid_sync(A)) goto done;
    {
        unsigned nc = ld_relaxed(A.ctr + kCtrCand);
        if (nc > A.cap_cand) nc = A.cap_cand;
        finalize_phase<KIND>(A, nc);
    }
    if (!grid_sync(A)) goto done;
    status_phase(A);

done:
    // per-CTA statistics
    {
        __shared__ unsigned long long s_pairs, s_bytes;
        __shared__ unsigned s_tri, s_ref;
        if (threadIdx.x == 0) { s_pairs = 0; s_bytes = 0; s_tri = 0; s_ref = 0; }
        __syncthreads();
        atomicAdd(&s_pairs, pairs);
        atomicAdd(&s_bytes, bytes);
        atomicAdd(&s_tri, tripairs);
        atomicAdd(&s_ref, refined);
        __syncthreads();
        if (threadIdx.x == 0) {
            atomicAdd(&A.stats->pairs_tested, s_pairs);
            atomicAdd(&A.stats->alg_bytes, s_bytes);
            atomicAdd(&A.stats->tri_pairs, s_tri);
            atomicAdd(&A.stats->refined, s_ref);
            // the last CTA out leaves the barrier and abort words clean for the
            // next launch and publishes this launch's abort flag
            __threadfence();
            unsigned e = atomicAdd(A.ctr + kCtrExit, 1u);
            if (e == gridDim.x - 1) {
                unsigned ab = atomicExch(A.ctr + kCtrAbort, 0u);
                atomicExch(A.ctr + kCtrLastAbort, ab);
                atomicExch(A.ctr + kCtrBarCount, 0u);
                atomicExch(A.ctr + kCtrExit, 0u);
                __threadfence();
            }
        }
    }
}

// ------------------------------------------------------------- host side

template <int KIND>
static int occupancy_blocks() {
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_query<KIND>, kBlock, 0);
    return nb;
}

int query_max_blocks_per_sm(int kind) { return kind == 0 ? occupancy_blocks<0>() : occupancy_blocks<1>(); }

cudaError_t launch_query(int kind, const KArgs& args, int grid, cudaStream_t stream) {
    void* params[] = {const_cast<KArgs*>(&args)};
    const void* fn = kind == 0 ? (const void*)k_query<0> : (const void*)k_query<1>;
    return cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(kBlock), params, 0, stream);
}

}  // namespace gd
