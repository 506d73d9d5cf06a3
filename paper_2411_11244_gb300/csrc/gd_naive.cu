// The "naive" GPU distance query the paper compares against (Section 8,
// Performance): one thread per triangle of A walks B's BVH depth first,
// nearer child first, and prunes with one global running bound that every
// thread reads and updates with atomics.  It is a comparator only: float32
// throughout, no BVTT front, no load balancing.  The paper reports that it
// visits at least nine times (usually dozens of times) more BVTT nodes than
// the front traversal and suffers from threads whose walks are far longer
// than the rest; node_tests and max_thread_tests measure exactly that.
//
// Every walk is bounded: by the size of B's tree, and by a deadline that the
// first thread to start stamps (threads past it stop, and the query reports
// a timeout).
#include <cfloat>
#include <cstdint>

#include "gd_geom.cuh"
#include "gd_internal.cuh"
#include "gd_launch.h"

namespace gd {

namespace {

constexpr int kNaiveThreads = 256;
constexpr int kStack = 40;  // B has at most 31 levels: a walk holds at most L_B + 2 entries

__device__ __forceinline__ unsigned leaf_begin(long long T, int L, unsigned leaf) {
    return (unsigned)(((unsigned long long)leaf * (unsigned long long)T) >> L);
}

__device__ __forceinline__ void load_tri3(const float4* tri, unsigned j, V3<float>* v) {
    const float4 p = __ldg(tri + 3ull * j), q = __ldg(tri + 3ull * j + 1), r = __ldg(tri + 3ull * j + 2);
    v[0] = mk3(p.x, p.y, p.z);
    v[1] = mk3(p.w, q.x, q.y);
    v[2] = mk3(q.z, q.w, r.x);
}

__device__ __forceinline__ Box load_box(const float* box, unsigned node) {
    const float* b = box + 6ull * node;
    Box x;
    x.lo[0] = __ldg(b); x.lo[1] = __ldg(b + 1); x.lo[2] = __ldg(b + 2);
    x.hi[0] = __ldg(b + 3); x.hi[1] = __ldg(b + 4); x.hi[2] = __ldg(b + 5);
    return x;
}

__global__ void k_naive_init(unsigned long long* ws, int kind) {
    if (threadIdx.x < kNaiveWords) ws[threadIdx.x] = 0ull;
    if (threadIdx.x == 0) ws[kNaiveU] = kind == 0 ? 0x7f800000ull : 0ull;  // +inf / 0 as float bits
}

// squared-distance bound of B's node against the box of the mapped triangle:
// Eqs. 5-6 (lower bound of the min) or Eqs. 7-8 (upper bound of the max)
template <int KIND>
__device__ __forceinline__ float node_bound(const float* box, unsigned node, const float* tlo, const float* thi) {
    const Box b = load_box(box, node);
    return KIND == 0 ? lower_min_sq(b, tlo, thi) : upper_max_sq(b, tlo, thi);
}

template <int KIND>
__device__ __forceinline__ bool prunes(float bound, float U) {
    return KIND == 0 ? bound > U : bound < U;
}

template <int KIND>
__global__ void __launch_bounds__(kNaiveThreads) k_naive(NaiveArgs g) {
    unsigned long long* ws = g.ws;
    unsigned* U = reinterpret_cast<unsigned*>(ws + kNaiveU);
    __shared__ unsigned long long s_deadline;
    __shared__ int s_late;
    if (threadIdx.x == 0) {
        const unsigned long long now = globaltimer();
        const unsigned long long old = atomicCAS(ws + kNaiveT0, 0ull, now);
        s_deadline = (old ? old : now) + (unsigned long long)g.timeout_ns;
        // a CTA that starts past the deadline does no work
        s_late = now > s_deadline || ld_relaxed64(ws + kNaiveTimeout) != 0ull;
        if (now > s_deadline) atomicExch(ws + kNaiveTimeout, 1ull);
    }
    __syncthreads();
    const unsigned long long deadline = s_deadline;
    const long long i = (long long)blockIdx.x * kNaiveThreads + threadIdx.x;
    unsigned long long tests = 0, leaves = 0;
    if (i < g.TA && !s_late) {
        // triangle i of A (leaf order), mapped into B's frame; its box widened
        // by the float32 mapping error
        V3<float> a[3];
        load_tri3(g.triA, (unsigned)i, a);
        Rigid32 X;
#pragma unroll
        for (int k = 0; k < 9; ++k) X.R[k] = g.R[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) X.t[k] = g.t[k];
        float tlo[3], thi[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) a[k] = map32(X, a[k].x, a[k].y, a[k].z);
        tlo[0] = fminf(a[0].x, fminf(a[1].x, a[2].x)) - g.E;
        tlo[1] = fminf(a[0].y, fminf(a[1].y, a[2].y)) - g.E;
        tlo[2] = fminf(a[0].z, fminf(a[1].z, a[2].z)) - g.E;
        thi[0] = fmaxf(a[0].x, fmaxf(a[1].x, a[2].x)) + g.E;
        thi[1] = fmaxf(a[0].y, fmaxf(a[1].y, a[2].y)) + g.E;
        thi[2] = fmaxf(a[0].z, fmaxf(a[1].z, a[2].z)) + g.E;
        const unsigned first_leaf = 1u << g.LB;
        unsigned st_node[kStack];
        float st_bound[kStack];
        int sp = 0;
        st_node[0] = 1u;
        st_bound[0] = node_bound<KIND>(g.boxB, 1u, tlo, thi);
        sp = 1;
        tests = 1;
        for (unsigned iter = 1; sp > 0; ++iter) {
            if ((iter & 127u) == 0u && globaltimer() > deadline) {
                atomicExch(ws + kNaiveTimeout, 1ull);
                break;
            }
            --sp;
            const unsigned node = st_node[sp];
            float u = __uint_as_float(ld_relaxed(U));
            if (prunes<KIND>(st_bound[sp], u)) continue;
            if (node >= first_leaf) {
                const unsigned l = node - first_leaf;
                const unsigned j1 = leaf_begin(g.TB, g.LB, l + 1);
                for (unsigned j = leaf_begin(g.TB, g.LB, l); j < j1; ++j) {
                    V3<float> b[3];
                    load_tri3(g.triB, j, b);
                    V3<float> P, Q;
                    float d2;
                    ++leaves;
                    if (KIND == 0) {
                        bool hit;
                        tri_tri_min<float>(a, b, &P, &Q, &d2, &hit);
                        if (hit) d2 = 0.f;
                        if (d2 < u) u = fminf(d2, __uint_as_float(atomicMin(U, __float_as_uint(d2))));
                    } else {
                        tri_tri_max<float>(a, b, &P, &Q, &d2);
                        if (d2 > u) u = fmaxf(d2, __uint_as_float(atomicMax(U, __float_as_uint(d2))));
                    }
                }
                continue;
            }
            if (sp + 2 > kStack) {  // cannot happen for a tree of at most 31 levels
                atomicExch(ws + kNaiveBad, 1ull);
                break;
            }
            const float b0 = node_bound<KIND>(g.boxB, 2u * node, tlo, thi);
            const float b1 = node_bound<KIND>(g.boxB, 2u * node + 1u, tlo, thi);
            tests += 2;
            // the more promising child goes on top
            const bool first0 = KIND == 0 ? b0 <= b1 : b0 >= b1;
            st_node[sp] = first0 ? 2u * node + 1u : 2u * node;
            st_bound[sp] = first0 ? b1 : b0;
            st_node[sp + 1] = first0 ? 2u * node : 2u * node + 1u;
            st_bound[sp + 1] = first0 ? b0 : b1;
            sp += 2;
        }
    }
    // warp totals, then one atomic per warp
    unsigned long long t = tests, l = leaves, m = tests;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        t += __shfl_down_sync(kFull, t, o);
        l += __shfl_down_sync(kFull, l, o);
        const unsigned long long mo = __shfl_down_sync(kFull, m, o);
        m = mo > m ? mo : m;
    }
    if ((threadIdx.x & 31) == 0) {
        if (t) atomicAdd(ws + kNaiveTests, t);
        if (l) atomicAdd(ws + kNaiveLeaves, l);
        if (m) atomicMax(ws + kNaiveMaxTests, m);
    }
}

}  // namespace

cudaError_t launch_naive(int kind, const NaiveArgs& g, cudaStream_t st) {
    k_naive_init<<<1, 32, 0, st>>>(g.ws, kind);
    const unsigned grid = (unsigned)((g.TA + kNaiveThreads - 1) / kNaiveThreads);
    if (kind == 0) k_naive<0><<<grid, kNaiveThreads, 0, st>>>(g);
    else k_naive<1><<<grid, kNaiveThreads, 0, st>>>(g);
    return cudaGetLastError();
}

}  // namespace gd
