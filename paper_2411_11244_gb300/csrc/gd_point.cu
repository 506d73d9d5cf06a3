// Point-to-mesh distance (the 1-to-N direction the paper names as future
// work in Section 10, with points as the N queries): for each query point,
// the closest point of a mesh placed by a rigid transform, exact in float64.
//
// One thread per point walks the mesh's f12-BVH depth first, nearer child
// first, with its own running bound (no atomics: the points are independent
// problems).  Float64 stays off the walk: every triangle reached gets its
// float32 closest point, which gives a rigorous float32 upper bound of its
// distance (lowering the bound) and a rigorous lower bound (its separation
// from the point along the direction to that closest point, widened for the
// float32 error of the mapped point and of the arithmetic); only triangles
// whose lower bound is within the bound get their float64 distance, and the
// least (d, original index) pair wins.  Pruning only ever drops triangles
// that are provably farther than a true distance, so the answer is the exact
// minimum over all triangles, the smallest original index among ties.  The
// separation test keeps float64 work to the near-ties even for a point that
// many triangles surround at nearly one distance (the centre of a ring or a
// sphere).
#include <cfloat>
#include <cstdint>

#include "gd_geom.cuh"
#include "gd_internal.cuh"
#include "gd_launch.h"

namespace gd {

namespace {

constexpr int kPointThreads = 128;
constexpr int kStack = 40;  // a walk of a tree of at most 31 levels holds at most L + 2 entries

__device__ __forceinline__ unsigned leaf_begin(long long T, int L, unsigned leaf) {
    return (unsigned)(((unsigned long long)leaf * (unsigned long long)T) >> L);
}

__device__ __forceinline__ void load_tri(const float4* tri, unsigned j, V3<float>* v, int* id) {
    const float4 p = __ldg(tri + 3ull * j), q = __ldg(tri + 3ull * j + 1), r = __ldg(tri + 3ull * j + 2);
    v[0] = mk3(p.x, p.y, p.z);
    v[1] = mk3(p.w, q.x, q.y);
    v[2] = mk3(q.z, q.w, r.x);
    *id = __float_as_int(r.y);
}

// squared distance from the box [c - E, c + E] to the box [lo, hi]; every
// float32 step rounds at most one unit, so the caller compares it against
// its bound grown by 2^-20 relative
__device__ __forceinline__ float gap_sq(const float* lo, const float* hi, V3<float> c, float E) {
    const float cc[3] = {c.x, c.y, c.z};
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float g = fmaxf(0.f, fmaxf(lo[k] - (cc[k] + E), (cc[k] - E) - hi[k]));
        s = fmaf(g, g, s);
    }
    return s;
}

__device__ __forceinline__ float node_gap_sq(const float* box, unsigned node, V3<float> c, float E) {
    const float* b = box + 6ull * node;
    const float lo[3] = {__ldg(b), __ldg(b + 1), __ldg(b + 2)};
    const float hi[3] = {__ldg(b + 3), __ldg(b + 4), __ldg(b + 5)};
    return gap_sq(lo, hi, c, E);
}

// Rigorous float32 lower bound of the squared distance from any point within
// E (per coordinate) of c to triangle v: the separation of the point from
// the triangle along the axis u = c - q, q the float32 closest point (any
// axis separates validly; this one is nearly the exact direction, so the
// bound is nearly tight).  Every dot product is taken down by a margin of
// 2^-20 of its absolute terms, and E is charged against the point.
__device__ __forceinline__ float sep_lower_sq(V3<float> c, float E, const V3<float>* v, V3<float> q) {
    const V3<float> u = c - q;
    const float uu = dot(u, u);
    if (!(uu > 0.f)) return 0.f;
    const float au = fabsf(u.x) + fabsf(u.y) + fabsf(u.z);
    float smin = INFINITY, mag = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const V3<float> w = c - v[k];
        smin = fminf(smin, dot(u, w));
        mag = fmaxf(mag, fabsf(u.x) * (fabsf(c.x) + fabsf(v[k].x)) + fabsf(u.y) * (fabsf(c.y) + fabsf(v[k].y)) +
                             fabsf(u.z) * (fabsf(c.z) + fabsf(v[k].z)));
    }
    const float num = smin - mag * 0x1p-20f - E * au;
    if (!(num > 0.f)) return 0.f;
    return num * num / uu * (1.f - 0x1p-20f);
}

__device__ __forceinline__ double dist2_64(V3<double> p, const V3<float>* v, V3<double>* q) {
    bool inside;
    const V3<double> a = mk3((double)v[0].x, (double)v[0].y, (double)v[0].z);
    const V3<double> b = mk3((double)v[1].x, (double)v[1].y, (double)v[1].z);
    const V3<double> c = mk3((double)v[2].x, (double)v[2].y, (double)v[2].z);
    *q = closest_on_triangle<double>(p, a, b, c, &inside);
    const V3<double> d = p - *q;
    return dot(d, d);
}

__device__ __forceinline__ float abs_max(V3<float> a) { return fmaxf(fabsf(a.x), fmaxf(fabsf(a.y), fabsf(a.z))); }

// Rigorous float32 upper bound of the squared distance from any point within
// E (per coordinate) of c to triangle v, given q, its float32 closest point
// to c: q lies within a few units in the last place of the largest vertex
// coordinate M of a point of the triangle (its barycentric or edge parameter
// is clamped to the triangle, the rounding of the point's arithmetic is
// charged as 2^-18 M per coordinate), so |c - q| grown by that and by E
// bounds the true distance from above.  Rounded up throughout.
__device__ __forceinline__ float upper_sq(V3<float> c, float E, const V3<float>* v, V3<float> q) {
    const V3<float> d = c - q;
    const float M = fmaxf(abs_max(v[0]), fmaxf(abs_max(v[1]), abs_max(v[2])));
    const float slack = __fmul_ru(1.7320509f, __fadd_ru(E, __fmul_ru(M, 0x1p-18f)));
    const float len = __fmul_ru(__fsqrt_ru(dot(d, d)), 1.f + 0x1p-20f);
    const float up = __fadd_ru(len, slack);
    return __fmul_ru(up, up);
}

// One depth-first walk, nearer child first, with a running bound U (squared)
// that is a true upper bound of the answer at every step: each triangle
// reached gets its float32 closest point, whose rigorous upper bound lowers
// U, and a rigorous lower bound (the separation along the direction to that
// point) decides whether the triangle can hold the minimum; those that can
// get their float64 distance at once (least (d2, original index) kept).
// Boxes and triangles beyond U are dropped, so every triangle at the
// minimum is evaluated in float64; one evaluated while U was still looser
// only costs work.
__device__ bool walk(const PointArgs& g, V3<float> c, float E, V3<double> p64, double* best_d2, int* best_id,
                     V3<double>* best_q, unsigned long long* tests, unsigned long long* exact,
                     unsigned long long deadline) {
    const unsigned first_leaf = 1u << g.L;
    const float grow = 1.f + 0x1p-20f;
    unsigned st_node[kStack];
    float st_gap[kStack];
    st_node[0] = 1u;
    st_gap[0] = node_gap_sq(g.box, 1u, c, E);
    int sp = 1;
    *tests += 1;
    float U = INFINITY;
    for (unsigned iter = 1; sp > 0; ++iter) {
        if ((iter & 127u) == 0u && globaltimer() > deadline) return false;
        --sp;
        const unsigned node = st_node[sp];
        if (st_gap[sp] > U * grow) continue;
        if (node >= first_leaf) {
            const unsigned l = node - first_leaf;
            const unsigned j1 = leaf_begin(g.T, g.L, l + 1);
            for (unsigned j = leaf_begin(g.T, g.L, l); j < j1; ++j) {
                V3<float> v[3];
                int id;
                load_tri(g.tri, j, v, &id);
                const float lo[3] = {fminf(v[0].x, fminf(v[1].x, v[2].x)), fminf(v[0].y, fminf(v[1].y, v[2].y)),
                                     fminf(v[0].z, fminf(v[1].z, v[2].z))};
                const float hi[3] = {fmaxf(v[0].x, fmaxf(v[1].x, v[2].x)), fmaxf(v[0].y, fmaxf(v[1].y, v[2].y)),
                                     fmaxf(v[0].z, fmaxf(v[1].z, v[2].z))};
                if (gap_sq(lo, hi, c, E) > U * grow) continue;
                bool inside;
                const V3<float> q32 = closest_on_triangle<float>(c, v[0], v[1], v[2], &inside);
                U = fminf(U, upper_sq(c, E, v, q32));
                if (sep_lower_sq(c, E, v, q32) > U * grow) continue;
                V3<double> q;
                const double d2 = dist2_64(p64, v, &q);
                *exact += 1;
                if (d2 < *best_d2 || (d2 == *best_d2 && id < *best_id)) {
                    *best_d2 = d2;
                    *best_id = id;
                    *best_q = q;
                    U = fminf(U, __double2float_ru(d2));
                }
            }
            continue;
        }
        if (sp + 2 > kStack) return false;  // cannot happen for a tree of at most 31 levels
        const float g0 = node_gap_sq(g.box, 2u * node, c, E);
        const float g1 = node_gap_sq(g.box, 2u * node + 1u, c, E);
        *tests += 2;
        const bool near0 = g0 <= g1;
        st_node[sp] = near0 ? 2u * node + 1u : 2u * node;
        st_gap[sp] = near0 ? g1 : g0;
        st_node[sp + 1] = near0 ? 2u * node : 2u * node + 1u;
        st_gap[sp + 1] = near0 ? g0 : g1;
        sp += 2;
    }
    return true;
}

__global__ void __launch_bounds__(kPointThreads) k_point(PointArgs g) {
    unsigned long long* ws = g.ws;
    __shared__ unsigned long long s_deadline;
    if (threadIdx.x == 0) {
        const unsigned long long now = globaltimer();
        const unsigned long long old = atomicCAS(ws + kPointT0, 0ull, now);
        s_deadline = (old ? old : now) + (unsigned long long)g.timeout_ns;
    }
    __syncthreads();
    const long long t = (long long)blockIdx.x * kPointThreads + threadIdx.x;
    const long long i = t < g.n && g.order ? (long long)g.order[t] : t;
    unsigned long long tests = 0, exact = 0;
    if (i < g.n && !(isfinite(g.pts[3 * i]) && isfinite(g.pts[3 * i + 1]) && isfinite(g.pts[3 * i + 2]))) {
        gd_point_result r{};
        r.d = NAN;
        r.tri = -1;
        r.status = GD_ERR_INVALID_ARG;
        g.out[i] = r;
    } else if (i < g.n) {
        // the point in the mesh's frame: R^T (p - t) in float64
        const double* P = g.pts + 3 * i;
        const double w0 = P[0] - g.x[3], w1 = P[1] - g.x[7], w2 = P[2] - g.x[11];
        const V3<double> p64 = mk3(fma(g.x[0], w0, fma(g.x[4], w1, g.x[8] * w2)),
                                   fma(g.x[1], w0, fma(g.x[5], w1, g.x[9] * w2)),
                                   fma(g.x[2], w0, fma(g.x[6], w1, g.x[10] * w2)));
        const V3<float> c = mk3((float)p64.x, (float)p64.y, (float)p64.z);
        // float32 rounding of the mapped point, plus margin
        const float E = fmaxf(fabsf(c.x), fmaxf(fabsf(c.y), fabsf(c.z))) * 0x1p-22f + FLT_MIN;
        gd_point_result r{};
        r.tri = -1;
        double d2 = INFINITY;
        int id = 0x7fffffff;
        V3<double> q = mk3(0.0, 0.0, 0.0);
        const bool ok = walk(g, c, E, p64, &d2, &id, &q, &tests, &exact, s_deadline);
        if (ok && id != 0x7fffffff) {
            r.d = sqrt(d2);
            r.tri = id;
            // the closest point in the world frame: R q + t
            r.p[0] = fma(g.x[0], q.x, fma(g.x[1], q.y, fma(g.x[2], q.z, g.x[3])));
            r.p[1] = fma(g.x[4], q.x, fma(g.x[5], q.y, fma(g.x[6], q.z, g.x[7])));
            r.p[2] = fma(g.x[8], q.x, fma(g.x[9], q.y, fma(g.x[10], q.z, g.x[11])));
            r.status = GD_OK;
        } else {
            r.status = GD_ERR_TIMEOUT;
            atomicExch(ws + kPointTimeout, 1ull);
        }
        g.out[i] = r;
    }
    unsigned long long nt = tests, ne = exact;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nt += __shfl_down_sync(kFull, nt, o);
        ne += __shfl_down_sync(kFull, ne, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (nt) atomicAdd(ws + kPointTests, nt);
        if (ne) atomicAdd(ws + kPointExact, ne);
    }
}

// 10 bits of v spread to every third bit
__device__ __forceinline__ unsigned long long spread10(unsigned v) {
    unsigned long long r = 0;
#pragma unroll
    for (int b = 0; b < 10; ++b) r |= (unsigned long long)((v >> b) & 1u) << (3 * b);
    return r;
}

// Morton key of each point in the mesh's frame, quantised in the root box
// (points outside clamp to its faces: the key only orders the work)
__global__ void k_point_keys(PointArgs g, unsigned long long* keys, unsigned* vals) {
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.n) return;
    const double* P = g.pts + 3 * i;
    const double w0 = P[0] - g.x[3], w1 = P[1] - g.x[7], w2 = P[2] - g.x[11];
    const double l[3] = {g.x[0] * w0 + g.x[4] * w1 + g.x[8] * w2, g.x[1] * w0 + g.x[5] * w1 + g.x[9] * w2,
                         g.x[2] * w0 + g.x[6] * w1 + g.x[10] * w2};
    unsigned long long key = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = g.box[6 + k], hi = g.box[9 + k];
        const float ext = hi - lo;
        float f = ext > 0.f ? (float)((l[k] - lo) / ext) : 0.f;
        f = f == f ? fminf(fmaxf(f, 0.f), 1.f) : 0.f;  // NaN (a non-finite point) to 0
        const unsigned c = min(1023u, (unsigned)(f * 1024.f));
        key |= spread10(c) << k;
    }
    keys[i] = key;
    vals[i] = (unsigned)i;
}

__global__ void k_point_init(unsigned long long* ws) {
    if (threadIdx.x < kPointWords) ws[threadIdx.x] = 0ull;
}

}  // namespace

int sort_points(const PointArgs& g, unsigned long long* const keys[2], unsigned* const vals[2], unsigned* hist,
                cudaStream_t st) {
    k_point_keys<<<(unsigned)((g.n + 255) / 256), 256, 0, st>>>(g, keys[0], vals[0]);
    return radix_sort_pairs(keys, vals, g.n, 30, hist, st);
}

cudaError_t launch_point(const PointArgs& g, cudaStream_t st) {
    k_point_init<<<1, 32, 0, st>>>(g.ws);
    if (g.n > 0) {
        const unsigned grid = (unsigned)((g.n + kPointThreads - 1) / kPointThreads);
        k_point<<<grid, kPointThreads, 0, st>>>(g);
    }
    return cudaGetLastError();
}

}  // namespace gd
