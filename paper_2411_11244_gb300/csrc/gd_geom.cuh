// Device geometry of the distance engine: closest points between triangle
// features (float32 for the narrow phase, float64 for the refinement) and
// the AABB distance bounds of Section 4 evaluated against a rigidly mapped
// box.
#pragma once

#include <cfloat>
#include <cmath>
#include <cuda_runtime.h>

namespace gd {

template <class T>
struct V3 {
    T x, y, z;
};

template <class T>
__device__ __forceinline__ V3<T> mk3(T x, T y, T z) {
    return V3<T>{x, y, z};
}

// Scalar arithmetic of the geometry.  float32: plain operators (the compiler
// may contract them into FMAs; every float32 result is only used inside
// bounds widened for such rounding).  float64: explicitly rounded
// intrinsics, never contracted, so that the float64 value of a feature is
// the same bits in every inlined copy and on every code path.
template <class T> __device__ __forceinline__ T sadd(T a, T b) { return a + b; }
template <class T> __device__ __forceinline__ T ssub(T a, T b) { return a - b; }
template <class T> __device__ __forceinline__ T smul(T a, T b) { return a * b; }
template <class T> __device__ __forceinline__ T sdiv(T a, T b) { return a / b; }
template <> __device__ __forceinline__ double sadd(double a, double b) { return __dadd_rn(a, b); }
template <> __device__ __forceinline__ double ssub(double a, double b) { return __dsub_rn(a, b); }
template <> __device__ __forceinline__ double smul(double a, double b) { return __dmul_rn(a, b); }
template <> __device__ __forceinline__ double sdiv(double a, double b) { return __ddiv_rn(a, b); }

template <class T>
__device__ __forceinline__ V3<T> operator+(V3<T> a, V3<T> b) {
    return mk3(sadd(a.x, b.x), sadd(a.y, b.y), sadd(a.z, b.z));
}
template <class T>
__device__ __forceinline__ V3<T> operator-(V3<T> a, V3<T> b) {
    return mk3(ssub(a.x, b.x), ssub(a.y, b.y), ssub(a.z, b.z));
}
template <class T>
__device__ __forceinline__ V3<T> operator*(V3<T> a, T s) {
    return mk3(smul(a.x, s), smul(a.y, s), smul(a.z, s));
}
template <class T>
__device__ __forceinline__ T dot(V3<T> a, V3<T> b) {
    return sadd(sadd(smul(a.x, b.x), smul(a.y, b.y)), smul(a.z, b.z));
}
template <class T>
__device__ __forceinline__ V3<T> cross(V3<T> a, V3<T> b) {
    return mk3(ssub(smul(a.y, b.z), smul(a.z, b.y)), ssub(smul(a.z, b.x), smul(a.x, b.z)),
               ssub(smul(a.x, b.y), smul(a.y, b.x)));
}
template <class T>
__device__ __forceinline__ T clamp01(T s) {
    return s < T(0) ? T(0) : (s > T(1) ? T(1) : s);
}

// num / den clamped to [0, 1], for den > 0: the clamped cases are decided on
// the numerator, so the (slow) division runs only for an interior value.
template <class T>
__device__ __forceinline__ T clamp_div(T num, T den) {
    if (!(num > T(0))) return T(0);
    if (num >= den) return T(1);
    return clamp01(sdiv(num, den));
}

// Closest point to p on the segment a + s d, s in [0, 1].
template <class T>
__device__ __forceinline__ V3<T> closest_on_segment(V3<T> p, V3<T> a, V3<T> d) {
    T dd = dot(d, d);
    T s = T(0);
    if (dd > T(0)) s = clamp_div(dot(p - a, d), dd);
    return a + d * s;
}

template <class T>
struct Tiny;
template <>
struct Tiny<float> {
    static constexpr float rel_det = 1e-7f;
};
template <>
struct Tiny<double> {
    static constexpr double rel_det = 1e-15;
};

// Closest point to p on triangle (a, b, c).  The projection onto the plane is
// expressed in the edge basis e0 = b - a, e1 = c - a by solving the 2x2 Gram
// system; if its barycentric weights lie in the triangle the projection is
// the answer, otherwise the answer lies on the boundary and is the nearest of
// the three edge projections.  *inside reports the first case.
template <class T>
__device__ __forceinline__ V3<T> closest_on_triangle(V3<T> p, V3<T> a, V3<T> b, V3<T> c, bool* inside) {
    V3<T> e0 = b - a, e1 = c - a, w = p - a;
    T g00 = dot(e0, e0), g01 = dot(e0, e1), g11 = dot(e1, e1);
    T det = ssub(smul(g00, g11), smul(g01, g01));
    if (det > smul(smul(Tiny<T>::rel_det, g00), g11) && det > T(0)) {
        T r0 = dot(w, e0), r1 = dot(w, e1);
        // barycentric weights u = un / det, v = vn / det: the inside test on
        // the numerators (det > 0), the divisions only for an inside point
        T un = ssub(smul(g11, r0), smul(g01, r1));
        T vn = ssub(smul(g00, r1), smul(g01, r0));
        if (un >= T(0) && vn >= T(0) && sadd(un, vn) <= det) {
            *inside = true;
            return a + e0 * sdiv(un, det) + e1 * sdiv(vn, det);
        }
    }
    *inside = false;
    V3<T> q0 = closest_on_segment(p, a, e0);
    V3<T> q1 = closest_on_segment(p, b, c - b);
    V3<T> q2 = closest_on_segment(p, a, e1);
    V3<T> d0 = p - q0, d1 = p - q1, d2 = p - q2;
    T n0 = dot(d0, d0), n1 = dot(d1, d1), n2 = dot(d2, d2);
    V3<T> q = q0;
    T n = n0;
    if (n1 < n) { n = n1; q = q1; }
    if (n2 < n) { q = q2; }
    return q;
}

// Projection of p onto the plane of triangle (a, b, c) when it falls inside
// the closed triangle (*inside), else nothing (p is returned).  The
// barycentric numerators and the determinant are dot products with the
// normal n = (b - a) x (c - a): u = ((p - a) x (c - a)).n, v = ((b - a) x
// (p - a)).n, det = n.n, which stay accurate for needle triangles where the
// Gram form g00 g11 - g01^2 cancels to nothing.  A feature pair whose
// projection falls outside needs no boundary fallback: the closest point is
// then on an edge of the triangle, at a distance no smaller than the
// edge-edge feature pair of that edge and an edge through p, which the
// triangle-pair distance takes anyway.
template <class T>
__device__ __forceinline__ V3<T> project_into_triangle(V3<T> p, V3<T> a, V3<T> b, V3<T> c, bool* inside) {
    const V3<T> e0 = b - a, e1 = c - a, w = p - a;
    const V3<T> n = cross(e0, e1);
    const T det = dot(n, n);
    const T un = dot(cross(w, e1), n), vn = dot(cross(e0, w), n);
    *inside = det > T(0) && un >= T(0) && vn >= T(0) && sadd(un, vn) <= det;
    if (!*inside) return p;
    return a + e0 * sdiv(un, det) + e1 * sdiv(vn, det);
}

// Whether the projection of p onto the plane of (a, b, c) falls inside the
// closed triangle (the test of project_into_triangle, without the point).
template <class T>
__device__ __forceinline__ bool projects_into_triangle(V3<T> p, V3<T> a, V3<T> b, V3<T> c) {
    const V3<T> e0 = b - a, e1 = c - a, w = p - a;
    const V3<T> n = cross(e0, e1);
    const T det = dot(n, n);
    const T un = dot(cross(w, e1), n), vn = dot(cross(e0, w), n);
    return det > T(0) && un >= T(0) && vn >= T(0) && sadd(un, vn) <= det;
}

// Closest points between segments p0 + s d1 and q0 + t d2, s, t in [0, 1].
// The squared distance is a convex quadratic in (s, t): take the stationary
// s (0 for parallel segments), clamp it, put t at its optimum for that s,
// and if t leaves [0, 1], clamp t and re-optimise s for the clamped t.
template <class T>
__device__ __forceinline__ void closest_segment_segment(V3<T> p0, V3<T> d1, V3<T> q0, V3<T> d2, V3<T>* P,
                                                        V3<T>* Q) {
    V3<T> r = p0 - q0;
    T a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r);
    T s, t;
    if (!(a > T(0)) && !(e > T(0))) {
        s = t = T(0);
    } else if (!(a > T(0))) {
        s = T(0);
        t = clamp_div(f, e);
    } else {
        T c = dot(d1, r);
        if (!(e > T(0))) {
            t = T(0);
            s = clamp_div(-c, a);
        } else {
            T b = dot(d1, d2);
            T den, num;
            if constexpr (sizeof(T) == 8) {
                // float64: the determinant a e - b^2 and the numerator
                // b f - c e as dot products of cross products (Binet-Cauchy:
                // (p x q).(u x v) = (p.u)(q.v) - (p.v)(q.u)), which keep
                // their accuracy for nearly parallel segments, where the
                // differences of products cancel to nothing and the interior
                // closest pair would be lost
                const V3<T> n = cross(d1, d2);
                den = dot(n, n);
                num = dot(n, cross(d2, r));
            } else {
                // float32 (bounds only, widened): the cheaper Gram form; a
                // stationary point lost to cancellation only loosens a bound
                den = ssub(smul(a, e), smul(b, b));
                num = ssub(smul(b, f), smul(c, e));
            }
            s = den > T(0) ? clamp_div(num, den) : T(0);
            T tn = sadd(smul(b, s), f);
            // t clamped to 0 or 1 re-optimises s; otherwise t = tn / e.  One
            // division on every path, so the lanes of a warp do not split
            // over three copies of it
            const bool lo = tn < T(0), hi = tn > e;
            const T r = clamp_div(lo ? -c : (hi ? ssub(b, c) : tn), (lo || hi) ? a : e);
            if (lo || hi) {
                t = lo ? T(0) : T(1);
                s = r;
            } else {
                t = r;
            }
        }
    }
    *P = p0 + d1 * s;
    *Q = q0 + d2 * t;
}

// Minimum distance between closed triangles A and B: the closest pair over the
// 6 vertex-face and 9 edge-edge feature pairs, plus, for every edge crossing
// the other triangle's plane, the crossing point against the other triangle
// (an interior crossing means the triangles intersect).  Returns the best
// pair (P on A, Q on B), its squared distance, and whether an interior
// crossing was found.
template <class T>
__device__ __forceinline__ void tri_tri_min(const V3<T>* A, const V3<T>* B, V3<T>* Pbest, V3<T>* Qbest, T* d2best,
                                            bool* hit) {
    T best = T(INFINITY);
    V3<T> P = A[0], Q = B[0];
    bool touched = false;
    auto consider = [&](V3<T> p, V3<T> q) {
        V3<T> d = p - q;
        T n = dot(d, d);
        if (n < best) { best = n; P = p; Q = q; }
    };
    bool in;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        consider(A[i], closest_on_triangle(A[i], B[0], B[1], B[2], &in));
        consider(closest_on_triangle(B[i], A[0], A[1], A[2], &in), B[i]);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            V3<T> p, q;
            closest_segment_segment(A[i], A[(i + 1) % 3] - A[i], B[j], B[(j + 1) % 3] - B[j], &p, &q);
            consider(p, q);
        }
    }
    // edges crossing the other triangle's plane
    V3<T> nA = cross(A[1] - A[0], A[2] - A[0]);
    V3<T> nB = cross(B[1] - B[0], B[2] - B[0]);
    T sa[3], sb[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        sa[i] = dot(nB, A[i] - B[0]);
        sb[i] = dot(nA, B[i] - A[0]);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        int j = (i + 1) % 3;
        if ((sa[i] <= T(0) && sa[j] >= T(0)) || (sa[i] >= T(0) && sa[j] <= T(0))) {
            T den = sa[i] - sa[j];
            if (den != T(0)) {
                V3<T> X = A[i] + (A[j] - A[i]) * clamp01(sa[i] / den);
                V3<T> Y = closest_on_triangle(X, B[0], B[1], B[2], &in);
                consider(X, Y);
                if (in) { touched = true; P = X; Q = X; best = T(0); }
            }
        }
        if ((sb[i] <= T(0) && sb[j] >= T(0)) || (sb[i] >= T(0) && sb[j] <= T(0))) {
            T den = sb[i] - sb[j];
            if (den != T(0)) {
                V3<T> X = B[i] + (B[j] - B[i]) * clamp01(sb[i] / den);
                V3<T> Y = closest_on_triangle(X, A[0], A[1], A[2], &in);
                consider(Y, X);
                if (in) { touched = true; P = X; Q = X; best = T(0); }
            }
        }
    }
    *Pbest = P;
    *Qbest = Q;
    *d2best = best;
    *hit = touched;
}

// Vertex i (0..2, a runtime value) of a triangle held in registers: a
// select chain, so that the triangle never has to live in local memory.
template <class T>
__device__ __forceinline__ V3<T> pick3(const V3<T>* X, int i) {
    V3<T> r = X[0];
    if (i == 1) r = X[1];
    if (i == 2) r = X[2];
    return r;
}

// One of the 21 feature pairs of the triangle-pair distance, for a warp that
// spreads them over its lanes: f in [0, 9) edge-edge, [9, 12) vertex of A
// vs B, [12, 15) vertex of B vs A, [15, 18) edge of A crossing B's plane,
// [18, 21) edge of B crossing A's plane.  A vertex-face pair counts only
// when the vertex projects inside the face, and a plane crossing only when it
// lies inside the face (then the triangles intersect: a hit); otherwise the
// closest pair of that feature is on an edge of the face, and the edge-edge
// pairs already hold a pair at most as far (see project_into_triangle).
// Lanes without a feature report an infinite distance.  The minimum over the
// 21 is the triangle-pair distance.
template <class T>
__device__ __forceinline__ void tri_feature(int f, const V3<T>* A, const V3<T>* B, V3<T>* P, V3<T>* Q, T* d2,
                                            bool* hit) {
    *hit = false;
    bool have = true, in = false;
    if (f < 9) {
        const int i = f / 3, j = f - 3 * (f / 3);
        const V3<T> a0 = pick3(A, i), a1 = pick3(A, i == 2 ? 0 : i + 1);
        const V3<T> b0 = pick3(B, j), b1 = pick3(B, j == 2 ? 0 : j + 1);
        closest_segment_segment(a0, a1 - a0, b0, b1 - b0, P, Q);
    } else if (f < 15) {
        // a vertex of one triangle against the other (one code path for both
        // directions: the lanes of a warp that hold f in [9, 15) do not split)
        const bool va = f < 12;
        const int i = f - (va ? 9 : 12);
        const V3<T> v = va ? pick3(A, i) : pick3(B, i);
        const V3<T> t0 = va ? B[0] : A[0], t1 = va ? B[1] : A[1], t2 = va ? B[2] : A[2];
        const V3<T> c = project_into_triangle(v, t0, t1, t2, &in);
        have = in;
        *P = va ? v : c;
        *Q = va ? c : v;
    } else if (f < 21) {
        const bool ea = f < 18;
        const int i = f - (ea ? 15 : 18), j = i == 2 ? 0 : i + 1;
        // edge owner E, plane owner F, all in registers
        const V3<T> e0 = ea ? pick3(A, i) : pick3(B, i), e1 = ea ? pick3(A, j) : pick3(B, j);
        const V3<T> f0 = ea ? B[0] : A[0], f1 = ea ? B[1] : A[1], f2 = ea ? B[2] : A[2];
        V3<T> n = cross(f1 - f0, f2 - f0);
        T si = dot(n, e0 - f0), sj = dot(n, e1 - f0);
        have = ((si <= T(0) && sj >= T(0)) || (si >= T(0) && sj <= T(0))) && ssub(si, sj) != T(0);
        if (have) {
            const V3<T> X = e0 + (e1 - e0) * clamp01(sdiv(si, ssub(si, sj)));
            have = projects_into_triangle(X, f0, f1, f2);
            if (have) { *hit = true; *P = X; *Q = X; }
        }
    } else {
        have = false;
    }
    if (have) {
        V3<T> d = *P - *Q;
        *d2 = *hit ? T(0) : dot(d, d);
    } else {
        *d2 = T(INFINITY);
    }
}

// The two point sets of feature pair f of tri_feature (an edge, a vertex or a
// whole triangle on each side), as three points each (an edge or a vertex
// repeats a point), for separation bounds.
template <class T>
__device__ __forceinline__ void feature_points(int f, const V3<T>* A, const V3<T>* B, V3<T>* PA, V3<T>* PB) {
    if (f < 9) {
        const int i = f / 3, j = f - 3 * (f / 3);
        PA[0] = pick3(A, i); PA[1] = pick3(A, i == 2 ? 0 : i + 1); PA[2] = PA[1];
        PB[0] = pick3(B, j); PB[1] = pick3(B, j == 2 ? 0 : j + 1); PB[2] = PB[1];
    } else if (f < 12) {
        PA[0] = pick3(A, f - 9); PA[1] = PA[0]; PA[2] = PA[0];
        PB[0] = B[0]; PB[1] = B[1]; PB[2] = B[2];
    } else if (f < 15) {
        PA[0] = A[0]; PA[1] = A[1]; PA[2] = A[2];
        PB[0] = pick3(B, f - 12); PB[1] = PB[0]; PB[2] = PB[0];
    } else if (f < 18) {
        const int i = f - 15;
        PA[0] = pick3(A, i); PA[1] = pick3(A, i == 2 ? 0 : i + 1); PA[2] = PA[1];
        PB[0] = B[0]; PB[1] = B[1]; PB[2] = B[2];
    } else {
        const int i = f - 18;
        PA[0] = A[0]; PA[1] = A[1]; PA[2] = A[2];
        PB[0] = pick3(B, i); PB[1] = pick3(B, i == 2 ? 0 : i + 1); PB[2] = PB[1];
    }
}

// Farthest vertex pair (the maximum over two triangles is attained at vertices).
template <class T>
__device__ __forceinline__ void tri_tri_max(const V3<T>* A, const V3<T>* B, V3<T>* P, V3<T>* Q, T* d2) {
    T best = T(-1);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            V3<T> d = A[i] - B[j];
            T n = dot(d, d);
            if (n > best) { best = n; *P = A[i]; *Q = B[j]; }
        }
    *d2 = best;
}

// ---------------------------------------------------------------- double-float
// A value carried as an unevaluated float32 sum hi + lo (about 48 significant
// bits), built from error-free transformations on the float32 pipe.  Every
// step uses explicitly rounded intrinsics so that no contraction or
// reassociation can change it.

struct DF {
    float hi, lo;
};

// s + e == a + b exactly (Knuth's two-sum)
__device__ __forceinline__ DF two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return DF{s, e};
}

// s + e == a + b exactly when |a| >= |b|
__device__ __forceinline__ DF fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF df_add(DF a, DF b) {
    DF s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

// (hi + lo) * b for a float32 b: the product of the leading parts is exact
// (its error term recovered by an FMA), the rest adds a relative 2^-48
__device__ __forceinline__ DF df_mul_f(DF a, float b) {
    float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    return fast_two_sum(p, __fmaf_rn(a.lo, b, e));
}

// ---------------------------------------------------------------- transforms

struct Rigid32 {
    float R[9], t[3];
};

// float32 map x -> R x + t, one FMA chain per coordinate
__device__ __forceinline__ V3<float> map32(const Rigid32& X, float x, float y, float z) {
    return mk3(fmaf(X.R[0], x, fmaf(X.R[1], y, fmaf(X.R[2], z, X.t[0]))),
               fmaf(X.R[3], x, fmaf(X.R[4], y, fmaf(X.R[5], z, X.t[1]))),
               fmaf(X.R[6], x, fmaf(X.R[7], y, fmaf(X.R[8], z, X.t[2]))));
}

__device__ __forceinline__ V3<double> map64(const double* X, double x, double y, double z) {
    return mk3(fma(X[0], x, fma(X[1], y, fma(X[2], z, X[3]))), fma(X[4], x, fma(X[5], y, fma(X[6], z, X[7]))),
               fma(X[8], x, fma(X[9], y, fma(X[10], z, X[11]))));
}

// ---------------------------------------------------------------- bounds

// Box with lo[3], hi[3].
struct Box {
    float lo[3], hi[3];
};

// Axis-aligned box enclosing the mapped box b (centre +- |R| half-extent).
__device__ __forceinline__ void enclose(const Rigid32& X, const Box& b, float* elo, float* ehi) {
    float m0 = 0.5f * (b.lo[0] + b.hi[0]), m1 = 0.5f * (b.lo[1] + b.hi[1]), m2 = 0.5f * (b.lo[2] + b.hi[2]);
    float h0 = 0.5f * (b.hi[0] - b.lo[0]), h1 = 0.5f * (b.hi[1] - b.lo[1]), h2 = 0.5f * (b.hi[2] - b.lo[2]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        float c = fmaf(X.R[3 * i], m0, fmaf(X.R[3 * i + 1], m1, fmaf(X.R[3 * i + 2], m2, X.t[i])));
        float e = fmaf(fabsf(X.R[3 * i]), h0, fmaf(fabsf(X.R[3 * i + 1]), h1, fabsf(X.R[3 * i + 2]) * h2));
        elo[i] = c - e;
        ehi[i] = c + e;
    }
}

// Eqs. 5-6: squared conventional lower bound of the min distance.
__device__ __forceinline__ float lower_min_sq(const Box& a, const float* elo, const float* ehi) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float g = fmaxf(0.f, fmaxf(a.lo[k] - ehi[k], elo[k] - a.hi[k]));
        s = fmaf(g, g, s);
    }
    return s;
}

// Eqs. 7-8: squared conventional upper bound of the max distance.
__device__ __forceinline__ float upper_max_sq(const Box& a, const float* elo, const float* ehi) {
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float f = fmaxf(fabsf(a.lo[k] - ehi[k]), fabsf(a.hi[k] - elo[k]));
        s = fmaf(f, f, s);
    }
    return s;
}

// Corner m of box b (bit k of m selects hi on axis k), mapped by X unless the
// box is already expressed in the working frame (AA).
template <bool AA>
__device__ __forceinline__ V3<float> mapped_corner(const Rigid32& X, const Box& b, int m) {
    const float x = (m & 1) ? b.hi[0] : b.lo[0], y = (m & 2) ? b.hi[1] : b.lo[1], z = (m & 4) ? b.hi[2] : b.lo[2];
    if (AA) return mk3(x, y, z);
    return map32(X, x, y, z);
}

// Eq. 10: squared enhanced upper bound of the min distance,
//   min over faces i of a, faces j of b of max over P in face i, Q in face j of |PQ|.
// For a fixed corner Q of the mapped face j, the farthest point of the
// axis-aligned face i (axis k at coordinate f) is at squared distance
//   (Q_k - f)^2 + sum over the other axes l of max((Q_l - lo_l)^2, (Q_l - hi_l)^2),
// and the maximum over face j is attained at one of its 4 corners.
template <bool AA>
__device__ __forceinline__ float upper_min_sq_enhanced(const Rigid32& X, const Box& a, const Box& b) {
    V3<float> c[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) c[m] = mapped_corner<AA>(X, b, m);
    float best = FLT_MAX;
    // face j of b: axis l, side sl; its corners are those with bit l == sl
#pragma unroll
    for (int l = 0; l < 3; ++l) {
#pragma unroll
        for (int sl = 0; sl < 2; ++sl) {
            float run[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                if (((m >> l) & 1) != sl) continue;
                const float cc[3] = {c[m].x, c[m].y, c[m].z};
                float dl[3], dh[3], M2[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    dl[k] = cc[k] - a.lo[k];
                    dh[k] = cc[k] - a.hi[k];
                    M2[k] = fmaxf(dl[k] * dl[k], dh[k] * dh[k]);
                }
                const float Pk[3] = {M2[1] + M2[2], M2[0] + M2[2], M2[0] + M2[1]};
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    run[2 * k] = fmaxf(run[2 * k], fmaf(dl[k], dl[k], Pk[k]));
                    run[2 * k + 1] = fmaxf(run[2 * k + 1], fmaf(dh[k], dh[k], Pk[k]));
                }
            }
#pragma unroll
            for (int i = 0; i < 6; ++i) best = fminf(best, run[i]);
        }
    }
    return best;
}

// Eq. 11 (as a valid lower bound): squared lower bound of the max distance,
//   max over faces i of a, faces j of b of the min distance between face i
//   and the axis-aligned box enclosing the 4 mapped corners of face j
//   (that box contains face j, so its distance does not exceed the face's;
//   with no rotation it is the face itself and the bound is Eq. 11 exactly).
template <bool AA>
__device__ __forceinline__ float lower_max_sq_enhanced(const Rigid32& X, const Box& a, const Box& b) {
    V3<float> c[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) c[m] = mapped_corner<AA>(X, b, m);
    float best = 0.f;
#pragma unroll
    for (int l = 0; l < 3; ++l) {
#pragma unroll
        for (int sl = 0; sl < 2; ++sl) {
            float flo[3] = {FLT_MAX, FLT_MAX, FLT_MAX}, fhi[3] = {-FLT_MAX, -FLT_MAX, -FLT_MAX};
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                if (((m >> l) & 1) != sl) continue;
                float cc[3] = {c[m].x, c[m].y, c[m].z};
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    flo[k] = fminf(flo[k], cc[k]);
                    fhi[k] = fmaxf(fhi[k], cc[k]);
                }
            }
            // per-axis gaps between a's full extent and the face box
            float g[3], gf[3][2];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                g[k] = fmaxf(0.f, fmaxf(a.lo[k] - fhi[k], flo[k] - a.hi[k]));
                gf[k][0] = fmaxf(0.f, fmaxf(a.lo[k] - fhi[k], flo[k] - a.lo[k]));
                gf[k][1] = fmaxf(0.f, fmaxf(a.hi[k] - fhi[k], flo[k] - a.hi[k]));
            }
            float g2[3] = {g[0] * g[0], g[1] * g[1], g[2] * g[2]};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                float o = g2[(k + 1) % 3] + g2[(k + 2) % 3];
#pragma unroll
                for (int s = 0; s < 2; ++s) best = fmaxf(best, fmaf(gf[k][s], gf[k][s], o));
            }
        }
    }
    return best;
}

}  // namespace gd
