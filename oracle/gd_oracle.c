/*
 * FP64 CPU oracle for mesh-mesh distance -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the package's smoke check and the benchmark's CPU-baseline
 * leg load this library.  It shares no code, header, table or helper with the
 * CUDA engine; it is a plain, slow, obviously correct statement of what the
 * engine computes:
 *
 *   D_min = min over p in P, q in Q of ||p - q||      (Section 3, Eq. 1)
 *   D_max = max over p in P, q in Q of ||p - q||      (Section 3, Eq. 2)
 *
 * with P and Q the closed triangle surfaces of two meshes placed in the world
 * by rigid transforms x = R v + t (row-major 3x4 [R|t], float64), applied in
 * float64 to the float32 input vertices.  Intersecting meshes have D_min = 0
 * (Section 8, implementation notes on penetration).
 *
 * Triangle-triangle distance: 0 if the closed triangles intersect, otherwise
 * the minimum over the 9 edge-edge segment distances and the 6 vertex-face
 * distances.  For disjoint triangles a closest pair always involves a vertex
 * of one triangle or a point on an edge of each, so these 15 cases cover it.
 * Each primitive is written from its definition:
 *   - point-segment: clamped projection onto the segment;
 *   - point-triangle: projection onto the plane if it falls inside, else the
 *     nearest of the three edges;
 *   - segment-segment: the convex quadratic |p(s) - q(t)|^2 on [0,1]^2 attains
 *     its minimum either at the interior stationary point or on the boundary
 *     of the square, and the boundary is four point-segment problems;
 *   - intersection: an edge of one triangle crosses the plane of the other at
 *     a point inside it (coplanar overlap shows up as a zero edge-edge or
 *     vertex-face distance instead).
 * D_max between two triangles is attained at a vertex pair, since the
 * distance is convex in each argument.
 *
 * Witness rule: among pairs with the same float64 distance the
 * lexicographically smallest (triangle of A, triangle of B) is reported.
 *
 * Two evaluation strategies, both exact definitions up to float64 rounding:
 *   brute force over all triangle pairs (threaded over rows), and
 *   a best-first traversal of the oracle's own median-split AABB tree (built
 *   in each mesh's local frame; node boxes are mapped to the world by the
 *   enclosing box of the transformed box), pruning a node pair only when its
 *   lower (upper) bound is strictly beyond the current best.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_API __attribute__((visibility("default")))

typedef struct { double x, y, z; } v3;

static inline v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static inline v3 vsub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static inline v3 vadd(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static inline v3 vscale(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static inline double vdot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static inline v3 vcross(v3 a, v3 b) {
    return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static inline double vdist(v3 a, v3 b) { v3 d = vsub(a, b); return sqrt(vdot(d, d)); }
static inline v3 ld(const double *p) { return mk(p[0], p[1], p[2]); }
static inline void st(double *p, v3 a) { p[0] = a.x; p[1] = a.y; p[2] = a.z; }

/* ---------------------------------------------------------------- primitives */

/* closest point on segment [a,b] to p */
static double pt_seg(v3 p, v3 a, v3 b, v3 *q) {
    v3 d = vsub(b, a);
    double dd = vdot(d, d), s = 0.0;
    if (dd > 0.0) {
        s = vdot(vsub(p, a), d) / dd;
        if (s < 0.0) s = 0.0;
        if (s > 1.0) s = 1.0;
    }
    *q = vadd(a, vscale(d, s));
    return vdist(p, *q);
}

/* is x (assumed in the plane of abc, normal n) inside the closed triangle? */
static int in_tri(v3 x, v3 a, v3 b, v3 c, v3 n) {
    double wa = vdot(vcross(vsub(b, x), vsub(c, x)), n);
    double wb = vdot(vcross(vsub(c, x), vsub(a, x)), n);
    double wc = vdot(vcross(vsub(a, x), vsub(b, x)), n);
    return wa >= 0.0 && wb >= 0.0 && wc >= 0.0;
}

/* closest point on triangle abc to p */
static double pt_tri(v3 p, v3 a, v3 b, v3 c, v3 *q) {
    v3 n = vcross(vsub(b, a), vsub(c, a));
    double nn = vdot(n, n);
    if (nn > 0.0) {
        double h = vdot(vsub(p, a), n) / nn;
        v3 x = vsub(p, vscale(n, h));
        if (in_tri(x, a, b, c, n)) {
            *q = x;
            return fabs(h) * sqrt(nn);
        }
    }
    v3 q1, q2, q3;
    double d1 = pt_seg(p, a, b, &q1), d2 = pt_seg(p, b, c, &q2), d3 = pt_seg(p, c, a, &q3);
    double best = d1;
    *q = q1;
    if (d2 < best) { best = d2; *q = q2; }
    if (d3 < best) { best = d3; *q = q3; }
    return best;
}

/* closest points between segments [p0,p1] and [q0,q1] */
static double seg_seg(v3 p0, v3 p1, v3 q0, v3 q1, v3 *cp, v3 *cq) {
    v3 t;
    double best = pt_seg(p0, q0, q1, &t);
    *cp = p0; *cq = t;
    double d = pt_seg(p1, q0, q1, &t);
    if (d < best) { best = d; *cp = p1; *cq = t; }
    d = pt_seg(q0, p0, p1, &t);
    if (d < best) { best = d; *cp = t; *cq = q0; }
    d = pt_seg(q1, p0, p1, &t);
    if (d < best) { best = d; *cp = t; *cq = q1; }
    /* The stationary point of |p0 + s d1 - q0 - u d2|^2 solves a 2x2 system
     * whose determinant and numerators, (d1.d1)(d2.d2) - (d1.d2)^2 and so on,
     * are written here through the Binet-Cauchy identity
     * (a x b).(c x d) = (a.c)(b.d) - (a.d)(b.c) as dot products of cross
     * products: the same values, but without the cancellation of the
     * difference of products, so nearly parallel segments keep an accurate
     * stationary point.  u is then taken as the exact minimiser over u for
     * that s, (d2.r + s d1.d2) / d2.d2, so that a rounding error in s moves
     * the pair along the nearly flat valley of the quadratic instead of
     * across it.  Any (s, u) in the square gives a pair of points on the two
     * segments, so taking it can never undercut the true minimum. */
    v3 d1 = vsub(p1, p0), d2 = vsub(q1, q0), r = vsub(p0, q0);
    v3 n = vcross(d1, d2);
    double det = vdot(n, n);
    if (det > 0.0) {
        double s = vdot(n, vcross(d2, r)) / det;
        double u = (vdot(d2, r) + s * vdot(d1, d2)) / vdot(d2, d2);
        if (s >= 0.0 && s <= 1.0 && u >= 0.0 && u <= 1.0) {
            v3 x = vadd(p0, vscale(d1, s)), y = vadd(q0, vscale(d2, u));
            double dd = vdist(x, y);
            if (dd < best) { best = dd; *cp = x; *cq = y; }
        }
    }
    return best;
}

/* does segment [p0,p1] cross triangle abc at a single point?  (coplanar: no) */
static int seg_tri_hit(v3 p0, v3 p1, v3 a, v3 b, v3 c, v3 *x) {
    v3 n = vcross(vsub(b, a), vsub(c, a));
    if (vdot(n, n) == 0.0) return 0;
    double s0 = vdot(n, vsub(p0, a)), s1 = vdot(n, vsub(p1, a));
    if ((s0 > 0.0 && s1 > 0.0) || (s0 < 0.0 && s1 < 0.0)) return 0;
    if (s0 == 0.0 && s1 == 0.0) return 0;
    double s = s0 / (s0 - s1);
    *x = vadd(p0, vscale(vsub(p1, p0), s));
    return in_tri(*x, a, b, c, n);
}

/* distance between closed triangles A = (a0,a1,a2), B = (b0,b1,b2) */
static double tri_tri(const v3 *A, const v3 *B, v3 *pa, v3 *pb) {
    v3 x;
    for (int i = 0; i < 3; ++i) {
        if (seg_tri_hit(A[i], A[(i + 1) % 3], B[0], B[1], B[2], &x)) { *pa = x; *pb = x; return 0.0; }
        if (seg_tri_hit(B[i], B[(i + 1) % 3], A[0], A[1], A[2], &x)) { *pa = x; *pb = x; return 0.0; }
    }
    double best = INFINITY;
    v3 cp, cq;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double d = seg_seg(A[i], A[(i + 1) % 3], B[j], B[(j + 1) % 3], &cp, &cq);
            if (d < best) { best = d; *pa = cp; *pb = cq; }
        }
    for (int i = 0; i < 3; ++i) {
        double d = pt_tri(A[i], B[0], B[1], B[2], &cq);
        if (d < best) { best = d; *pa = A[i]; *pb = cq; }
        d = pt_tri(B[i], A[0], A[1], A[2], &cp);
        if (d < best) { best = d; *pa = cp; *pb = B[i]; }
    }
    return best;
}

/* farthest vertex pair between two triangles */
static double tri_tri_max(const v3 *A, const v3 *B, v3 *pa, v3 *pb) {
    double best = -1.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double d = vdist(A[i], B[j]);
            if (d > best) { best = d; *pa = A[i]; *pb = B[j]; }
        }
    return best;
}

/* ---------------------------------------------------------- exported kernels */

OR_API double or_point_segment(const double *p, const double *a, const double *b, double *q) {
    v3 r;
    double d = pt_seg(ld(p), ld(a), ld(b), &r);
    st(q, r);
    return d;
}

OR_API double or_point_triangle(const double *p, const double *a, const double *b,
                                const double *c, double *q) {
    v3 r;
    double d = pt_tri(ld(p), ld(a), ld(b), ld(c), &r);
    st(q, r);
    return d;
}

OR_API double or_segment_segment(const double *p0, const double *p1, const double *q0,
                                 const double *q1, double *cp, double *cq) {
    v3 a, b;
    double d = seg_seg(ld(p0), ld(p1), ld(q0), ld(q1), &a, &b);
    st(cp, a);
    st(cq, b);
    return d;
}

/* A, B: 9 doubles each (three vertices) */
OR_API double or_tri_tri(const double *A, const double *B, double *pa, double *pb) {
    v3 a[3] = {ld(A), ld(A + 3), ld(A + 6)}, b[3] = {ld(B), ld(B + 3), ld(B + 6)}, x, y;
    double d = tri_tri(a, b, &x, &y);
    st(pa, x);
    st(pb, y);
    return d;
}

OR_API double or_tri_tri_max(const double *A, const double *B, double *pa, double *pb) {
    v3 a[3] = {ld(A), ld(A + 3), ld(A + 6)}, b[3] = {ld(B), ld(B + 3), ld(B + 6)}, x, y;
    double d = tri_tri_max(a, b, &x, &y);
    st(pa, x);
    st(pb, y);
    return d;
}

/* ------------------------------------------------------------------ meshes */

typedef struct {
    double d;
    int64_t ta, tb;
    double pa[3], pb[3];
} or_result;

static v3 xf(const double *X, double x, double y, double z) {
    return mk(X[0] * x + X[1] * y + X[2] * z + X[3],
              X[4] * x + X[5] * y + X[6] * z + X[7],
              X[8] * x + X[9] * y + X[10] * z + X[11]);
}

/* world-space triangle vertices, 3 v3 per triangle */
static v3 *world_tris(const float *v, const int32_t *t, int64_t nt, const double *X) {
    v3 *w = (v3 *)malloc(sizeof(v3) * 3 * (size_t)nt);
    if (!w) return NULL;
    for (int64_t i = 0; i < nt; ++i)
        for (int k = 0; k < 3; ++k) {
            const float *p = v + 3 * (int64_t)t[3 * i + k];
            w[3 * i + k] = xf(X, (double)p[0], (double)p[1], (double)p[2]);
        }
    return w;
}

/* "is (d, a, b) a better min-witness than (bd, ba, bb)?" */
static inline int better_min(double d, int64_t a, int64_t b, double bd, int64_t ba, int64_t bb) {
    if (d < bd) return 1;
    if (d > bd) return 0;
    return (a < ba) || (a == ba && b < bb);
}
static inline int better_max(double d, int64_t a, int64_t b, double bd, int64_t ba, int64_t bb) {
    if (d > bd) return 1;
    if (d < bd) return 0;
    return (a < ba) || (a == ba && b < bb);
}

typedef struct {
    const v3 *wa, *wb;
    int64_t na, nb, i0, i1;
    int kind;
    or_result r;
} brute_job;

static void *brute_worker(void *arg) {
    brute_job *J = (brute_job *)arg;
    or_result r;
    r.d = J->kind ? -1.0 : INFINITY;
    r.ta = r.tb = INT64_MAX;
    v3 pa, pb;
    for (int64_t i = J->i0; i < J->i1; ++i)
        for (int64_t j = 0; j < J->nb; ++j) {
            double d = J->kind ? tri_tri_max(J->wa + 3 * i, J->wb + 3 * j, &pa, &pb)
                               : tri_tri(J->wa + 3 * i, J->wb + 3 * j, &pa, &pb);
            int b = J->kind ? better_max(d, i, j, r.d, r.ta, r.tb) : better_min(d, i, j, r.d, r.ta, r.tb);
            if (b) { r.d = d; r.ta = i; r.tb = j; st(r.pa, pa); st(r.pb, pb); }
        }
    J->r = r;
    return NULL;
}

/* kind 0 = min, 1 = max.  Returns 0 on success. */
OR_API int or_brute(const float *va, int64_t nva, const int32_t *ta, int64_t nta, const double *xa,
                    const float *vb, int64_t nvb, const int32_t *tb, int64_t ntb, const double *xb,
                    int kind, int nthreads, or_result *out) {
    (void)nva; (void)nvb;
    if (nta <= 0 || ntb <= 0) return 1;
    v3 *wa = world_tris(va, ta, nta, xa), *wb = world_tris(vb, tb, ntb, xb);
    if (!wa || !wb) { free(wa); free(wb); return 2; }
    if (nthreads < 1) nthreads = 1;
    if (nthreads > nta) nthreads = (int)nta;
    brute_job *jobs = (brute_job *)calloc((size_t)nthreads, sizeof(brute_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int k = 0; k < nthreads; ++k) {
        jobs[k].wa = wa; jobs[k].wb = wb; jobs[k].na = nta; jobs[k].nb = ntb; jobs[k].kind = kind;
        jobs[k].i0 = nta * k / nthreads; jobs[k].i1 = nta * (k + 1) / nthreads;
        pthread_create(&th[k], NULL, brute_worker, &jobs[k]);
    }
    for (int k = 0; k < nthreads; ++k) pthread_join(th[k], NULL);
    or_result best = jobs[0].r;
    for (int k = 1; k < nthreads; ++k) {
        or_result *r = &jobs[k].r;
        int b = kind ? better_max(r->d, r->ta, r->tb, best.d, best.ta, best.tb)
                     : better_min(r->d, r->ta, r->tb, best.d, best.ta, best.tb);
        if (b) best = *r;
    }
    *out = best;
    free(jobs); free(th); free(wa); free(wb);
    return 0;
}

/* ----------------------------------------------------- point to mesh (N points)
 *
 * The distance from a point p to a mesh Q is Eq. 1 with P = {p}: the minimum
 * over the triangles of Q of the point-triangle distance.  Brute force over
 * all triangles, threaded over the points; among triangles at the same
 * float64 distance the smallest index is reported, with its closest point.
 */

typedef struct {
    const v3 *w;
    int64_t nt;
    const double *pts;
    int64_t i0, i1;
    double *d, *q;
    int64_t *tri;
} point_job;

static void *point_worker(void *arg) {
    point_job *J = (point_job *)arg;
    for (int64_t i = J->i0; i < J->i1; ++i) {
        const v3 p = ld(J->pts + 3 * i);
        double best = INFINITY;
        int64_t bt = -1;
        v3 bq = p, q;
        for (int64_t j = 0; j < J->nt; ++j) {
            const double d = pt_tri(p, J->w[3 * j], J->w[3 * j + 1], J->w[3 * j + 2], &q);
            if (d < best) { best = d; bt = j; bq = q; }
        }
        J->d[i] = best;
        J->tri[i] = bt;
        st(J->q + 3 * i, bq);
    }
    return NULL;
}

/* pts: n x 3 world points; out: d[n], tri[n], q[3n] (closest points, world). */
OR_API int or_point_mesh(const float *v, int64_t nv, const int32_t *t, int64_t nt, const double *X,
                         const double *pts, int64_t n, int nthreads, double *d, int64_t *tri, double *q) {
    (void)nv;
    if (nt <= 0 || n < 0) return 1;
    if (n == 0) return 0;
    v3 *w = world_tris(v, t, nt, X);
    if (!w) return 2;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > n) nthreads = (int)n;
    point_job *jobs = (point_job *)calloc((size_t)nthreads, sizeof(point_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int k = 0; k < nthreads; ++k) {
        point_job *J = &jobs[k];
        J->w = w; J->nt = nt; J->pts = pts; J->d = d; J->q = q; J->tri = tri;
        J->i0 = n * k / nthreads; J->i1 = n * (k + 1) / nthreads;
        pthread_create(&th[k], NULL, point_worker, J);
    }
    for (int k = 0; k < nthreads; ++k) pthread_join(th[k], NULL);
    free(jobs); free(th); free(w);
    return 0;
}

/* -------------------------------------------------------------- AABB tree */

typedef struct {
    double lo[3], hi[3];
    int32_t left, right; /* children, -1 for a leaf */
    int32_t start, count; /* leaf triangle range in `order` */
} onode;

typedef struct {
    int64_t nt;
    int32_t nnodes;
    onode *nodes;
    int32_t *order;  /* triangle ids in leaf order */
    double *tv;      /* local float64 vertices, 9 per original triangle */
} or_bvh;

#define OR_LEAF 4

static void tri_box(const double *p, double *lo, double *hi) {
    for (int k = 0; k < 3; ++k) {
        double a = p[k], b = p[3 + k], c = p[6 + k];
        lo[k] = fmin(a, fmin(b, c));
        hi[k] = fmax(a, fmax(b, c));
    }
}

/* quickselect: reorder idx[0..n) so that element m has the m-th smallest key */
static void select_kth(int32_t *idx, const double *key, int64_t n, int64_t m) {
    int64_t l = 0, r = n - 1;
    while (l < r) {
        double piv = key[idx[(l + r) / 2]];
        int64_t i = l, j = r;
        while (i <= j) {
            while (key[idx[i]] < piv) ++i;
            while (key[idx[j]] > piv) --j;
            if (i <= j) { int32_t t = idx[i]; idx[i] = idx[j]; idx[j] = t; ++i; --j; }
        }
        if (m <= j) r = j;
        else if (m >= i) l = i;
        else break;
    }
}

OR_API or_bvh *or_bvh_build(const float *v, int64_t nv, const int32_t *t, int64_t nt) {
    (void)nv;
    if (nt <= 0 || nt > INT32_MAX / 2) return NULL;
    or_bvh *B = (or_bvh *)calloc(1, sizeof(or_bvh));
    B->nt = nt;
    B->tv = (double *)malloc(sizeof(double) * 9 * (size_t)nt);
    B->order = (int32_t *)malloc(sizeof(int32_t) * (size_t)nt);
    int32_t cap = (int32_t)(2 * nt + 1);
    B->nodes = (onode *)malloc(sizeof(onode) * (size_t)cap);
    double *cen = (double *)malloc(sizeof(double) * 3 * (size_t)nt);
    double *key = (double *)malloc(sizeof(double) * (size_t)nt);
    double *tbox = (double *)malloc(sizeof(double) * 6 * (size_t)nt);
    for (int64_t i = 0; i < nt; ++i) {
        for (int k = 0; k < 3; ++k) {
            const float *p = v + 3 * (int64_t)t[3 * i + k];
            for (int c = 0; c < 3; ++c) B->tv[9 * i + 3 * k + c] = (double)p[c];
        }
        for (int c = 0; c < 3; ++c)
            cen[3 * i + c] = (B->tv[9 * i + c] + B->tv[9 * i + 3 + c] + B->tv[9 * i + 6 + c]) / 3.0;
        tri_box(B->tv + 9 * i, tbox + 6 * i, tbox + 6 * i + 3);
        B->order[i] = (int32_t)i;
    }
    /* explicit stack of (node, start, count) */
    int32_t *stk = (int32_t *)malloc(sizeof(int32_t) * 3 * 128);
    int sp = 0;
    B->nnodes = 1;
    stk[0] = 0; stk[1] = 0; stk[2] = (int32_t)nt; sp = 1;
    while (sp > 0) {
        --sp;
        int32_t ni = stk[3 * sp], s = stk[3 * sp + 1], c = stk[3 * sp + 2];
        onode *N = &B->nodes[ni];
        double clo[3] = {INFINITY, INFINITY, INFINITY}, chi[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int k = 0; k < 3; ++k) { N->lo[k] = INFINITY; N->hi[k] = -INFINITY; }
        for (int32_t i = s; i < s + c; ++i) {
            int32_t id = B->order[i];
            const double *lo = tbox + 6 * (int64_t)id, *hi = lo + 3;
            for (int k = 0; k < 3; ++k) {
                N->lo[k] = fmin(N->lo[k], lo[k]);
                N->hi[k] = fmax(N->hi[k], hi[k]);
                clo[k] = fmin(clo[k], cen[3 * (int64_t)id + k]);
                chi[k] = fmax(chi[k], cen[3 * (int64_t)id + k]);
            }
        }
        if (c <= OR_LEAF) {
            N->left = N->right = -1;
            N->start = s; N->count = c;
            continue;
        }
        int ax = 0;
        for (int k = 1; k < 3; ++k)
            if (chi[k] - clo[k] > chi[ax] - clo[ax]) ax = k;
        for (int32_t i = s; i < s + c; ++i) key[B->order[i]] = cen[3 * (int64_t)B->order[i] + ax];
        int32_t half = c / 2;
        select_kth(B->order + s, key, c, half);
        int32_t l = B->nnodes++, r = B->nnodes++;
        N->left = l; N->right = r; N->start = s; N->count = c;
        stk[3 * sp] = l; stk[3 * sp + 1] = s; stk[3 * sp + 2] = half; ++sp;
        stk[3 * sp] = r; stk[3 * sp + 1] = s + half; stk[3 * sp + 2] = c - half; ++sp;
    }
    free(stk); free(cen); free(key); free(tbox);
    return B;
}

OR_API void or_bvh_free(or_bvh *B) {
    if (!B) return;
    free(B->nodes); free(B->order); free(B->tv); free(B);
}

OR_API int32_t or_bvh_nodes(const or_bvh *B) { return B ? B->nnodes : 0; }

/* world-space enclosing box of a local box under X, widened by a float64
 * rounding allowance so that it always contains the exactly mapped box */
static void world_box(const double *X, const double *lo, const double *hi, double *wlo, double *whi) {
    for (int i = 0; i < 3; ++i) {
        double c = X[4 * i + 3], h = 0.0, mag = fabs(X[4 * i + 3]);
        for (int j = 0; j < 3; ++j) {
            double m = 0.5 * (lo[j] + hi[j]), e = 0.5 * (hi[j] - lo[j]);
            c += X[4 * i + j] * m;
            h += fabs(X[4 * i + j]) * e;
            mag += fabs(X[4 * i + j]) * (fabs(m) + e);
        }
        double slack = 1e-12 * (mag + 1e-300);
        wlo[i] = c - h - slack;
        whi[i] = c + h + slack;
    }
}

static double box_min_dist(const double *alo, const double *ahi, const double *blo, const double *bhi) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
        double g = 0.0;
        if (blo[k] > ahi[k]) g = blo[k] - ahi[k];
        else if (alo[k] > bhi[k]) g = alo[k] - bhi[k];
        s += g * g;
    }
    return sqrt(s);
}

static double box_max_dist(const double *alo, const double *ahi, const double *blo, const double *bhi) {
    double s = 0.0;
    for (int k = 0; k < 3; ++k) {
        double g = fmax(fabs(ahi[k] - blo[k]), fabs(bhi[k] - alo[k]));
        s += g * g;
    }
    return sqrt(s);
}

typedef struct { double key; int32_t a, b; } hent;
typedef struct { hent *h; int64_t n, cap; int maxheap; } heap;

static inline int hless(const heap *H, const hent *x, const hent *y) {
    return H->maxheap ? (x->key > y->key) : (x->key < y->key);
}
static int hpush(heap *H, hent e) {
    if (H->n == H->cap) {
        int64_t nc = H->cap ? 2 * H->cap : 1024;
        hent *nh = (hent *)realloc(H->h, sizeof(hent) * (size_t)nc);
        if (!nh) return 1;
        H->h = nh; H->cap = nc;
    }
    int64_t i = H->n++;
    H->h[i] = e;
    while (i > 0) {
        int64_t p = (i - 1) / 2;
        if (!hless(H, &H->h[i], &H->h[p])) break;
        hent t = H->h[i]; H->h[i] = H->h[p]; H->h[p] = t;
        i = p;
    }
    return 0;
}
static hent hpop(heap *H) {
    hent top = H->h[0];
    H->h[0] = H->h[--H->n];
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < H->n && hless(H, &H->h[l], &H->h[m])) m = l;
        if (r < H->n && hless(H, &H->h[r], &H->h[m])) m = r;
        if (m == i) break;
        hent t = H->h[i]; H->h[i] = H->h[m]; H->h[m] = t;
        i = m;
    }
    return top;
}

/* world-space box of node i, computed on first use and cached */
typedef struct { const or_bvh *B; const double *X; double *w; uint8_t *have; } wcache;

static const double *wbox(wcache *W, int32_t i) {
    if (!W->have[i]) {
        world_box(W->X, W->B->nodes[i].lo, W->B->nodes[i].hi, W->w + 6 * (int64_t)i, W->w + 6 * (int64_t)i + 3);
        W->have[i] = 1;
    }
    return W->w + 6 * (int64_t)i;
}

static int wcache_init(wcache *W, const or_bvh *B, const double *X) {
    W->B = B; W->X = X;
    W->w = (double *)malloc(sizeof(double) * 6 * (size_t)B->nnodes);
    W->have = (uint8_t *)calloc((size_t)B->nnodes, 1);
    return W->w && W->have;
}

static void wcache_free(wcache *W) { free(W->w); free(W->have); }

static void world_tri(const or_bvh *B, int32_t id, const double *X, v3 *o) {
    const double *p = B->tv + 9 * (int64_t)id;
    for (int k = 0; k < 3; ++k) o[k] = xf(X, p[3 * k], p[3 * k + 1], p[3 * k + 2]);
}

/* kind 0 = min, 1 = max; nodes_visited (optional) counts popped node pairs */
OR_API int or_bvh_query(const or_bvh *A, const double *xa, const or_bvh *B, const double *xb, int kind,
                        or_result *out, int64_t *nodes_visited) {
    if (!A || !B) return 1;
    wcache WA, WB;
    if (!wcache_init(&WA, A, xa) || !wcache_init(&WB, B, xb)) { wcache_free(&WA); wcache_free(&WB); return 2; }
    heap H = {0};
    H.maxheap = kind;
    or_result r;
    r.d = kind ? -1.0 : INFINITY;
    r.ta = r.tb = INT64_MAX;
    int64_t visited = 0;
    hent e0;
    e0.a = 0; e0.b = 0;
    {
        const double *a0 = wbox(&WA, 0), *b0 = wbox(&WB, 0);
        e0.key = kind ? box_max_dist(a0, a0 + 3, b0, b0 + 3) : box_min_dist(a0, a0 + 3, b0, b0 + 3);
    }
    hpush(&H, e0);
    while (H.n > 0) {
        hent e = hpop(&H);
        ++visited;
        if (kind ? (e.key < r.d) : (e.key > r.d)) break;
        const onode *na = &A->nodes[e.a], *nb = &B->nodes[e.b];
        int la = na->left < 0, lb = nb->left < 0;
        if (la && lb) {
            for (int32_t i = na->start; i < na->start + na->count; ++i) {
                v3 ta[3];
                int32_t ia = A->order[i];
                world_tri(A, ia, xa, ta);
                for (int32_t j = nb->start; j < nb->start + nb->count; ++j) {
                    v3 tb[3], pa, pb;
                    int32_t ib = B->order[j];
                    world_tri(B, ib, xb, tb);
                    double d = kind ? tri_tri_max(ta, tb, &pa, &pb) : tri_tri(ta, tb, &pa, &pb);
                    int b = kind ? better_max(d, ia, ib, r.d, r.ta, r.tb) : better_min(d, ia, ib, r.d, r.ta, r.tb);
                    if (b) { r.d = d; r.ta = ia; r.tb = ib; st(r.pa, pa); st(r.pb, pb); }
                }
            }
            continue;
        }
        /* split the side with the larger world box (or the only non-leaf side) */
        int split_a;
        if (la) split_a = 0;
        else if (lb) split_a = 1;
        else {
            double sa = 0, sb = 0;
            const double *pa_ = wbox(&WA, e.a), *pb_ = wbox(&WB, e.b);
            for (int k = 0; k < 3; ++k) {
                sa += (pa_[3 + k] - pa_[k]);
                sb += (pb_[3 + k] - pb_[k]);
            }
            split_a = sa >= sb;
        }
        int32_t ch[2];
        if (split_a) { ch[0] = na->left; ch[1] = na->right; } else { ch[0] = nb->left; ch[1] = nb->right; }
        for (int c = 0; c < 2; ++c) {
            hent f;
            f.a = split_a ? ch[c] : e.a;
            f.b = split_a ? e.b : ch[c];
            const double *al = wbox(&WA, f.a), *bl = wbox(&WB, f.b);
            f.key = kind ? box_max_dist(al, al + 3, bl, bl + 3) : box_min_dist(al, al + 3, bl, bl + 3);
            if (kind ? (f.key >= r.d) : (f.key <= r.d)) {
                if (hpush(&H, f)) { free(H.h); wcache_free(&WA); wcache_free(&WB); return 2; }
            }
        }
    }
    free(H.h); wcache_free(&WA); wcache_free(&WB);
    *out = r;
    if (nodes_visited) *nodes_visited = visited;
    return 0;
}

typedef struct {
    const or_bvh *A, *B;
    const double *xa, *xb;
    int kind;
    int64_t n;
    int64_t *next;
    pthread_mutex_t *mu;
    or_result *out;
    int rc;
} batch_job;

static void *batch_worker(void *arg) {
    batch_job *J = (batch_job *)arg;
    for (;;) {
        pthread_mutex_lock(J->mu);
        int64_t i = (*J->next)++;
        pthread_mutex_unlock(J->mu);
        if (i >= J->n) break;
        int rc = or_bvh_query(J->A, J->xa + 12 * i, J->B, J->xb + 12 * i, J->kind, &J->out[i], NULL);
        if (rc) J->rc = rc;
    }
    return NULL;
}

/* n independent queries of the same mesh pair, spread over nthreads threads */
OR_API int or_bvh_query_batch(const or_bvh *A, const double *xa, const or_bvh *B, const double *xb,
                              int64_t n, int kind, int nthreads, or_result *out) {
    if (nthreads < 1) nthreads = 1;
    int64_t next = 0;
    pthread_mutex_t mu;
    pthread_mutex_init(&mu, NULL);
    batch_job *jobs = (batch_job *)calloc((size_t)nthreads, sizeof(batch_job));
    pthread_t *th = (pthread_t *)calloc((size_t)nthreads, sizeof(pthread_t));
    for (int k = 0; k < nthreads; ++k) {
        jobs[k].A = A; jobs[k].B = B; jobs[k].xa = xa; jobs[k].xb = xb; jobs[k].kind = kind;
        jobs[k].n = n; jobs[k].next = &next; jobs[k].mu = &mu; jobs[k].out = out;
        pthread_create(&th[k], NULL, batch_worker, &jobs[k]);
    }
    int rc = 0;
    for (int k = 0; k < nthreads; ++k) {
        pthread_join(th[k], NULL);
        if (jobs[k].rc) rc = jobs[k].rc;
    }
    pthread_mutex_destroy(&mu);
    free(jobs); free(th);
    return rc;
}

/* distance of one triangle pair given float32 local vertices (9 floats each)
 * and the two world transforms, mapped exactly as the mesh queries map them */
OR_API double or_tri_pair_world(const float *A9, const double *xa, const float *B9, const double *xb,
                                int kind, double *pa, double *pb) {
    v3 a[3], b[3], x, y;
    for (int k = 0; k < 3; ++k) {
        a[k] = xf(xa, (double)A9[3 * k], (double)A9[3 * k + 1], (double)A9[3 * k + 2]);
        b[k] = xf(xb, (double)B9[3 * k], (double)B9[3 * k + 1], (double)B9[3 * k + 2]);
    }
    double d = kind ? tri_tri_max(a, b, &x, &y) : tri_tri(a, b, &x, &y);
    st(pa, x);
    st(pb, y);
    return d;
}
