"""Pins for the FP64 oracle against facts that do not come from the oracle.

Each test fixes the oracle to a closed form, an invariant of Eqs. 1-2
(Section 3), a brute-force sampling bound, or an independent numpy
computation, so that a dropped term, a wrong sign, an index slip or a
transposed operand in the oracle fails somewhere here.
"""

import json
import math
import os

import numpy as np
import pytest

from paper_2411_11244_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# ----------------------------------------------------------- primitives


def test_point_segment_closed_forms(oracle_mod):
    o = oracle_mod
    d, q = o.point_segment((0, 1, 0), (-1, 0, 0), (1, 0, 0))
    assert d == pytest.approx(1.0, abs=1e-15) and np.allclose(q, 0)
    d, q = o.point_segment((3, 4, 0), (-1, 0, 0), (0, 0, 0))  # endpoint region
    assert d == pytest.approx(5.0, abs=1e-15) and np.allclose(q, 0)
    d, q = o.point_segment((2, 2, 2), (1, 1, 1), (1, 1, 1))  # degenerate segment
    assert d == pytest.approx(math.sqrt(3), abs=1e-15)


def test_point_triangle_regions(oracle_mod):
    o = oracle_mod
    a, b, c = (0, 0, 0), (1, 0, 0), (0, 1, 0)
    d, q = o.point_triangle((0.2, 0.3, 2.5), a, b, c)  # face interior: plane distance
    assert d == pytest.approx(2.5, abs=1e-15) and np.allclose(q, (0.2, 0.3, 0))
    d, q = o.point_triangle((0.2, 0.3, -1.5), a, b, c)  # below the face
    assert d == pytest.approx(1.5, abs=1e-15)
    d, q = o.point_triangle((-3, -4, 0), a, b, c)  # vertex region
    assert d == pytest.approx(5.0, abs=1e-15) and np.allclose(q, a)
    d, q = o.point_triangle((0.5, -2, 0), a, b, c)  # edge region (ab)
    assert d == pytest.approx(2.0, abs=1e-15) and np.allclose(q, (0.5, 0, 0))
    d, q = o.point_triangle((1, 1, 1), a, b, c)  # edge region (bc), out of plane
    assert d == pytest.approx(math.sqrt(1.5), abs=1e-15) and np.allclose(q, (0.5, 0.5, 0))
    d, q = o.point_triangle((1, 1, 0), (0, 0, 0), (1, 0, 0), (2, 0, 0))  # collinear triangle
    assert d == pytest.approx(1.0, abs=1e-15)


def test_point_triangle_general_plane_distance(oracle_mod):
    """A point above the interior of a tilted triangle: |n^ . (p - a)|."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        a, b, c = rng.normal(size=(3, 3))
        n = np.cross(b - a, c - a)
        n /= np.linalg.norm(n)
        w = rng.dirichlet((2, 2, 2))
        inside = w[0] * a + w[1] * b + w[2] * c
        h = rng.uniform(-2, 2)
        d, q = oracle_mod.point_triangle(inside + h * n, a, b, c)
        assert d == pytest.approx(abs(h), rel=1e-12, abs=1e-14)
        assert np.allclose(q, inside, atol=1e-12)


def test_segment_segment_closed_forms(oracle_mod):
    o = oracle_mod
    h = 0.37
    d, cp, cq = o.segment_segment((-1, 0, 0), (1, 0, 0), (0, -1, h), (0, 1, h))  # perpendicular skew
    assert d == pytest.approx(h, abs=1e-15)
    assert np.allclose(cp, (0, 0, 0)) and np.allclose(cq, (0, 0, h))
    th = 0.3
    d, _, _ = o.segment_segment((-1, 0, 0), (1, 0, 0), (-math.cos(th), -math.sin(th), h),
                                (math.cos(th), math.sin(th), h))  # oblique skew, interior
    assert d == pytest.approx(h, abs=1e-14)
    g = 0.25
    d, _, _ = o.segment_segment((0, 0, 0), (2, 0, 0), (1, g, 0), (3, g, 0))  # parallel overlap
    assert d == pytest.approx(g, abs=1e-15)
    d, _, _ = o.segment_segment((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0))  # crossing
    assert d == pytest.approx(0.0, abs=1e-15)
    d, _, _ = o.segment_segment((0, 0, 0), (1, 0, 0), (3, 0, 0), (4, 0, 0))  # collinear apart
    assert d == pytest.approx(2.0, abs=1e-15)
    d, _, _ = o.segment_segment((0, 0, 0), (0, 0, 0), (1, -1, 1), (1, 1, 1))  # point vs segment
    assert d == pytest.approx(math.sqrt(2), abs=1e-15)


def test_segment_segment_nearly_parallel(oracle_mod):
    """Two segments at a tiny angle eps whose projections cross at their
    midpoints, h apart: the distance is h, attained at the midpoints (the
    interior stationary point).  With eps^2 below the float64 resolution of
    |d1|^2 |d2|^2 the difference-of-products determinant vanishes; a stationary
    point lost that way leaves only endpoint pairs, at sqrt(h^2 + eps^2) (for
    eps = 2^-26, h = 2^-10: 1.2e-10 relative too high)."""
    h = 2.0 ** -10
    for k in (20, 26, 40):
        eps = 2.0 ** -k
        d, cp, cq = oracle_mod.segment_segment((-1, 0, 0), (1, 0, 0), (-1, -eps, h), (1, eps, h))
        assert d == h, (k, d)
        if k <= 26:  # (for eps = 2^-40 the endpoint pairs are at h in float64 too)
            assert np.array_equal(cp, [0, 0, 0]) and np.array_equal(cq, [0, 0, h])
    # the same under rigid motions: within the rounding of the moved inputs
    rng = np.random.default_rng(5)
    for _ in range(50):
        R, t = synth.random_rotation(rng), rng.normal(size=3)
        eps = 2.0 ** -int(rng.integers(12, 44))
        P = [R @ np.asarray(x, dtype=np.float64) + t for x in ((-1, 0, 0), (1, 0, 0), (-1, -eps, h), (1, eps, h))]
        d, _, _ = oracle_mod.segment_segment(*P)
        assert abs(d - h) <= 4e-15, (eps, d - h)


def test_segment_segment_matches_line_distance(oracle_mod):
    """Interior closest points: distance equals |(q0 - p0) . (d1 x d2)| / |d1 x d2|."""
    rng = np.random.default_rng(11)
    hits = 0
    for _ in range(200):
        p0, d1, q0, d2 = rng.normal(size=(4, 3))
        p1, q1 = p0 + d1, q0 + d2
        d, cp, cq = oracle_mod.segment_segment(p0, p1, q0, q1)
        # closest points of the infinite lines
        A = np.array([[d1 @ d1, -(d1 @ d2)], [d1 @ d2, -(d2 @ d2)]])
        s, t = np.linalg.solve(A, [-(d1 @ (p0 - q0)), -(d2 @ (p0 - q0))])
        if 0 < s < 1 and 0 < t < 1:
            n = np.cross(d1, d2)
            ref = abs((q0 - p0) @ n) / np.linalg.norm(n)
            assert d == pytest.approx(ref, rel=1e-10, abs=1e-12)
            hits += 1
        else:
            assert d >= abs((q0 - p0) @ np.cross(d1, d2)) / np.linalg.norm(np.cross(d1, d2)) - 1e-12
    assert hits > 10


def test_tri_tri_constructed_cases(oracle_mod):
    o = oracle_mod
    A = np.array([(0, 0, 0), (1, 0, 0), (0, 1, 0)], float)
    g = 0.125
    assert o.tri_tri(A, A + (0, 0, g))[0] == pytest.approx(g, abs=1e-15)  # stacked faces
    # edge-edge: A's top edge along x at z = 0, B's bottom edge along y at z = h
    Ae = np.array([(-1, 0, 0), (1, 0, 0), (0, 0, -1)], float)
    Be = np.array([(0, -1, 0.3), (0, 1, 0.3), (0, 0, 1.3)], float)
    d, pa, pb = o.tri_tri(Ae, Be)
    assert d == pytest.approx(0.3, abs=1e-15) and np.allclose(pa, 0) and np.allclose(pb, (0, 0, 0.3))
    # vertex-face: B's lowest vertex above A's interior
    Bv = np.array([(0.2, 0.2, 0.4), (0.5, 0.5, 2.0), (-0.5, 0.6, 1.5)], float)
    d, pa, pb = o.tri_tri(A, Bv)
    assert d == pytest.approx(0.4, abs=1e-15) and np.allclose(pa, (0.2, 0.2, 0))
    # piercing: a vertical triangle through A's interior
    Bp = np.array([(0.25, 0.25, -1), (0.25, 0.25, 1), (0.3, 0.35, 0.5)], float)
    assert o.tri_tri(A, Bp)[0] == 0.0
    # sharing a vertex
    Bs = np.array([(0, 0, 0), (-1, 0, 0), (0, 0, 1)], float)
    assert o.tri_tri(A, Bs)[0] == 0.0
    # coplanar overlap
    Bc = np.array([(0.2, 0.2, 0), (2, 0.2, 0), (0.2, 2, 0)], float)
    assert o.tri_tri(A, Bc)[0] <= 1e-15
    # coplanar, apart: vertex (1,0,0) to vertex (2,0,0)
    Bd = A + (2, 0, 0) - (1, 0, 0) + (1, 0, 0)
    assert o.tri_tri(A, Bd)[0] == pytest.approx(1.0, abs=1e-15)
    # symmetric in its arguments
    assert o.tri_tri(Bv, A)[0] == pytest.approx(0.4, abs=1e-15)


def _bary_samples(T, n):
    pts = []
    for i in range(n + 1):
        for j in range(n + 1 - i):
            pts.append(T[0] + (i / n) * (T[1] - T[0]) + (j / n) * (T[2] - T[0]))
    return np.array(pts)


def test_tri_tri_against_dense_sampling(oracle_mod):
    """Sampled distances are never below the exact minimum and approach it
    within the sampling resolution; sampled farthest distance equals the max."""
    rng = np.random.default_rng(7)
    n = 24
    for k in range(120):
        A = rng.uniform(-1, 1, (3, 3))
        B = rng.uniform(-1, 1, (3, 3)) + rng.normal(scale=0.8, size=3) * (k % 3)
        d, pa, pb = oracle_mod.tri_tri(A, B)
        SA, SB = _bary_samples(A, n), _bary_samples(B, n)
        D = np.linalg.norm(SA[:, None] - SB[None], axis=-1)
        emax = max(np.linalg.norm(A[i] - A[(i + 1) % 3]) for i in range(3))
        emax += max(np.linalg.norm(B[i] - B[(i + 1) % 3]) for i in range(3))
        assert D.min() >= d - 1e-12
        assert D.min() <= d + emax / n + 1e-12
        assert abs(np.linalg.norm(pa - pb) - d) <= 1e-12
        # witness points lie on their triangles
        assert oracle_mod.point_triangle(pa, *A)[0] <= 1e-12
        assert oracle_mod.point_triangle(pb, *B)[0] <= 1e-12
        dm, _, _ = oracle_mod.tri_tri_max(A, B)
        assert dm == pytest.approx(D.max(), rel=1e-14)


# ------------------------------------------------------------ meshes


def _rigid(rng):
    return synth.xform(synth.random_rotation(rng), rng.normal(size=3))


def test_two_boxes_closed_form(oracle_mod):
    g = 0.0625
    A = synth.box((0, 0, 0), (1, 1, 1))
    B = synth.box((1 + g, 0.25, 0.5), (2 + g, 0.75, 1.5))
    dmax = math.sqrt((2 + g) ** 2 + 0.75 ** 2 + 1.5 ** 2)
    rng = np.random.default_rng(3)
    for k in range(4):
        X = synth.identity_xform() if k == 0 else _rigid(rng)  # same motion for both
        for f in (oracle_mod.brute, ):
            r = f(A, X, B, X)
            assert r.d == pytest.approx(g, abs=1e-12)
            rm = f(A, X, B, X, "max")
            assert rm.d == pytest.approx(dmax, rel=1e-13)
        bA, bB = oracle_mod.Bvh(A), oracle_mod.Bvh(B)
        assert oracle_mod.bvh_query(bA, X, bB, X).d == pytest.approx(g, abs=1e-12)
        assert oracle_mod.bvh_query(bA, X, bB, X, "max").d == pytest.approx(dmax, rel=1e-13)


def test_parallel_grids_closed_form(oracle_mod):
    g = 0.01
    A = synth.grid(8, 1.0, 0.0)
    B = synth.grid(8, 1.0, g, x0=0.3, y0=0.25)
    r = oracle_mod.brute(A, synth.identity_xform(), B, synth.identity_xform())
    assert r.d == pytest.approx(g, abs=1e-9)
    # massive ties: the witness is the smallest (ta, tb) at distance g
    rm = oracle_mod.brute(A, synth.identity_xform(), B, synth.identity_xform(), "max")
    assert rm.d == pytest.approx(math.sqrt(1.3 ** 2 + 1.25 ** 2 + g * g), rel=1e-7)


def _tie_meshes(kind):
    """Meshes whose extreme pairs tie exactly by construction.  Min: triangle
    a (index 5 of A) lies in z = 0 and b (index 2 of B) right above its
    interior in z = 1/2, so they are 1/2 apart; a copy of both shifted by 8
    along x sits at indices 3 (A) and 6 (B); a duplicate of b at index 4 of B.
    Max: a (5) around (-2, 0, 0) and b (2) around (6, 0, 0), 8 apart at their
    outer vertices, and their mirror images through the origin at 3 (A) and
    6 (B).  The other triangles are fillers that stay clear of the extreme.
    Every coordinate is a small dyadic rational and the transforms are the
    identity, so the tied pairs repeat the same float64 operations on the
    same differences and their distances are bit for bit equal.  Returns
    (A, B, d_extreme, tied pairs)."""
    def mesh(tris):
        v = np.asarray([p for t in tris for p in t], dtype=np.float32)
        return v, np.arange(len(v), dtype=np.int32).reshape(-1, 3)

    def tri(o, pts):
        return [tuple(np.add(o, p)) for p in pts]

    if kind == "min":
        ta = [(0, 0, 0), (1, 0, 0), (0, 1, 0)]
        tb = [(0.25, 0.25, 0.5), (0.5, 0.25, 0.5), (0.25, 0.5, 0.5)]
        fa = lambda i: tri((4 * i, 20, -8), ta)  # far below and aside
        fb = lambda i: tri((4 * i, -20, 8), tb)
        A = [fa(0), fa(1), fa(2), tri((8, 0, 0), ta), fa(4), tri((0, 0, 0), ta), fa(6)]
        B = [fb(0), fb(1), tri((0, 0, 0), tb), fb(3), tri((0, 0, 0), tb), fb(5), tri((8, 0, 0), tb)]
        return mesh(A), mesh(B), 0.5, {(5, 2), (5, 4), (3, 6)}
    ta = [(-2, 0, 0), (-1.5, 0.5, 0), (-1.5, -0.5, 0)]
    tb = [(6, 0, 0), (5.5, 0.5, 0), (5.5, -0.5, 0)]
    neg = lambda t: [tuple(-np.asarray(p)) for p in t]
    fa = lambda i: tri((0, 0, 0.25 * i), [(0, 0, 0), (0.25, 0, 0), (0, 0.25, 0)])
    fb = lambda i: tri((0.5, 0, 0.25 * i), [(0, 0, 0), (0.25, 0, 0), (0, 0.25, 0)])
    A = [fa(0), fa(1), fa(2), neg(ta), fa(4), ta, fa(6)]
    B = [fb(0), fb(1), tb, fb(3), fb(4), fb(5), neg(tb)]
    return mesh(A), mesh(B), 8.0, {(5, 2), (3, 6)}


@pytest.mark.parametrize("kind", ["min", "max"])
def test_witness_tie_break_is_smallest_pair(oracle_mod, kind):
    """Among pairs at the same float64 extreme the witness is the smallest
    (tri_a, tri_b).  The tied set is not a product of index sets: (3, 6) is
    smallest by tri_a first, (5, 2) by tri_b first or by the largest pair, so
    a reversed or transposed comparison fails here."""
    A, B, dx, tied = _tie_meshes(kind)
    I = synth.identity_xform()
    # the construction's ties are exact in the oracle's arithmetic
    for ta, tb in tied:
        assert oracle_mod.witness_distance(A, I, B, I, ta, tb, kind)[0] == dx
    want = min(tied)
    assert want == (3, 6)
    r = oracle_mod.brute(A, I, B, I, kind)
    assert r.d == dx and (r.ta, r.tb) == want, (r.d, r.ta, r.tb)
    for threads in (1, 2, 3):
        r = oracle_mod.brute(A, I, B, I, kind, threads=threads)
        assert (r.ta, r.tb) == want
    bA, bB = oracle_mod.Bvh(A), oracle_mod.Bvh(B)
    r = oracle_mod.bvh_query(bA, I, bB, I, kind)
    assert r.d == dx and (r.ta, r.tb) == want, (r.d, r.ta, r.tb)


def test_bvh_batch_equals_single_queries(oracle_mod):
    """The threaded batch wrapper returns, query by query, what the single
    BVH query and brute force return (value and witness), with one A
    transform for all queries and with one per query, on more queries than
    threads and on fewer."""
    rng = np.random.default_rng(77)
    A = synth.torus(1.0, 0.25, 14, 9)
    B = synth.geosphere(3, 0.7, 0.01, 3)
    bA, bB = oracle_mod.Bvh(A), oracle_mod.Bvh(B)
    n = 7
    xas = [_rigid(rng) for _ in range(n)]
    xbs = [synth.compose(synth.xform(np.eye(3), rng.normal(size=3) * 1.5), x) for x in xas]
    for kind in ("min", "max"):
        for threads in (1, 3, 16):
            per = oracle_mod.bvh_query_batch(bA, xas, bB, xbs, kind, threads=threads)
            one = oracle_mod.bvh_query_batch(bA, xas[0], bB, xbs, kind, threads=threads)
            assert len(per) == n and len(one) == n
            for i in range(n):
                s = oracle_mod.bvh_query(bA, xas[i], bB, xbs[i], kind)
                b = oracle_mod.brute(A, xas[i], B, xbs[i], kind)
                assert (per[i].d, per[i].ta, per[i].tb) == (s.d, s.ta, s.tb) == (b.d, b.ta, b.tb)
                s0 = oracle_mod.bvh_query(bA, xas[0], bB, xbs[i], kind)
                assert (one[i].d, one[i].ta, one[i].tb) == (s0.d, s0.ta, s0.tb)


def test_geospheres_within_tessellation_bounds(oracle_mod):
    r1, r2, s = 1.0, 0.5, 2.0
    A = synth.geosphere(4, r1)
    B = synth.geosphere(3, r2)
    xb = synth.xform(np.eye(3), (s, 0, 0))
    r = oracle_mod.brute(A, synth.identity_xform(), B, xb)

    def inrad(m, rad):
        v = m[0].astype(np.float64)
        T = v[m[1]]
        n = np.cross(T[:, 1] - T[:, 0], T[:, 2] - T[:, 0])
        n /= np.linalg.norm(n, axis=1, keepdims=True)
        return float(np.min(np.abs(np.sum(n * T[:, 0], axis=1)))) / rad

    rho1, rho2 = inrad(A, r1), inrad(B, r2)
    vmax1 = float(np.max(np.linalg.norm(A[0].astype(np.float64), axis=1)))
    vmax2 = float(np.max(np.linalg.norm(B[0].astype(np.float64), axis=1)))
    assert s - vmax1 - vmax2 - 1e-12 <= r.d <= s - r1 * rho1 - r2 * rho2 + 1e-12
    rm = oracle_mod.brute(A, synth.identity_xform(), B, xb, "max")
    assert rm.d <= s + vmax1 + vmax2 + 1e-12
    assert rm.d >= s + 0.95 * (r1 + r2)


def _vertex_max(A, xa, B, xb, oracle_mod):
    wa = oracle_mod.world_vertices(A, xa)[np.unique(A[1])]
    wb = oracle_mod.world_vertices(B, xb)[np.unique(B[1])]
    return float(np.max(np.linalg.norm(wa[:, None] - wb[None], axis=-1)))


def test_invariants_symmetry_rigid_zero_and_vertex_max(oracle_mod):
    rng = np.random.default_rng(21)
    A = synth.torus(1.0, 0.3, 12, 10)
    B = synth.geosphere(3, 0.6, 0.01, 4)
    for k in range(6):
        xa, xb = _rigid(rng), _rigid(rng)
        xb = synth.compose(synth.xform(np.eye(3), (1.5 + 0.3 * k, 0, 0)), xb)
        r = oracle_mod.brute(A, xa, B, xb)
        rs = oracle_mod.brute(B, xb, A, xa)
        assert rs.d == pytest.approx(r.d, rel=1e-12, abs=1e-14)  # symmetry
        M = _rigid(rng)
        rr = oracle_mod.brute(A, synth.compose(M, xa), B, synth.compose(M, xb))
        assert rr.d == pytest.approx(r.d, rel=1e-9, abs=1e-12)  # rigid invariance
        rm = oracle_mod.brute(A, xa, B, xb, "max")
        assert rm.d == pytest.approx(_vertex_max(A, xa, B, xb, oracle_mod), rel=1e-14)
        assert oracle_mod.brute(B, xb, A, xa, "max").d == pytest.approx(rm.d, rel=1e-14)
    # intersecting meshes: a sphere through the torus tube
    xb = synth.xform(np.eye(3), (1.0, 0, 0))
    assert oracle_mod.brute(A, synth.identity_xform(), B, xb).d == 0.0


def _soup(rng, n, spread):
    v = rng.uniform(-spread, spread, (3 * n, 3)).astype(np.float32)
    t = np.arange(3 * n, dtype=np.int32).reshape(n, 3)
    return v, t


@pytest.mark.parametrize("seed", range(6))
def test_bvh_oracle_equals_brute_force(oracle_mod, seed):
    rng = np.random.default_rng(100 + seed)
    kinds = [
        lambda: synth.torus(1.0, 0.25, 10 + seed, 8),
        lambda: synth.geosphere(3 + seed % 3, 0.8, 0.02, seed),
        lambda: _soup(rng, 150 + 30 * seed, 1.0),
        lambda: synth.gear(64, 2, teeth=8, seed=seed),
    ]
    A = kinds[seed % 4]()
    B = kinds[(seed + 1) % 4]()
    bA, bB = oracle_mod.Bvh(A), oracle_mod.Bvh(B)
    for k in range(3):
        xa = _rigid(rng)
        xb = synth.compose(synth.xform(np.eye(3), rng.normal(size=3) * (0.5 + k)), xa)
        xb = synth.compose(xb, synth.xform(synth.random_rotation(rng), (0, 0, 0)))
        for kind in ("min", "max"):
            r1 = oracle_mod.brute(A, xa, B, xb, kind)
            r2 = oracle_mod.bvh_query(bA, xa, bB, xb, kind)
            assert r2.d == r1.d
            assert (r2.ta, r2.tb) == (r1.ta, r1.tb)


def test_config1_seed_fixture(oracle_mod):
    """The stored two-tori seed is the first seed whose draw does not intersect."""
    with open(os.path.join(GOLDEN, "tori_seed.json")) as f:
        fx = json.load(f)
    A, B, xa, xb = synth.config_tori(fx["seed"])
    r = oracle_mod.brute(A, xa, B, xb)
    assert r.d > 0.0
    assert r.d == pytest.approx(fx["d_min"], rel=1e-12)
    for s in range(fx["seed"]):
        A, B, xa, xb = synth.config_tori(s)
        assert oracle_mod.brute(A, xa, B, xb).d == 0.0


# ----------------------------------------------------------- point to mesh

def test_point_mesh_box_closed_forms(oracle_mod):
    """Distance from points to the surface of the unit cube (12 triangles):
    face, edge and corner regions outside, and the nearest face from inside;
    the same under a rigid motion of cube and points together."""
    cube = synth.box((0, 0, 0), (1, 1, 1))
    pts = np.array([
        [2.0, 0.5, 0.5],      # face region: 1
        [0.25, -0.75, 0.5],   # face region: 0.75
        [1.5, 1.25, 0.5],     # edge region: sqrt(0.5^2 + 0.25^2)
        [-1.0, -2.0, 3.0],    # corner region: sqrt(1 + 4 + 4)
        [0.5, 0.5, 0.3],      # inside, nearest face z = 0: 0.3
        [0.9, 0.4, 0.5],      # inside, nearest face x = 1: 0.1
        [1.0, 0.5, 0.5],      # on the surface: 0
    ])
    want = [1.0, 0.75, math.hypot(0.5, 0.25), 3.0, 0.3, 0.1, 0.0]
    I = synth.identity_xform()
    d, tri, q = oracle_mod.point_mesh(cube, I, pts)
    assert np.allclose(d, want, rtol=0, atol=1e-15)
    assert np.allclose(np.linalg.norm(pts - q, axis=1), want, atol=1e-15)
    # every closest point lies on the cube's surface
    inside = np.all((q >= -1e-15) & (q <= 1 + 1e-15), axis=1)
    on_face = np.any(np.isclose(q, 0, atol=1e-15) | np.isclose(q, 1, atol=1e-15), axis=1)
    assert inside.all() and on_face.all()
    assert ((tri >= 0) & (tri < 12)).all()
    # rigid invariance
    rng = np.random.default_rng(3)
    X = synth.xform(synth.random_rotation(rng), rng.normal(size=3))
    Xm = np.asarray(X).reshape(3, 4)
    d2, tri2, _ = oracle_mod.point_mesh(cube, X, pts @ Xm[:, :3].T + Xm[:, 3])
    assert np.allclose(d2, want, atol=1e-14)


def test_point_mesh_sphere_bounds(oracle_mod):
    """A point at distance s from the centre of a geodesic sphere of radius r
    (vertices on the sphere): s - r <= d <= s - r cos(theta) outside, where
    theta bounds the angle from a face's centre to its vertices."""
    f = 6
    S = synth.geosphere(f, 1.0)
    v, t = S
    w = np.asarray(v, dtype=np.float64)[np.asarray(t)]
    cen = w.mean(1)
    cos_t = min(float(np.min(np.sum(w[:, k] * cen, 1) / (np.linalg.norm(w[:, k], axis=1) * np.linalg.norm(cen, axis=1))))
                for k in range(3))
    r = float(np.linalg.norm(np.asarray(v, dtype=np.float64), axis=1).max())
    rng = np.random.default_rng(8)
    dirs = rng.normal(size=(20, 3))
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    s = rng.uniform(1.2, 3.0, 20)
    d, _, _ = oracle_mod.point_mesh(S, synth.identity_xform(), dirs * s[:, None])
    assert np.all(d >= s - r - 1e-12)
    assert np.all(d <= s - r * cos_t + 1e-12)
