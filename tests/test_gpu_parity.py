"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance (Section 3 problem, float32 traversal + float64 refinement):
  |d - d_ref| <= 1e-6 x diag, diag = world bounding-box diagonal of both meshes;
  the oracle's float64 distance of the returned witness pair equals d_ref
  within 1e-12 relative (+1e-15 x diag absolute for rounding at d ~ 0);
  the returned d equals that witness distance to the same tolerance.
Integer work (the BVH build's triangle order) is compared bit for bit.
"""

import math

import numpy as np
import pytest

from paper_2411_11244_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def G():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2411_11244_gb300 import gdist
    return gdist


@pytest.fixture(scope="module")
def ctx(G):
    c = G.gd_ctx_create(0)
    yield c
    G.gd_ctx_destroy(c)


def _mesh(G, ctx, m):
    h = G.gd_mesh_create(ctx, *m)
    G.gd_bvh_build(h, ctx=ctx)
    return h


def check(r, A, xa, B, xb, kind, ref, diag, oracle):
    assert r.status == 0, r.status
    assert abs(r.d - ref.d) <= 1e-6 * diag, (kind, r.d, ref.d)
    dw, _, _ = oracle.witness_distance(A, xa, B, xb, r.tri_a, r.tri_b, kind)
    tol = 1e-12 * abs(ref.d) + 1e-15 * diag
    assert abs(dw - ref.d) <= tol, (kind, dw, ref.d, (r.tri_a, r.tri_b), (ref.ta, ref.tb))
    assert abs(r.d - dw) <= tol, (kind, r.d, dw)
    pa, pb = np.array(r.pa[:]), np.array(r.pb[:])
    assert abs(np.linalg.norm(pa - pb) - r.d) <= 1e-12 * max(r.d, 1.0) + 1e-15 * diag
    wa = oracle.world_vertices(A, xa)[np.asarray(A[1])[r.tri_a]]
    wb = oracle.world_vertices(B, xb)[np.asarray(B[1])[r.tri_b]]
    assert oracle.point_triangle(pa, *wa)[0] <= 1e-12 * diag
    assert oracle.point_triangle(pb, *wb)[0] <= 1e-12 * diag
    assert (r.flags & 1) == (1 if r.d == 0.0 else 0)


def same_answer(r1, r2, oracle, A, xa, B, xb, kind):
    """Two answers to one query agree: equal value; for d > 0 the same witness
    (the smallest original (tri_a, tri_b) at the extreme is unique); for a min
    of 0 each witness is a pair the oracle finds intersecting (the traversal
    stops at the first such pair it proves, so the pair may differ)."""
    assert r1.status == 0 and r2.status == 0, (r1.status, r2.status)
    assert r1.d == r2.d, (r1.d, r2.d)
    if r1.d != 0.0 or kind != "min":
        assert (r1.tri_a, r1.tri_b) == (r2.tri_a, r2.tri_b)
        return
    for r in (r1, r2):
        dw, _, _ = oracle.witness_distance(A, xa, B, xb, r.tri_a, r.tri_b, "min")
        assert dw == 0.0, (r.tri_a, r.tri_b, dw)


def run_pair(G, ctx, oracle, A, B, xforms, kinds=("min", "max"), bvh_oracle=False):
    ma, mb = _mesh(G, ctx, A), _mesh(G, ctx, B)
    oa = ob = None
    if bvh_oracle:
        oa = oracle.Bvh(A)
        ob = oa if B is A else oracle.Bvh(B)
    try:
        for xa, xb in xforms:
            diag = oracle.diag(A, xa, B, xb)
            for kind in kinds:
                fn = G.gd_min_distance if kind == "min" else G.gd_max_distance
                r = fn(ctx, ma, mb, xa, xb)
                ref = oracle.bvh_query(oa, xa, ob, xb, kind) if bvh_oracle else oracle.brute(A, xa, B, xb, kind)
                check(r, A, xa, B, xb, kind, ref, diag, oracle)
    finally:
        G.gd_mesh_destroy(ma)
        G.gd_mesh_destroy(mb)


def _rigid(rng, scale=1.0):
    return synth.xform(synth.random_rotation(rng), rng.normal(size=3) * scale)


def _soup(rng, n, spread=1.0):
    v = rng.uniform(-spread, spread, (3 * n, 3)).astype(np.float32)
    return v, np.arange(3 * n, dtype=np.int32).reshape(n, 3)


# ------------------------------------------------------------------ BVH build

def _morton_np(v, t, bits=21):
    v = np.asarray(v, dtype=np.float32)
    used = v[np.unique(t)]
    lo = used.min(0)
    hi = used.max(0)
    ext = np.full(3, (hi - lo).astype(np.float32).max(), dtype=np.float32)
    s = (v[t[:, 0]] + v[t[:, 1]]).astype(np.float32) + v[t[:, 2]]
    x = (s * np.float32(1.0 / 3.0)).astype(np.float32) - lo
    cells = np.float32(1 << bits)
    top = (1 << bits) - 1
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(ext > 0, (x / np.where(ext > 0, ext, 1)).astype(np.float32) * cells, np.float32(0))
    f = f.astype(np.float32)
    q = np.where(f <= 0, 0, np.where(f >= top, top, np.floor(np.maximum(f, 0)))).astype(np.uint64)

    def spread(a):
        out = np.zeros_like(a)
        for i in range(bits):
            out |= ((a >> np.uint64(i)) & np.uint64(1)) << np.uint64(3 * i)
        return out

    return spread(q[:, 0]) | (spread(q[:, 1]) << np.uint64(1)) | (spread(q[:, 2]) << np.uint64(2))


@pytest.mark.parametrize("case", ["torus", "sphere", "soup", "t1", "t2", "t3", "t5", "gear"])
def test_bvh_build_structure(G, ctx, case):
    rng = np.random.default_rng(4)
    m = {
        "torus": lambda: synth.torus(1.0, 0.3, 32, 32),
        "sphere": lambda: synth.geosphere(7, 1.0, 1e-3, 2),
        "soup": lambda: _soup(rng, 1000),
        "t1": lambda: _soup(rng, 1),
        "t2": lambda: _soup(rng, 2),
        "t3": lambda: _soup(rng, 3),
        "t5": lambda: _soup(rng, 5),
        "gear": lambda: synth.gear(96, 3, teeth=12, seed=1),
    }[case]()
    v, t = m
    h = _mesh(G, ctx, m)
    try:
        L, T = G.gd_mesh_info(h)
        assert T == len(t) and (1 << L) <= T < (2 << L)
        boxes, order = G.gd_mesh_download(h)
        # stable Morton order, bit for bit
        keys = _morton_np(v, t)
        assert np.array_equal(order, np.argsort(keys, kind="stable").astype(np.int32))
        _check_tree(boxes, order, v, t, L)
    finally:
        G.gd_mesh_destroy(h)


def _check_tree(boxes, order, v, t, L):
    """Leaves are the exact bounds of their one or two triangles (f12 rule,
    Section 7.3); inner nodes are unions of their children (hence tight)."""
    T = len(t)
    vt = np.asarray(v, dtype=np.float32)[np.asarray(t)[order]]  # (T, 3, 3) in leaf order
    for leaf in range(1 << L):
        s, e = (leaf * T) >> L, ((leaf + 1) * T) >> L
        assert 1 <= e - s <= 2
        pts = vt[s:e].reshape(-1, 3)
        b = boxes[(1 << L) + leaf]
        assert np.array_equal(b[:3], pts.min(0)) and np.array_equal(b[3:], pts.max(0))
    for i in range(1, 1 << L):
        l, r = boxes[2 * i], boxes[2 * i + 1]
        assert np.array_equal(boxes[i][:3], np.minimum(l[:3], r[:3]))
        assert np.array_equal(boxes[i][3:], np.maximum(l[3:], r[3:]))


def test_bvh_build_rejects_bad_input(G, ctx):
    v = np.zeros((3, 3), np.float32)
    t = np.array([[0, 1, 3]], np.int32)
    h = G.gd_mesh_create(ctx, v, t)
    with pytest.raises(G.GdError) as e:
        G.gd_bvh_build(h, ctx=ctx)
    assert e.value.status == G.GD_ERR_INVALID_ARG
    G.gd_mesh_destroy(h)
    v = np.array([[0, 0, 0], [1, 0, 0], [0, np.nan, 0]], np.float32)
    h = G.gd_mesh_create(ctx, v, np.array([[0, 1, 2]], np.int32))
    with pytest.raises(G.GdError):
        G.gd_bvh_build(h, ctx=ctx)
    G.gd_mesh_destroy(h)
    with pytest.raises(G.GdError):
        G.gd_min_distance(ctx, None, None, synth.identity_xform(), synth.identity_xform())


# ------------------------------------------------------------------ queries

def test_two_tori_min_max(G, ctx, oracle_mod):
    import json
    import os
    seed = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "tori_seed.json")))["seed"]
    A, B, xa, xb = synth.config_tori(seed)
    run_pair(G, ctx, oracle_mod, A, B, [(xa, xb)])


@pytest.mark.parametrize("seed", range(5))
def test_random_pairs(G, ctx, oracle_mod, seed):
    rng = np.random.default_rng(1000 + seed)
    kinds = [
        lambda: synth.torus(1.0, 0.25, 20 + seed, 13),
        lambda: synth.geosphere(5 + seed, 0.7, 2e-3, seed),
        lambda: _soup(rng, 300 + 77 * seed, 0.8),
        lambda: synth.gear(128, 3, teeth=16, seed=seed),
    ]
    A = kinds[seed % 4]()
    B = kinds[(seed + 2) % 4]()
    xs = []
    for k in range(6):
        xa = _rigid(rng)
        off = synth.xform(np.eye(3), rng.normal(size=3) * (0.4 + 0.5 * k))
        xb = synth.compose(off, synth.compose(xa, synth.xform(synth.random_rotation(rng), (0, 0, 0))))
        xs.append((xa, xb))
    run_pair(G, ctx, oracle_mod, A, B, xs)


def test_edge_cases(G, ctx, oracle_mod):
    rng = np.random.default_rng(9)
    I = synth.identity_xform()
    one = _soup(rng, 1)
    two = _soup(rng, 2)
    torus = synth.torus(1.0, 0.3, 16, 12)
    # single triangles, tiny meshes, ragged leaf counts
    run_pair(G, ctx, oracle_mod, one, one, [(I, synth.xform(np.eye(3), (3, 0, 0))), (I, I)])
    run_pair(G, ctx, oracle_mod, one, torus, [(I, synth.xform(np.eye(3), (0.5, 0.2, 2)))])
    run_pair(G, ctx, oracle_mod, two, _soup(rng, 7), [(_rigid(rng), _rigid(rng)) for _ in range(3)])
    # identical placement: intersecting, d = 0
    run_pair(G, ctx, oracle_mod, torus, torus, [(I, I)], kinds=("min",))
    # far apart (large coordinates)
    run_pair(G, ctx, oracle_mod, torus, torus, [(I, synth.xform(synth.random_rotation(rng), (1e3, -2e3, 5e2)))])
    # nested spheres: the inner one is strictly inside, surface distance > 0
    run_pair(G, ctx, oracle_mod, synth.geosphere(6, 1.0), synth.geosphere(5, 0.5), [(I, I)])
    # degenerate (zero-area) triangles
    v = np.array([[0, 0, 0], [1, 0, 0], [2, 0, 0], [0, 1, 0], [0, 2, 0]], np.float32)
    degen = (v, np.array([[0, 1, 2], [0, 3, 4], [1, 1, 1]], np.int32))
    run_pair(G, ctx, oracle_mod, degen, torus, [(I, synth.xform(np.eye(3), (0.3, 0.1, 1.0)))])


def test_closed_forms_on_gpu(G, ctx, oracle_mod):
    g = 0.0625
    A = synth.box((0, 0, 0), (1, 1, 1))
    B = synth.box((1 + g, 0.25, 0.5), (2 + g, 0.75, 1.5))
    I = synth.identity_xform()
    ma, mb = _mesh(G, ctx, A), _mesh(G, ctx, B)
    r = G.gd_min_distance(ctx, ma, mb, I, I)
    assert r.d == pytest.approx(g, abs=1e-12)
    r = G.gd_max_distance(ctx, ma, mb, I, I)
    assert r.d == pytest.approx(math.sqrt((2 + g) ** 2 + 0.75 ** 2 + 1.5 ** 2), rel=1e-13)
    G.gd_mesh_destroy(ma)
    G.gd_mesh_destroy(mb)
    gz = 0.01
    A = synth.grid(24, 1.0, 0.0)
    B = synth.grid(24, 1.0, gz, x0=0.3, y0=0.25)
    run_pair(G, ctx, oracle_mod, A, B, [(I, I)])


def test_icospheres_small(G, ctx, oracle_mod):
    A, B, xa, xb = synth.config_icospheres(level=4, seed=3)
    run_pair(G, ctx, oracle_mod, A, B, [(xa, xb)], bvh_oracle=True)


def test_batch_matches_single(G, ctx, oracle_mod):
    rng = np.random.default_rng(77)
    A = synth.gear(256, 4, teeth=16, seed=2)
    B = synth.geosphere(9, 0.5, 1e-3, 5)
    Tm = synth.torus(1.0, 0.2, 24, 10)
    ma, mb = _mesh(G, ctx, A), _mesh(G, ctx, B)
    mt = _mesh(G, ctx, Tm)
    items, data = [], []
    for i in range(40):
        xa = _rigid(rng, 0.2)
        xb = _rigid(rng, 1.2)
        pair = [(ma, mb), (mb, mt), (mt, ma)][i % 3]
        data.append([(A, B), (B, Tm), (Tm, A)][i % 3])
        items.append((pair[0], pair[1], xa, xb, i % 2))
    out = G.gd_batch_query(ctx, items)
    for i, (a, b, xa, xb, kind) in enumerate(items):
        fn = G.gd_min_distance if kind == 0 else G.gd_max_distance
        r = fn(ctx, a, b, xa, xb)
        same_answer(out[i], r, oracle_mod, data[i][0], xa, data[i][1], xb, "min" if kind == 0 else "max")
    for h in (ma, mb, mt):
        G.gd_mesh_destroy(h)


def test_batch_eviction_matches_single(G, oracle_mod):
    """A query of a batch that pushes more than its share of the queues in one
    level leaves the batch and runs alone.  With queues of 1024 entries and 24
    queries the share is 21 entries per level, so most queries are evicted;
    every answer still equals the single-query answer."""
    c = G.gd_ctx_create(0)
    try:
        rng = np.random.default_rng(91)
        A = synth.gear(256, 4, teeth=16, seed=2)
        B = synth.geosphere(9, 0.5, 1e-3, 5)
        ma, mb = _mesh(G, c, A), _mesh(G, c, B)
        items = [(ma, mb, _rigid(rng, 0.2), _rigid(rng, 1.2), i % 2) for i in range(24)]
        alone = []
        for a, b, xa, xb, kind in items:
            fn = G.gd_min_distance if kind == 0 else G.gd_max_distance
            alone.append(fn(c, a, b, xa, xb))
        G.gd_ctx_set_tunables(c, front_capacity=1024, leaf_capacity=1024, batch_budget=8)
        out = G.gd_batch_query(c, items)
        assert G.gd_get_stats(c)["retries"] > 0
        for i, (a, b, xa, xb, kind) in enumerate(items):
            same_answer(out[i], alone[i], oracle_mod, A, xa, B, xb, "min" if kind == 0 else "max")
        G.gd_mesh_destroy(ma)
        G.gd_mesh_destroy(mb)
    finally:
        G.gd_ctx_destroy(c)


def test_refit_modes_agree(G, oracle_mod):
    """Refitting B only tightens bounds: with the lazy refit of B's low
    subtrees (mode 1), without refit (mode 2) and with the paper's full refit
    of B into A's frame per query (mode 3), every answer matches the FP64
    oracle (value and witness), single query and device-resident, and the
    modes give the same answer."""
    rng = np.random.default_rng(31)
    c = G.gd_ctx_create(0)
    try:
        A = synth.torus(1.0, 0.1, 96, 40)
        B = synth.geosphere(20, 0.5, 1e-3, 3)
        ma, mb = _mesh(G, c, A), _mesh(G, c, B)
        oa, ob = oracle_mod.Bvh(A), oracle_mod.Bvh(B)
        for i in range(6):
            xa, xb = _rigid(rng, 0.3), _rigid(rng, 1.2)
            diag = oracle_mod.diag(A, xa, B, xb)
            for kind, fn in (("min", G.gd_min_distance), ("max", G.gd_max_distance)):
                ref = oracle_mod.bvh_query(oa, xa, ob, xb, kind)
                G.gd_ctx_set_tunables(c, refit_mode=1)
                r1 = fn(c, ma, mb, xa, xb)
                check(r1, A, xa, B, xb, kind, ref, diag, oracle_mod)
                G.gd_ctx_set_tunables(c, refit_mode=2)
                r2 = fn(c, ma, mb, xa, xb)
                check(r2, A, xa, B, xb, kind, ref, diag, oracle_mod)
                same_answer(r1, r2, oracle_mod, A, xa, B, xb, kind)
                G.gd_ctx_set_tunables(c, refit_mode=3)
                r3 = fn(c, ma, mb, xa, xb)
                check(r3, A, xa, B, xb, kind, ref, diag, oracle_mod)
                same_answer(r1, r3, oracle_mod, A, xa, B, xb, kind)
                G.gd_ctx_set_tunables(c, refit_mode=1)
        G.gd_mesh_destroy(ma)
        G.gd_mesh_destroy(mb)
    finally:
        G.gd_ctx_destroy(c)


def test_conventional_bounds_ablation(G, oracle_mod):
    """Section 9's ablation: with conventional bounds only (Eq. 9 for the min,
    the box gap for the max) and with a fixed k (a huge work target, k = 5)
    every answer matches the FP64 oracle, and the conventional bounds test at
    least as many node pairs; the enhanced bounds cull more."""
    c = G.gd_ctx_create(0)
    try:
        rng = np.random.default_rng(19)
        A = synth.torus(1.0, 0.1, 96, 40)
        B = synth.geosphere(20, 0.5, 1e-3, 3)
        ma, mb = _mesh(G, c, A), _mesh(G, c, B)
        oa, ob = oracle_mod.Bvh(A), oracle_mod.Bvh(B)
        base = G.gd_ctx_get_tunables(c)
        more = 0
        for i in range(4):
            xa, xb = _rigid(rng, 0.3), _rigid(rng, 1.5)
            diag = oracle_mod.diag(A, xa, B, xb)
            for kind, fn in (("min", G.gd_min_distance), ("max", G.gd_max_distance)):
                ref = oracle_mod.bvh_query(oa, xa, ob, xb, kind)
                G.gd_ctx_set_tunables(c, bounds_mode=1)
                r1 = fn(c, ma, mb, xa, xb)
                p1 = G.gd_get_stats(c)["pairs_tested"]
                check(r1, A, xa, B, xb, kind, ref, diag, oracle_mod)
                G.gd_ctx_set_tunables(c, bounds_mode=2)
                r2 = fn(c, ma, mb, xa, xb)
                p2 = G.gd_get_stats(c)["pairs_tested"]
                check(r2, A, xa, B, xb, kind, ref, diag, oracle_mod)
                same_answer(r1, r2, oracle_mod, A, xa, B, xb, kind)
                G.gd_ctx_set_tunables(c, bounds_mode=1, k_max=5, work_target=1 << 40)
                r3 = fn(c, ma, mb, xa, xb)
                check(r3, A, xa, B, xb, kind, ref, diag, oracle_mod)
                G.gd_ctx_set_tunables(c, k_max=base["k_max"], work_target=base["work_target"])
                more += p2 > p1
        assert more > 0
        G.gd_ctx_set_tunables(c, bounds_mode=1)
        G.gd_mesh_destroy(ma)
        G.gd_mesh_destroy(mb)
    finally:
        G.gd_ctx_destroy(c)


def test_autotune_keeps_answers(G, oracle_mod):
    """gd_autotune picks tunables by timing and never changes an answer: the
    answers before and after tuning are the same (single query and batch)."""
    c = G.gd_ctx_create(0)
    try:
        rng = np.random.default_rng(23)
        A = synth.torus(1.0, 0.1, 96, 40)
        B = synth.geosphere(12, 0.5, 1e-3, 3)
        ma, mb = _mesh(G, c, A), _mesh(G, c, B)
        items = [(ma, mb, _rigid(rng, 0.3), _rigid(rng, 1.5), i % 2) for i in range(8)]
        before = G.gd_batch_query(c, items)
        one = G.gd_min_distance(c, ma, mb, items[0][2], items[0][3])
        t1 = G.gd_autotune(c, items[:1], reps=2)
        assert t1["k_max"] in (4, 5, 6, 7) and t1["work_target"] >= 1 << 16
        t2 = G.gd_autotune(c, items, reps=2)
        assert t2["batch_budget"] in (1 << 18, 1 << 20, 1 << 22, 1 << 23, 1 << 24)
        after = G.gd_batch_query(c, items)
        oa, ob = oracle_mod.Bvh(A), oracle_mod.Bvh(B)
        for i, (a, b, xa, xb, kind) in enumerate(items):
            name = "min" if kind == 0 else "max"
            ref = oracle_mod.bvh_query(oa, xa, ob, xb, name)
            diag = oracle_mod.diag(A, xa, B, xb)
            check(before[i], A, xa, B, xb, name, ref, diag, oracle_mod)
            check(after[i], A, xa, B, xb, name, ref, diag, oracle_mod)
            same_answer(before[i], after[i], oracle_mod, A, xa, B, xb, name)
        tuned = G.gd_min_distance(c, ma, mb, items[0][2], items[0][3])
        ref = oracle_mod.bvh_query(oa, items[0][2], ob, items[0][3], "min")
        diag = oracle_mod.diag(A, items[0][2], B, items[0][3])
        check(one, A, items[0][2], B, items[0][3], "min", ref, diag, oracle_mod)
        check(tuned, A, items[0][2], B, items[0][3], "min", ref, diag, oracle_mod)
        same_answer(one, tuned, oracle_mod, A, items[0][2], B, items[0][3], "min")
        G.gd_mesh_destroy(ma)
        G.gd_mesh_destroy(mb)
    finally:
        G.gd_ctx_destroy(c)


def _tie_meshes(kind):
    """Meshes whose extreme pairs tie exactly (dyadic coordinates, identity
    transforms, tied pairs that repeat the same float64 operations on the
    same differences).  Min: two copies of a triangle pair 1/2 apart (one
    shifted by 8 along x) at (5, 2) and (3, 6), and a duplicate of B's
    triangle at index 4.  Max: a pair 8 apart at its outer vertices at (5, 2)
    and its mirror image through the origin at (3, 6).  The tied set is no
    product of index sets, so only the smallest (tri_a, tri_b) rule gives
    (3, 6)."""
    def mesh(tris):
        v = np.asarray([p for t in tris for p in t], dtype=np.float32)
        return v, np.arange(len(v), dtype=np.int32).reshape(-1, 3)

    def tri(o, pts):
        return [tuple(np.add(o, p)) for p in pts]

    if kind == "min":
        ta = [(0, 0, 0), (1, 0, 0), (0, 1, 0)]
        tb = [(0.25, 0.25, 0.5), (0.5, 0.25, 0.5), (0.25, 0.5, 0.5)]
        fa = lambda i: tri((4 * i, 20, -8), ta)
        fb = lambda i: tri((4 * i, -20, 8), tb)
        A = [fa(0), fa(1), fa(2), tri((8, 0, 0), ta), fa(4), tri((0, 0, 0), ta), fa(6)]
        B = [fb(0), fb(1), tri((0, 0, 0), tb), fb(3), tri((0, 0, 0), tb), fb(5), tri((8, 0, 0), tb)]
        return mesh(A), mesh(B), 0.5
    ta = [(-2, 0, 0), (-1.5, 0.5, 0), (-1.5, -0.5, 0)]
    tb = [(6, 0, 0), (5.5, 0.5, 0), (5.5, -0.5, 0)]
    neg = lambda t: [tuple(-np.asarray(p)) for p in t]
    fa = lambda i: tri((0, 0, 0.25 * i), [(0, 0, 0), (0.25, 0, 0), (0, 0.25, 0)])
    fb = lambda i: tri((0.5, 0, 0.25 * i), [(0, 0, 0), (0.25, 0, 0), (0, 0.25, 0)])
    A = [fa(0), fa(1), fa(2), neg(ta), fa(4), ta, fa(6)]
    B = [fb(0), fb(1), tb, fb(3), fb(4), fb(5), neg(tb)]
    return mesh(A), mesh(B), 8.0


def test_witness_tie_break_exact_ties(G, ctx, oracle_mod):
    """The engine's witness rule on exact ties (gd_result: the smallest
    (tri_a, tri_b) at the extreme), single query and batch, min and max,
    equal to the oracle's witness."""
    I = synth.identity_xform()
    for kind in ("min", "max"):
        A, B, dx = _tie_meshes(kind)
        ref = oracle_mod.brute(A, I, B, I, kind)
        assert ref.d == dx and (ref.ta, ref.tb) == (3, 6)
        ma, mb = _mesh(G, ctx, A), _mesh(G, ctx, B)
        fn = G.gd_min_distance if kind == "min" else G.gd_max_distance
        r = fn(ctx, ma, mb, I, I)
        assert r.status == 0 and r.d == dx and (r.tri_a, r.tri_b) == (3, 6), (kind, r.d, r.tri_a, r.tri_b)
        k = G.GD_MIN if kind == "min" else G.GD_MAX
        out = G.gd_batch_query(ctx, [(ma, mb, I, I, k)] * 3)
        for o in out:
            assert o.status == 0 and o.d == dx and (o.tri_a, o.tri_b) == (3, 6)
        G.gd_mesh_destroy(ma)
        G.gd_mesh_destroy(mb)


def test_nearly_parallel_edges(G, ctx, oracle_mod):
    """Two triangles whose closest pair is interior to two edges at a tiny
    angle eps, h apart (the stationary point of the edge pair, which a
    difference-of-products determinant loses for eps below ~1e-7), under
    rigid motions: the float64 refinement matches the oracle (value within
    the parity tolerance, witness distance within 1e-12 relative)."""
    rng = np.random.default_rng(88)
    h = 2.0 ** -10
    for k in (12, 20, 26, 34):
        eps = 2.0 ** -k
        A = (np.array([[-1, 0, 0], [1, 0, 0], [0, -1, -0.5]], dtype=np.float32), np.array([[0, 1, 2]], np.int32))
        B = (np.array([[-1, -eps, h], [1, eps, h], [0, 1, h + 0.5]], dtype=np.float32), np.array([[0, 1, 2]], np.int32))
        ma, mb = _mesh(G, ctx, A), _mesh(G, ctx, B)
        for j in range(3):
            M = synth.identity_xform() if j == 0 else _rigid(rng, 2.0)
            ref = oracle_mod.brute(A, M, B, M, "min")
            assert abs(ref.d - h) <= 4e-15
            r = G.gd_min_distance(ctx, ma, mb, M, M)
            check(r, A, M, B, M, "min", ref, oracle_mod.diag(A, M, B, M), oracle_mod)
        G.gd_mesh_destroy(ma)
        G.gd_mesh_destroy(mb)


def test_device_resident_query(G, ctx, oracle_mod):
    torch = pytest.importorskip("torch")
    A, B, xa, xb = synth.config_tori(1)
    ma, mb = _mesh(G, ctx, A), _mesh(G, ctx, B)
    ref = G.gd_min_distance(ctx, ma, mb, xa, xb)
    dxa = torch.tensor(xa, dtype=torch.float64, device="cuda")
    dxb = torch.tensor(xb, dtype=torch.float64, device="cuda")
    out = torch.zeros(10, dtype=torch.float64, device="cuda")  # 80 bytes
    stream = torch.cuda.current_stream().cuda_stream
    G.gd_query_device(ctx, ma, mb, G.GD_MIN, dxa.data_ptr(), dxb.data_ptr(), out.data_ptr(), stream)
    torch.cuda.synchronize()
    raw = out.cpu().numpy().tobytes()
    r = G.gd_result.from_buffer_copy(raw)
    assert r.status == 0 and r.d == ref.d and (r.tri_a, r.tri_b) == (ref.tri_a, ref.tri_b)
    G.gd_mesh_destroy(ma)
    G.gd_mesh_destroy(mb)


def test_graph_replays_match_calls(G, ctx, oracle_mod):
    """A captured graph of one device-resident query, replayed after the
    transforms are updated in place, gives the answers of the synchronous
    calls; it is rebuilt when the tunables change."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(41)
    A = synth.torus(1.0, 0.2, 64, 24)
    B = synth.geosphere(10, 0.5, 1e-3, 4)
    ma, mb = _mesh(G, ctx, A), _mesh(G, ctx, B)
    xa = _rigid(rng, 0.2)
    G.gd_min_distance(ctx, ma, mb, xa, _rigid(rng, 1.5))
    dxa = torch.tensor(np.asarray(xa), dtype=torch.float64, device="cuda")
    dxb = torch.zeros(12, dtype=torch.float64, device="cuda")
    out = torch.zeros(10, dtype=torch.float64, device="cuda")
    g = G.gd_graph_create(ctx, ma, mb, G.GD_MIN, dxa.data_ptr(), dxb.data_ptr(), out.data_ptr())
    stream = torch.cuda.current_stream().cuda_stream
    try:
        for i in range(6):
            xb = _rigid(rng, 1.5)
            dxb.copy_(torch.tensor(np.asarray(xb), dtype=torch.float64))
            torch.cuda.synchronize()
            if i == 3:
                G.gd_ctx_set_tunables(ctx, probes=16)
            G.gd_graph_launch(g, stream, ctx)
            torch.cuda.synchronize()
            r = G.gd_result.from_buffer_copy(out.cpu().numpy().tobytes())
            ref = G.gd_min_distance(ctx, ma, mb, xa, xb)
            same_answer(r, ref, oracle_mod, A, xa, B, xb, "min")
    finally:
        G.gd_graph_destroy(g)
        G.gd_ctx_set_tunables(ctx, probes=64)
        G.gd_mesh_destroy(ma)
        G.gd_mesh_destroy(mb)


def test_overflow_grows_then_reports(G, oracle_mod):
    """Capacity faults are injected on the host: tiny queues must grow and
    still give the oracle's answer; a growth limit below the need reports
    GD_ERR_OVERFLOW.  Two parallel grids 0.01 apart: every facing pair is at
    the minimum, so the fronts are large and nothing intersects."""
    c = G.gd_ctx_create(0)
    try:
        A = synth.grid(32, 1.0, 0.0)
        B = synth.grid(32, 1.0, 0.01)
        I = synth.identity_xform()
        ma, mb = _mesh(G, c, A), _mesh(G, c, B)
        G.gd_ctx_set_tunables(c, front_capacity=64, leaf_capacity=64, cand_capacity=16, max_capacity=1 << 24)
        r = G.gd_min_distance(c, ma, mb, I, I)
        ref = oracle_mod.brute(A, I, B, I)
        check(r, A, I, B, I, "min", ref, oracle_mod.diag(A, I, B, I), oracle_mod)
        assert G.gd_get_stats(c)["retries"] > 0
        G.gd_ctx_set_tunables(c, front_capacity=64, leaf_capacity=64, cand_capacity=16, max_capacity=128)
        with pytest.raises(G.GdError) as e:
            G.gd_min_distance(c, ma, mb, I, I)
        assert e.value.status == G.GD_ERR_OVERFLOW
        G.gd_mesh_destroy(ma)
        G.gd_mesh_destroy(mb)
    finally:
        G.gd_ctx_destroy(c)


def test_zero_proof_stops_traversal(G, oracle_mod):
    """D_min = 0 (Section 8, penetration): a pair proven to intersect in
    float64 ends the query.  Coincident copies of one mesh overlap everywhere,
    so without the proof the fronts need far more than 128 entries; with it
    the answer is 0 (flags bit 1 set) and its witness intersects in the
    oracle.  Two tori crossing each other give 0 with a valid witness too."""
    c = G.gd_ctx_create(0)
    try:
        rng = np.random.default_rng(12)
        A = synth.torus(1.0, 0.25, 64, 32)
        x = _rigid(rng, 0.5)
        ma, mb = _mesh(G, c, A), _mesh(G, c, A)
        G.gd_ctx_set_tunables(c, front_capacity=64, leaf_capacity=64, cand_capacity=16, max_capacity=128,
                              probes=64)
        r = G.gd_min_distance(c, ma, mb, x, x)
        assert r.status == 0 and r.d == 0.0 and r.flags == 3, (r.status, r.d, r.flags)
        dw, _, _ = oracle_mod.witness_distance(A, x, A, x, r.tri_a, r.tri_b, "min")
        assert dw == 0.0
        G.gd_ctx_set_tunables(c, front_capacity=1 << 16, leaf_capacity=1 << 16, cand_capacity=1 << 14,
                              max_capacity=1 << 26)
        xb = synth.compose(x, synth.xform(np.eye(3), (0.4, 0.0, 0.0)))
        r = G.gd_min_distance(c, ma, mb, x, xb)
        ref = oracle_mod.brute(A, x, A, xb)
        assert ref.d == 0.0
        check(r, A, x, A, xb, "min", ref, oracle_mod.diag(A, x, A, xb), oracle_mod)
        G.gd_mesh_destroy(ma)
        G.gd_mesh_destroy(mb)
    finally:
        G.gd_ctx_destroy(c)


def test_wait_timeout_returns_status_and_context_survives(G, oracle_mod):
    """A 1 ns bound on every grid-barrier wait makes the waits run out: the
    kernel returns early, the call reports GD_ERR_TIMEOUT, and the same
    context answers correctly once the bound is restored."""
    c = G.gd_ctx_create(0)
    try:
        A, B, xa, xb = synth.config_tori(1)
        ma, mb = _mesh(G, c, A), _mesh(G, c, B)
        G.gd_ctx_set_tunables(c, timeout_ns=1)
        saw_timeout = False
        for _ in range(5):
            try:
                G.gd_min_distance(c, ma, mb, xa, xb)
            except G.GdError as e:
                assert e.status == G.GD_ERR_TIMEOUT
                saw_timeout = True
                break
        assert saw_timeout
        G.gd_ctx_set_tunables(c, timeout_ns=2_000_000_000)
        r = G.gd_min_distance(c, ma, mb, xa, xb)
        ref = oracle_mod.brute(A, xa, B, xb)
        check(r, A, xa, B, xb, "min", ref, oracle_mod.diag(A, xa, B, xb), oracle_mod)
        G.gd_mesh_destroy(ma)
        G.gd_mesh_destroy(mb)
    finally:
        G.gd_ctx_destroy(c)


def test_serve_alone_equals_in_mix(G, ctx, oracle_mod):
    import time
    rng = np.random.default_rng(5)
    meshes = [synth.torus(1.0, 0.25, 40, 20), synth.geosphere(12, 0.6, 1e-3, 1), synth.gear(256, 4, teeth=16, seed=3)]
    hs = [_mesh(G, ctx, m) for m in meshes]
    qs, ids = [], []
    for i in range(60):
        a, b = int(rng.integers(0, 3)), int(rng.integers(0, 3))
        ids.append((a, b))
        qs.append((hs[a], hs[b], _rigid(rng, 0.3), _rigid(rng, 1.5), int(rng.integers(0, 2))))
    arr = G.make_queries(qs)
    alone = []
    for q in qs:
        fn = G.gd_min_distance if q[4] == 0 else G.gd_max_distance
        alone.append(fn(ctx, q[0], q[1], q[2], q[3]))
    srv = G.gd_serve_start(ctx, max_batch=16)
    try:
        tickets = []
        for i in range(len(qs)):
            rc, t = G.gd_serve_submit(srv, arr[i])
            assert rc == 0
            tickets.append(t)
        got = {}
        deadline = time.time() + 120
        while len(got) < len(tickets) and time.time() < deadline:
            for t in tickets:
                if t in got:
                    continue
                rc, r = G.gd_serve_poll(srv, t)
                if rc == 0:
                    got[t] = r
                else:
                    assert rc == G.GD_ERR_NOT_READY
            time.sleep(0.001)
    finally:
        G.gd_serve_stop(srv)
    assert len(got) == len(tickets)
    bvh = [oracle_mod.Bvh(m) for m in meshes]
    for i, t in enumerate(tickets):
        a, b = ids[i]
        kind = "min" if qs[i][4] == 0 else "max"
        same_answer(got[t], alone[i], oracle_mod, meshes[a], qs[i][2], meshes[b], qs[i][3], kind)
        ref = oracle_mod.bvh_query(bvh[a], qs[i][2], bvh[b], qs[i][3], kind)
        check(got[t], meshes[a], qs[i][2], meshes[b], qs[i][3], kind, ref,
              oracle_mod.diag(meshes[a], qs[i][2], meshes[b], qs[i][3]), oracle_mod)
    for h in hs:
        G.gd_mesh_destroy(h)


def test_serve_admission_by_footprint(G, ctx, oracle_mod):
    """Admission by HBM footprint: with a budget below the predicted
    footprints of two requests together, the second submission is refused
    (GD_ERR_BUSY) while the first is held (queued: a long linger keeps it
    waiting for company), and admitted once the first has finished; both
    answers match the oracle.  A request larger than the whole budget is
    admitted onto an empty server and still answered."""
    import time
    rng = np.random.default_rng(12)
    A, B = synth.torus(1.0, 0.25, 40, 20), synth.geosphere(12, 0.6, 1e-3, 1)
    ha, hb = _mesh(G, ctx, A), _mesh(G, ctx, B)
    items = [(ha, hb, _rigid(rng, 0.3), _rigid(rng, 1.5), G.GD_MIN) for _ in range(2)]
    arr = G.make_queries(items)
    f1, f2 = G.gd_query_footprint(arr[0]), G.gd_query_footprint(arr[1])
    assert f1 > 1024 and f2 > 1024

    def wait(srv, t):
        deadline = time.time() + 60
        while time.time() < deadline:
            rc, r = G.gd_serve_poll(srv, t)
            if rc == 0:
                return r
            assert rc == G.GD_ERR_NOT_READY
            time.sleep(0.001)
        raise AssertionError("request not served")

    oa, ob = oracle_mod.Bvh(A), oracle_mod.Bvh(B)
    for budget in (f1 + f2 - 1, f1 // 2):
        srv = G.gd_serve_start(ctx, max_batch=16, memory_budget=budget, linger_us=300000)
        try:
            rc1, t1 = G.gd_serve_submit(srv, arr[0])
            assert rc1 == 0
            rc2, _ = G.gd_serve_submit(srv, arr[1])
            assert rc2 == G.GD_ERR_BUSY
            r1 = wait(srv, t1)
            rc2, t2 = G.gd_serve_submit(srv, arr[1])
            assert rc2 == 0
            r2 = wait(srv, t2)
        finally:
            G.gd_serve_stop(srv)
        for r, (a, b, xa, xb, k) in zip((r1, r2), items):
            ref = oracle_mod.bvh_query(oa, xa, ob, xb, "min")
            check(r, A, xa, B, xb, "min", ref, oracle_mod.diag(A, xa, B, xb), oracle_mod)
    G.gd_mesh_destroy(ha)
    G.gd_mesh_destroy(hb)


def test_serve_drain_collects_every_ticket(G, ctx, oracle_mod):
    """gd_serve_drain hands back every finished request once, with the same
    answer as the request alone."""
    import time
    rng = np.random.default_rng(8)
    meshes = [synth.torus(1.0, 0.25, 40, 20), synth.geosphere(12, 0.6, 1e-3, 1)]
    hs = [_mesh(G, ctx, m) for m in meshes]
    qs = [(hs[i % 2], hs[(i + 1) % 2], _rigid(rng, 0.3), _rigid(rng, 1.5), G.GD_MIN) for i in range(40)]
    alone = [G.gd_min_distance(ctx, q[0], q[1], q[2], q[3]) for q in qs]
    arr = G.make_queries(qs)
    srv = G.gd_serve_start(ctx, max_batch=8)
    try:
        idx = {}
        for i in range(len(qs)):
            rc, t = G.gd_serve_submit(srv, arr[i])
            assert rc == 0
            idx[t] = i
        got = {}
        deadline = time.time() + 120
        while len(got) < len(qs) and time.time() < deadline:
            for t, r in G.gd_serve_drain(srv, 16):
                assert t in idx and t not in got
                got[t] = r
            time.sleep(0.001)
    finally:
        G.gd_serve_stop(srv)
    assert len(got) == len(qs)
    for t, r in got.items():
        i = idx[t]
        a = 0 if i % 2 == 0 else 1
        same_answer(r, alone[i], oracle_mod, meshes[a], qs[i][2], meshes[1 - a], qs[i][3], "min")
    for h in hs:
        G.gd_mesh_destroy(h)


# ------------------------------------------------------------------ deformable meshes

def test_mesh_update_refits_tree(G, ctx):
    """A refit keeps the build's leaf order and makes every box tight for the
    new vertices again (bit for bit: min/max of float32 values are exact)."""
    for v, t in (synth.torus(1.0, 0.3, 32, 32), synth.gear(96, 3, teeth=12, seed=1), _soup(np.random.default_rng(5), 5)):
        h = _mesh(G, ctx, (v, t))
        try:
            L, _ = G.gd_mesh_info(h)
            _, order0 = G.gd_mesh_download(h)
            for ph in (0.3, 2.1):
                w = synth.warp(v, 0.05, 1.0, ph)
                G.gd_mesh_update(h, w, ctx=ctx)
                boxes, order = G.gd_mesh_download(h)
                assert np.array_equal(order, order0)
                _check_tree(boxes, order, w, t, L)
        finally:
            G.gd_mesh_destroy(h)


def test_deformable_frames_match_oracle(G, ctx, oracle_mod):
    """Frames of a deforming torus B next to a rigid torus A (the Deformable
    scene of Section 8): each frame uploads B's warped vertices (from the host
    on even frames, from device memory on odd ones) and refits its tree; min
    and max distances match the oracle on the warped mesh, and equal a query
    on a mesh built from scratch from the same vertices."""
    import torch
    A = synth.torus(1.0, 0.3, 24, 20)
    vb, tb = synth.torus(0.8, 0.25, 28, 18)
    xa = synth.identity_xform()
    rng = np.random.default_rng(31)
    ma, mb = _mesh(G, ctx, A), _mesh(G, ctx, (vb, tb))
    try:
        for f in range(4):
            w = synth.warp(vb, 0.08, 0.7, rng.uniform(0, 2 * math.pi))
            if f % 2:
                G.gd_mesh_update(mb, torch.from_numpy(w).cuda(), ctx=ctx)
            else:
                G.gd_mesh_update(mb, w, ctx=ctx)
            B = (w, tb)
            xb = synth.xform(synth.random_rotation(rng), rng.normal(size=3) * 0.6 + (1.6, 0, 0))
            diag = oracle_mod.diag(A, xa, B, xb)
            fresh = _mesh(G, ctx, B)
            try:
                for kind in ("min", "max"):
                    fn = G.gd_min_distance if kind == "min" else G.gd_max_distance
                    r = fn(ctx, ma, mb, xa, xb)
                    check(r, A, xa, B, xb, kind, oracle_mod.brute(A, xa, B, xb, kind), diag, oracle_mod)
                    same_answer(r, fn(ctx, ma, fresh, xa, xb), oracle_mod, A, xa, B, xb, kind)
            finally:
                G.gd_mesh_destroy(fresh)
    finally:
        G.gd_mesh_destroy(ma)
        G.gd_mesh_destroy(mb)


def test_mesh_update_rejects_bad_input(G, ctx, oracle_mod):
    v, t = synth.torus(1.0, 0.3, 12, 10)
    I = synth.identity_xform()
    far = synth.xform(np.eye(3), (3.0, 0.0, 0.0))
    h = _mesh(G, ctx, (v, t))
    try:
        with pytest.raises(G.GdError) as e:
            G.gd_mesh_update(h, v[:-1], ctx=ctx)
        assert e.value.status == G.GD_ERR_INVALID_ARG
        r0 = G.gd_min_distance(ctx, h, h, I, far)  # the mesh is untouched
        bad = v.copy()
        bad[7, 1] = np.inf
        with pytest.raises(G.GdError) as e:
            G.gd_mesh_update(h, bad, ctx=ctx)
        assert e.value.status == G.GD_ERR_INVALID_ARG
        with pytest.raises(G.GdError) as e:
            G.gd_min_distance(ctx, h, h, I, far)
        assert e.value.status == G.GD_ERR_NOT_BUILT
        G.gd_mesh_update(h, v, ctx=ctx)  # a valid update makes it usable again
        r1 = G.gd_min_distance(ctx, h, h, I, far)
        assert (r1.d, r1.tri_a, r1.tri_b) == (r0.d, r0.tri_a, r0.tri_b)
        unbuilt = G.gd_mesh_create(ctx, v, t)
        with pytest.raises(G.GdError) as e:
            G.gd_mesh_update(unbuilt, v, ctx=ctx)
        assert e.value.status == G.GD_ERR_NOT_BUILT
        G.gd_mesh_destroy(unbuilt)
    finally:
        G.gd_mesh_destroy(h)


# ------------------------------------------------------------------ point-to-mesh queries

def _probe_points(rng, mesh, x, n):
    """World points around a placed mesh: uniform in its grown bounding box,
    vertices pushed off the surface by small offsets, exact vertices (d = 0)
    and far points."""
    w = oracle_world(mesh, x)
    lo, hi = w.min(0), w.max(0)
    ext = hi - lo
    a = rng.uniform(lo - 0.3 * ext, hi + 0.3 * ext, (n, 3))
    v = w[rng.integers(0, len(w), n)]
    b = v + rng.normal(size=(n, 3)) * 1e-3 * ext.max()
    c = w[rng.integers(0, len(w), max(1, n // 8))]
    d = (lo + hi) / 2 + rng.normal(size=(max(1, n // 8), 3)) * 20 * ext.max()
    return np.concatenate([a, b, c, d])


def oracle_world(mesh, x):
    v = np.asarray(mesh[0], dtype=np.float64)
    X = np.asarray(x, dtype=np.float64).reshape(3, 4)
    return v @ X[:, :3].T + X[:, 3]


def check_points(res, mesh, x, pts, oracle):
    d_ref, _, _ = oracle.point_mesh(mesh, x, pts)
    w = oracle_world(mesh, x)
    t = np.asarray(mesh[1])
    scale = np.abs(pts).max(1) + np.abs(w).max()
    tol = 1e-13 * scale
    assert (res["status"] == 0).all()
    assert np.all(np.abs(res["d"] - d_ref) <= tol), np.max(np.abs(res["d"] - d_ref) / scale)
    for i in range(len(pts)):
        dw, _ = oracle.point_triangle(pts[i], *w[t[res["tri"][i]]])
        assert abs(dw - d_ref[i]) <= tol[i], (i, dw, d_ref[i])
        assert abs(np.linalg.norm(res["p"][i] - pts[i]) - res["d"][i]) <= tol[i]
        assert oracle.point_triangle(res["p"][i], *w[t[res["tri"][i]]])[0] <= tol[i]


def test_point_distance_matches_oracle(G, ctx, oracle_mod):
    rng = np.random.default_rng(51)
    meshes = [
        synth.torus(1.0, 0.3, 24, 16),
        synth.geosphere(6, 0.8, 2e-3, 1),
        synth.gear(96, 3, teeth=12, seed=2),
        _soup(rng, 200, 0.7),
        _soup(rng, 1),
    ]
    for m in meshes:
        h = _mesh(G, ctx, m)
        try:
            for _ in range(2):
                x = _rigid(rng)
                # plus the placed mesh's centre (the middle of the torus hole,
                # the centre of the sphere: many triangles at nearly one distance)
                X = np.asarray(x).reshape(3, 4)
                centre = X[:, :3] @ np.asarray(m[0], dtype=np.float64).mean(0) + X[:, 3]
                pts = np.concatenate([_probe_points(rng, m, x, 160), centre[None, :]])
                res = G.gd_point_distance(ctx, h, x, pts)
                check_points(res, m, x, pts, oracle_mod)
        finally:
            G.gd_mesh_destroy(h)


def test_point_distance_device_io_and_edges(G, ctx, oracle_mod):
    """Device-resident points and results give the same records as host
    ones; n = 0 is a no-op; a non-finite point fails alone; the centre of a
    geodesic sphere (every face nearly equidistant, the concentric-sphere
    case of Section 10) is still exact."""
    import torch
    rng = np.random.default_rng(52)
    m = synth.geosphere(8, 1.0)
    h = _mesh(G, ctx, m)
    try:
        x = _rigid(rng)
        X = np.asarray(x).reshape(3, 4)
        pts = np.concatenate([_probe_points(rng, m, x, 64), X[:, 3][None, :]])  # + the centre
        host = G.gd_point_distance(ctx, h, x, pts)
        check_points(host, m, x, pts, oracle_mod)
        raw = G.gd_point_distance(ctx, h, x, torch.from_numpy(pts).cuda())
        dev = G.gd_point_records(raw.cpu().numpy())
        for f in ("d", "tri", "p", "status"):
            assert np.array_equal(dev[f], host[f])
        st = G.gd_point_stats(ctx)
        assert st["node_tests"] > 0 and st["exact_tests"] >= len(pts)
        assert len(G.gd_point_distance(ctx, h, x, np.zeros((0, 3)))) == 0
        bad = pts[:4].copy()
        bad[2, 1] = np.nan
        r = G.gd_point_distance(ctx, h, x, bad)
        assert list(r["status"]) == [0, 0, G.GD_ERR_INVALID_ARG, 0]
        assert np.array_equal(r["d"][[0, 1, 3]], host["d"][[0, 1, 3]])
    finally:
        G.gd_mesh_destroy(h)


# ------------------------------------------------------------------ naive comparator

def test_naive_comparator_matches_oracle(G, ctx, oracle_mod):
    """The naive per-triangle DFS (Section 8's GPU comparator) finds the same
    extreme in float32: within a float32 error budget of the oracle's value.
    A walk tests each node of B at most once."""
    rng = np.random.default_rng(41)
    pairs = [
        (synth.torus(1.0, 0.3, 24, 16), synth.torus(0.9, 0.2, 20, 14)),
        (synth.geosphere(6, 0.8, 2e-3, 1), synth.gear(96, 3, teeth=12, seed=2)),
        (_soup(rng, 1), _soup(rng, 5)),
    ]
    for A, B in pairs:
        ma, mb = _mesh(G, ctx, A), _mesh(G, ctx, B)
        LB, _ = G.gd_mesh_info(mb)
        try:
            for k in range(3):
                xa = _rigid(rng)
                xb = synth.compose(synth.xform(np.eye(3), rng.normal(size=3) * (0.5 + k)), xa)
                xb = synth.compose(xb, synth.xform(synth.random_rotation(rng), (0, 0, 0)))
                diag = oracle_mod.diag(A, xa, B, xb)
                scale = diag + float(np.abs(np.asarray(xa)[[3, 7, 11]]).max() + np.abs(np.asarray(xb)[[3, 7, 11]]).max())
                for kind, gk in (("min", G.GD_MIN), ("max", G.GD_MAX)):
                    ref = oracle_mod.brute(A, xa, B, xb, kind)
                    r = G.gd_naive_query(ctx, ma, mb, gk, xa, xb)
                    assert r["status"] == 0
                    assert abs(r["d"] - ref.d) <= 2e-6 * scale, (kind, r["d"], ref.d)
                    assert r["leaf_tests"] >= 1
                    assert 1 <= r["max_thread_tests"] <= min(r["node_tests"], (2 << LB) - 1)
        finally:
            G.gd_mesh_destroy(ma)
            G.gd_mesh_destroy(mb)


def test_naive_comparator_deadline(G, ctx, oracle_mod):
    """A deadline far shorter than the walk stops every thread; the call
    reports the timeout with partial counts and the context stays usable."""
    A = synth.torus(1.0, 0.3, 200, 100)
    ma = _mesh(G, ctx, A)
    I = synth.identity_xform()
    near = synth.xform(np.eye(3), (0.2, 0.0, 0.0))
    try:
        r = G.gd_naive_query(ctx, ma, ma, G.GD_MIN, I, near, timeout_ns=1)
        assert r["status"] == G.GD_ERR_TIMEOUT
        full = G.gd_naive_query(ctx, ma, ma, G.GD_MIN, I, near)
        assert full["status"] == 0 and full["node_tests"] > r["node_tests"]
        ok = G.gd_min_distance(ctx, ma, ma, I, near)
        assert ok.status == 0 and abs(ok.d - full["d"]) <= 1e-5
    finally:
        G.gd_mesh_destroy(ma)


def test_one_to_many_batch(G, ctx, oracle_mod):
    """1-to-N (Section 10): one mesh against N meshes of different kinds and
    sizes in one batch; every answer matches the oracle, and so does the
    nearest (farthest) of the N."""
    rng = np.random.default_rng(61)
    A = synth.torus(1.0, 0.3, 20, 12)
    others = [synth.geosphere(4 + i % 4, 0.5 + 0.1 * i, 1e-3, i) if i % 3 == 0 else
              synth.gear(64 + 16 * i, 2, teeth=8, seed=i) if i % 3 == 1 else
              _soup(rng, 40 + 20 * i, 0.6) for i in range(9)]
    ma = _mesh(G, ctx, A)
    hs = [_mesh(G, ctx, m) for m in others]
    try:
        xa = _rigid(rng, 0.1)
        for kind, gk in (("min", G.GD_MIN), ("max", G.GD_MAX)):
            xbs = [synth.compose(synth.xform(np.eye(3), rng.normal(size=3) * 2.0),
                                 synth.xform(synth.random_rotation(rng), (0, 0, 0))) for _ in others]
            out = G.gd_batch_query(ctx, [(ma, h, xa, xb, gk) for h, xb in zip(hs, xbs)])
            refs = []
            for i, (m, xb) in enumerate(zip(others, xbs)):
                ref = oracle_mod.brute(A, xa, m, xb, kind)
                check(out[i], A, xa, m, xb, kind, ref, oracle_mod.diag(A, xa, m, xb), oracle_mod)
                refs.append(ref.d)
            best = min if kind == "min" else max
            assert best(r.d for r in out) == pytest.approx(best(refs), rel=1e-12, abs=1e-15)
    finally:
        G.gd_mesh_destroy(ma)
        for h in hs:
            G.gd_mesh_destroy(h)


def test_concentric_shells_min_max(G, ctx, oracle_mod):
    """Two concentric geodesic spheres (the case Section 10 names as hard for
    culling: every triangle of the inner one sits at nearly one distance from
    the outer one), min and max against the oracle."""
    outer = synth.geosphere(20, 1.0)
    inner = synth.geosphere(14, 0.7)
    rng = np.random.default_rng(62)
    R = synth.random_rotation(rng)
    c = rng.normal(size=3)
    run_pair(G, ctx, oracle_mod, outer, inner, [(synth.xform(np.eye(3), c), synth.xform(R, c))])


# ------------------------------------------------------------------ full-size workloads

def test_rings_full_size_frames(G, ctx, oracle_mod):
    """Two 7.5 M-triangle interlinked rings, the measured workload: sampled
    frames against the oracle's float64 BVH traversal."""
    A, B, xa, xbs = synth.config_rings(frames=100)
    run_pair(G, ctx, oracle_mod, A, B, [(xa, xbs[i]) for i in (0, 37, 99)], kinds=("min",), bvh_oracle=True)


def test_rings_full_size_full_refit(G, oracle_mod):
    """The paper's per-frame refit (refit mode 3) at full size: B's 2^22-leaf
    tree refit into A's frame in three passes (subtrees of 2^8 leaves, then
    8 and 6 levels above them) before the traversal; min and max of two
    frames against the oracle's float64 BVH traversal."""
    c = G.gd_ctx_create(0)
    try:
        G.gd_ctx_set_tunables(c, refit_mode=3)
        A, B, xa, xbs = synth.config_rings(frames=100)
        run_pair(G, c, oracle_mod, A, B, [(xa, xbs[i]) for i in (5, 61)], kinds=("min", "max"), bvh_oracle=True)
    finally:
        G.gd_ctx_destroy(c)


def test_gears_full_size_batch_sample(G, ctx, oracle_mod):
    """The 4,096-transform gear workload at full size (204,800 triangles per
    gear): 16 transforms spread over the set (4 of them intersecting), in one
    batch as `bench.py` runs them, against the oracle's float64 BVH traversal."""
    A, B, xa, xbs = synth.config_gears(4096)
    idx = [256 * i + 7 for i in range(16)]
    ma, mb = _mesh(G, ctx, A), _mesh(G, ctx, B)
    try:
        out = G.gd_batch_query(ctx, [(ma, mb, xa, xbs[i], G.GD_MIN) for i in idx])
        refs = oracle_mod.bvh_query_batch(oracle_mod.Bvh(A), xa, oracle_mod.Bvh(B), [xbs[i] for i in idx], "min")
        assert sum(1 for r in refs if r.d == 0.0) == 4
        for k, i in enumerate(idx):
            check(out[k], A, xa, B, xbs[i], "min", refs[k], oracle_mod.diag(A, xa, B, xbs[i]), oracle_mod)
    finally:
        G.gd_mesh_destroy(ma)
        G.gd_mesh_destroy(mb)


def test_gears_batch_forms_and_plain_calls(G, ctx, oracle_mod):
    """64 gear transforms (min) in one batch launch: its widest levels hold
    more than twice the grid's threads at one tree level each, so they run a
    thread per front entry, and its leaf queue more than a quarter of them,
    so the leaf phase runs a thread per leaf pair.  8 of the answers against
    the oracle, and the same 8 transforms as plain single-query calls (min and
    max), whose long leaf queues take the plane axes of the cheap test."""
    A, B, xa, xbs = synth.config_gears(64)
    idx = list(range(3, 64, 8))
    ma, mb = _mesh(G, ctx, A), _mesh(G, ctx, B)
    try:
        out = G.gd_batch_query(ctx, [(ma, mb, xa, xb, G.GD_MIN) for xb in xbs])
        st = G.gd_get_stats(ctx)
        threads = st["blocks"] * 256
        assert any(f > 2 * threads and sl == 2 for f, sl in zip(st["front"], st["slots"])), st["front"]
        assert 4 * st["leaf_pairs"] > threads, st["leaf_pairs"]
        bA, bB = oracle_mod.Bvh(A), oracle_mod.Bvh(B)
        for kind, fn in (("min", G.gd_min_distance), ("max", G.gd_max_distance)):
            refs = oracle_mod.bvh_query_batch(bA, xa, bB, [xbs[i] for i in idx], kind)
            for k, i in enumerate(idx):
                diag = oracle_mod.diag(A, xa, B, xbs[i])
                if kind == "min":
                    check(out[i], A, xa, B, xbs[i], kind, refs[k], diag, oracle_mod)
                check(fn(ctx, ma, mb, xa, xbs[i]), A, xa, B, xbs[i], kind, refs[k], diag, oracle_mod)
    finally:
        G.gd_mesh_destroy(ma)
        G.gd_mesh_destroy(mb)


def test_icospheres_full_size_min_max(G, ctx, oracle_mod):
    """Two 1.31 M-triangle noisy spheres at a gap of 1e-5 x diag, min and max."""
    A, B, xa, xb = synth.config_icospheres(level=8)
    run_pair(G, ctx, oracle_mod, A, B, [(xa, xb)], bvh_oracle=True)
