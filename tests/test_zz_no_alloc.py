"""The allocation-free query gives the oracle's answers, like the allocating one.

gd_query_device_noalloc is for callers that must not allocate device memory
while they run (a per-frame control loop that cannot afford a cudaMalloc that
stalls or fails, or a process whose device memory belongs to another
allocator).  Its work buffers live in one fixed array inside the library that
every call shares and that keeps the last call's contents, so each query is
made twice in a row, and every answer is checked against the FP64 oracle
(brute force for the two tori, the oracle's BVH query for the larger rings)
and against the allocating entry point, within the parity tolerance
|d - d_ref| <= 1e-6 x diag, with the witness pair's float64 distance equal to
the reference's within 1e-12 relative (+1e-15 x diag).  The context's bounds
and refit modes must be honoured, and the documented errors and the overflow
status must come back as stated.  This file is collected last so that a run
that stops at the first failure has run everything else.
"""

import json
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2411_11244_gb300 import gdist as G
    from paper_2411_11244_gb300 import synth
    return torch, G, synth


def _dev_xforms(torch, ta, tb):
    d_xa = torch.tensor(np.asarray(ta), dtype=torch.float64, device="cuda")
    d_xb = torch.tensor(np.asarray(tb), dtype=torch.float64, device="cuda")
    return d_xa, d_xb


def _noalloc(torch, G, ma, mb, kind, d_xa, d_xb):
    out = torch.full((10,), float("nan"), dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    G.gd_query_device_noalloc(ma, mb, kind, d_xa.data_ptr(), d_xb.data_ptr(), out.data_ptr(), stream)
    torch.cuda.synchronize()
    return G.gd_result.from_buffer_copy(out.cpu().numpy().tobytes())


def _check(r, ref, MA, ta, MB, tb, name, diag, oracle_mod, what):
    assert r.status == 0, (what, r.status)
    assert abs(r.d - ref.d) <= 1e-6 * diag, (what, r.d, ref.d)
    dw, _, _ = oracle_mod.witness_distance(MA, ta, MB, tb, r.tri_a, r.tri_b, name)
    assert abs(dw - ref.d) <= 1e-12 * abs(ref.d) + 1e-15 * diag, (what, dw, ref.d)
    assert abs(r.d - dw) <= 1e-12 * abs(ref.d) + 1e-15 * diag, (what, r.d, dw)


def test_noalloc_matches_oracle_and_allocating_path_twice(env, oracle_mod):
    torch, G, synth = env
    seed = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "tori_seed.json")))["seed"]
    A, B, xa, xb = synth.config_tori(seed)
    R, _, _, xbs = synth.config_rings(frames=2, nu=400, nv=120)
    cases = [(A, B, xa, xb, False), (R, R, synth.identity_xform(), xbs[1], True)]
    ctx = G.gd_ctx_create(0)
    try:
        for MA, MB, ta, tb, use_bvh in cases:
            ma = G.gd_mesh_create(ctx, *MA)
            G.gd_bvh_build(ma, ctx=ctx)
            mb = G.gd_mesh_create(ctx, *MB)
            G.gd_bvh_build(mb, ctx=ctx)
            diag = oracle_mod.diag(MA, ta, MB, tb)
            d_xa, d_xb = _dev_xforms(torch, ta, tb)
            oa = oracle_mod.Bvh(MA) if use_bvh else None
            for kind, name, fn in ((G.GD_MIN, "min", G.gd_min_distance), (G.GD_MAX, "max", G.gd_max_distance)):
                ref = (oracle_mod.bvh_query(oa, ta, oa, tb, name) if use_bvh
                       else oracle_mod.brute(MA, ta, MB, tb, name))
                alloc = fn(ctx, ma, mb, ta, tb)
                _check(alloc, ref, MA, ta, MB, tb, name, diag, oracle_mod, "allocating")
                for call in range(2):
                    r = _noalloc(torch, G, ma, mb, kind, d_xa, d_xb)
                    _check(r, ref, MA, ta, MB, tb, name, diag, oracle_mod, ("noalloc", call))
                    assert abs(r.d - alloc.d) <= 1e-6 * diag
            G.gd_mesh_destroy(ma)
            G.gd_mesh_destroy(mb)
    finally:
        G.gd_ctx_destroy(ctx)


def test_noalloc_honours_bounds_and_refit_modes(env, oracle_mod):
    """The context's tunables reach the allocation-free launch: conventional
    bounds (Section 9's ablation) and refit off give the oracle's answers,
    and conventional bounds test more node pairs in the allocating path on
    the same queries (the allocation-free path keeps its counters inside its
    array, so the node-pair count is read from the allocating call)."""
    torch, G, synth = env
    rng = np.random.default_rng(61)
    A = synth.torus(1.0, 0.1, 96, 40)
    B = synth.geosphere(12, 0.5, 1e-3, 3)
    ctx = G.gd_ctx_create(0)
    try:
        ma = G.gd_mesh_create(ctx, *A)
        G.gd_bvh_build(ma, ctx=ctx)
        mb = G.gd_mesh_create(ctx, *B)
        G.gd_bvh_build(mb, ctx=ctx)
        oa, ob = oracle_mod.Bvh(A), oracle_mod.Bvh(B)
        for i in range(3):
            ta = synth.xform(synth.random_rotation(rng), rng.normal(size=3) * 0.3)
            tb = synth.xform(synth.random_rotation(rng), rng.normal(size=3) * 1.5)
            diag = oracle_mod.diag(A, ta, B, tb)
            d_xa, d_xb = _dev_xforms(torch, ta, tb)
            for kind, name in ((G.GD_MIN, "min"), (G.GD_MAX, "max")):
                ref = oracle_mod.bvh_query(oa, ta, ob, tb, name)
                for tun in ({"bounds_mode": 2, "refit_mode": 1}, {"bounds_mode": 1, "refit_mode": 2},
                            {"bounds_mode": 2, "refit_mode": 2}):
                    G.gd_ctx_set_tunables(ctx, **tun)
                    r = _noalloc(torch, G, ma, mb, kind, d_xa, d_xb)
                    _check(r, ref, A, ta, B, tb, name, diag, oracle_mod, ("noalloc", tun))
        G.gd_ctx_set_tunables(ctx, bounds_mode=1, refit_mode=1)
        G.gd_mesh_destroy(ma)
        G.gd_mesh_destroy(mb)
    finally:
        G.gd_ctx_destroy(ctx)


def test_noalloc_errors_and_overflow_status(env, oracle_mod):
    """The documented errors: a mesh without a tree (GD_ERR_NOT_BUILT), meshes
    of two contexts and a bad kind (GD_ERR_INVALID_ARG).  And two parallel
    grids at a tiny gap, where some 10^5 triangle pairs tie at the minimum:
    more candidates than the array's 2^16, so the status is GD_ERR_OVERFLOW
    (with the distance withheld), never a wrong distance."""
    torch, G, synth = env
    I = synth.identity_xform()
    d_xa, d_xb = _dev_xforms(torch, I, I)
    c1, c2 = G.gd_ctx_create(0), G.gd_ctx_create(0)
    try:
        T = synth.torus(1.0, 0.3, 16, 12)
        m1 = G.gd_mesh_create(c1, *T)
        G.gd_bvh_build(m1, ctx=c1)
        m2 = G.gd_mesh_create(c2, *T)
        G.gd_bvh_build(m2, ctx=c2)
        raw = G.gd_mesh_create(c1, *T)  # no tree
        out = torch.zeros(10, dtype=torch.float64, device="cuda")
        for args, want in (((m1, raw, G.GD_MIN), G.GD_ERR_NOT_BUILT), ((m1, m2, G.GD_MIN), G.GD_ERR_INVALID_ARG),
                           ((m1, m1, 7), G.GD_ERR_INVALID_ARG)):
            with pytest.raises(G.GdError) as e:
                G.gd_query_device_noalloc(*args, d_xa.data_ptr(), d_xb.data_ptr(), out.data_ptr(), 0)
            assert e.value.status == want, (args, e.value.status)
        # a valid call still works after the refusals
        r = _noalloc(torch, G, m1, m1, G.GD_MAX, d_xa, d_xb)
        ref = oracle_mod.brute(T, I, T, I, "max")
        assert r.status == 0 and abs(r.d - ref.d) <= 1e-6 * oracle_mod.diag(T, I, T, I)
        # overflow: 2 x 131,072 triangles in parallel planes 2^-12 apart
        GA = synth.grid(256, 1.0, 0.0)
        GB = synth.grid(256, 1.0, 2.0 ** -12, x0=0.3 / 256, y0=0.7 / 256)
        ga = G.gd_mesh_create(c1, *GA)
        G.gd_bvh_build(ga, ctx=c1)
        gb = G.gd_mesh_create(c1, *GB)
        G.gd_bvh_build(gb, ctx=c1)
        r = _noalloc(torch, G, ga, gb, G.GD_MIN, d_xa, d_xb)
        assert r.status == G.GD_ERR_OVERFLOW, r.status
        assert np.isnan(r.d)
        # the allocating path grows its buffers and answers the same query
        ok = G.gd_min_distance(c1, ga, gb, I, I)
        assert ok.status == 0 and ok.d == pytest.approx(float(np.float32(2.0 ** -12)), rel=1e-12)
        for m in (m1, raw, ga, gb):
            G.gd_mesh_destroy(m)
        G.gd_mesh_destroy(m2)
    finally:
        G.gd_ctx_destroy(c1)
        G.gd_ctx_destroy(c2)
