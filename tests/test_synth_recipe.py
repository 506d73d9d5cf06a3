"""The seeded synthetic inputs follow their stated recipes (no GPU).

The workloads stand in for the paper's meshes (interlinked rings, noisy
spheres, gears, a pool of mixed meshes); these tests check the generators
against the closed forms and counts they are defined by: the torus
parametrisation, the geodesic sphere's counts and radius, the gear's
triangle count, closed surfaces (every edge shared by two triangles, each
direction once), and the placement of the rings, tori and spheres.
"""
import math

import numpy as np

from paper_2411_11244_gb300 import synth


def _closed_oriented(tris):
    """Every undirected edge in exactly two triangles, each directed edge once."""
    t = np.asarray(tris, dtype=np.int64)
    d = np.concatenate([t[:, [0, 1]], t[:, [1, 2]], t[:, [2, 0]]])
    directed = set(map(tuple, d.tolist()))
    if len(directed) != len(d):
        return False
    return all((b, a) in directed for a, b in directed)


def test_torus_parametrisation_and_surface():
    R, r, nu, nv = 1.0, 0.3, 24, 10
    v, t = synth.torus(R, r, nu, nv)
    assert v.dtype == np.float32 and t.dtype == np.int32
    assert v.shape == (nu * nv, 3) and t.shape == (2 * nu * nv, 3)
    for i, j in ((0, 0), (5, 3), (23, 9), (12, 7)):
        u, w = 2 * math.pi * i / nu, 2 * math.pi * j / nv
        ref = np.float32([(R + r * math.cos(w)) * math.cos(u), (R + r * math.cos(w)) * math.sin(u), r * math.sin(w)])
        assert np.array_equal(v[i * nv + j], ref)
    assert _closed_oriented(t)


def test_geosphere_counts_radius_and_surface():
    for f in (1, 2, 4):
        v, t = synth.geosphere(f, 0.7)
        assert len(t) == 20 * f * f and len(v) == 10 * f * f + 2
        assert np.allclose(np.linalg.norm(v.astype(np.float64), axis=1), 0.7, rtol=2e-7, atol=0)
        assert _closed_oriented(t)
    # noise moves vertices radially only
    v0, _ = synth.geosphere(4, 1.0)
    v1, _ = synth.geosphere(4, 1.0, noise=1e-3, seed=3)
    a = v0.astype(np.float64) / np.linalg.norm(v0, axis=1, keepdims=True)
    b = v1.astype(np.float64) / np.linalg.norm(v1.astype(np.float64), axis=1, keepdims=True)
    assert np.max(np.abs(a - b)) < 1e-6


def test_gear_count_and_surface():
    v, t = synth.gear(M=256, K=3, teeth=16)
    assert len(t) == 4 * 256 * 3 + 4 * 256
    assert _closed_oriented(t)
    # the workload's gear: 4 M K + 4 M = 204,800 triangles
    v, t = synth.gear()
    assert len(t) == 204800
    rad = np.linalg.norm(v[:, :2].astype(np.float64), axis=1)
    assert abs(rad.min() - 0.4) < 1e-6 and 0.9 < rad.max() < 1.0 + 0.01 * 0.1 * 4


def test_rings_placement():
    A, B, xa, xbs = synth.config_rings(frames=5, nu=40, nv=12)
    assert np.array_equal(xa, synth.identity_xform())
    c = 2 * 0.05 + synth.RING_GAP
    for x in xbs:
        x = np.asarray(x, dtype=np.float64).reshape(3, 4)
        Rm, t = x[:, :3], x[:, 3]
        assert np.allclose(Rm @ Rm.T, np.eye(3), atol=1e-12) and abs(np.linalg.det(Rm) - 1) < 1e-12
        assert np.allclose(t, (c, 0, 0))
        # B's symmetry axis (local z) lies along world y: B is in the xz-plane
        assert np.allclose(np.abs(Rm @ (0, 0, 1)), (0, 1, 0), atol=1e-12)


def test_tori_and_spheres_placement():
    A, B, xa, xb = synth.config_tori(3)
    assert len(A[1]) == 2048 and len(B[1]) == 2048
    assert np.allclose(np.asarray(xb).reshape(3, 4)[:, 3], (2.5, 0, 0))
    A, B, xa, xb = synth.config_icospheres(level=2, seed=1)
    shift = np.asarray(xb).reshape(3, 4)[0, 3]
    va, vb = A[0].astype(np.float64), B[0].astype(np.float64) + (shift, 0, 0)
    diag = np.linalg.norm(np.maximum(va.max(0), vb.max(0)) - np.minimum(va.min(0), vb.min(0)))
    assert abs((vb[:, 0].min() - va[:, 0].max()) - 1e-5 * diag) < 1e-9
