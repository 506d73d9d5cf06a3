"""Seeded synthetic inputs: triangle meshes and rigid transforms.

This module is shared by the tests, the benchmark and the oracle checks.  It
holds geometry generators only (tessellated tori, geodesic spheres, extruded
gears, boxes, grids, random rotations); none of the distance method's
arithmetic lives here.  Every generator works in float64 and rounds the
vertices to float32 at the end, so the float32 arrays are the exact input that
both the CUDA path and the FP64 oracle consume.

Workload shapes follow the paper's benchmarks (Section 8 of the paper lists
Rings, Balls, Tools, ...): the paper's meshes are not public here, so these
procedural stand-ins reproduce their sizes and proximity structure.

Transforms are float64 arrays of 12 values, a row-major 3x4 matrix [R | t],
mapping a mesh's local coordinates x to world coordinates R x + t.
"""

from __future__ import annotations

import math

import numpy as np

__all__ = [
    "torus", "geosphere", "gear", "box", "grid", "random_rotation",
    "xform", "compose", "identity_xform", "rot_axis",
    "config_tori", "config_rings", "config_icospheres", "config_gears",
    "mesh_pool", "warp", "config_deforming_rings",
]


# --------------------------------------------------------------------------
# transforms


def identity_xform() -> np.ndarray:
    return xform(np.eye(3), np.zeros(3))


def xform(R, t) -> np.ndarray:
    """Pack a rotation matrix and a translation into the 12-value [R|t] layout."""
    R = np.asarray(R, dtype=np.float64).reshape(3, 3)
    t = np.asarray(t, dtype=np.float64).reshape(3)
    return np.concatenate([R, t[:, None]], axis=1).reshape(12).copy()


def compose(x2, x1) -> np.ndarray:
    """Transform that applies x1 first, then x2."""
    a = np.asarray(x2, dtype=np.float64).reshape(3, 4)
    b = np.asarray(x1, dtype=np.float64).reshape(3, 4)
    R = a[:, :3] @ b[:, :3]
    t = a[:, :3] @ b[:, 3] + a[:, 3]
    return xform(R, t)


def rot_axis(axis, angle) -> np.ndarray:
    """Rotation matrix about a unit axis (Rodrigues' formula)."""
    k = np.asarray(axis, dtype=np.float64)
    k = k / np.linalg.norm(k)
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * (K @ K)


def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniformly distributed rotation (Shoemake's unit-quaternion sampling)."""
    u1, u2, u3 = rng.random(3)
    a = math.sqrt(1 - u1)
    b = math.sqrt(u1)
    x, y = a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2)
    z, w = b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3)
    return np.array([
        [1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
        [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
        [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)],
    ])


# --------------------------------------------------------------------------
# meshes


def _f32(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64).astype(np.float32))


def _i32(t):
    return np.ascontiguousarray(np.asarray(t, dtype=np.int64).astype(np.int32))


def torus(R: float, r: float, nu: int, nv: int):
    """Torus in the local xy-plane around the z axis: nu x nv quads, 2*nu*nv triangles.

    Vertex (i, j) sits at ((R + r cos v) cos u, (R + r cos v) sin u, r sin v) with
    u = 2 pi i / nu and v = 2 pi j / nv; each quad is split on a fixed diagonal.
    """
    i = np.arange(nu, dtype=np.float64)[:, None]
    j = np.arange(nv, dtype=np.float64)[None, :]
    u = 2 * np.pi * i / nu
    v = 2 * np.pi * j / nv
    x = (R + r * np.cos(v)) * np.cos(u)
    y = (R + r * np.cos(v)) * np.sin(u)
    z = r * np.sin(v) * np.ones_like(u)
    verts = np.stack([x, y, z], axis=-1).reshape(-1, 3)
    ii = np.arange(nu)[:, None]
    jj = np.arange(nv)[None, :]
    a = ii * nv + jj
    b = ((ii + 1) % nu) * nv + jj
    c = ((ii + 1) % nu) * nv + (jj + 1) % nv
    d = ii * nv + (jj + 1) % nv
    t1 = np.stack([a, b, c], axis=-1).reshape(-1, 3)
    t2 = np.stack([a, c, d], axis=-1).reshape(-1, 3)
    tris = np.stack([t1, t2], axis=1).reshape(-1, 3)
    return _f32(verts), _i32(tris)


_ICO_F = [
    (0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
    (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
    (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
    (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1),
]


def _icosahedron():
    p = (1 + math.sqrt(5)) / 2
    v = np.array([
        (-1, p, 0), (1, p, 0), (-1, -p, 0), (1, -p, 0),
        (0, -1, p), (0, 1, p), (0, -1, -p), (0, 1, -p),
        (p, 0, -1), (p, 0, 1), (-p, 0, -1), (-p, 0, 1),
    ], dtype=np.float64)
    return v / np.linalg.norm(v, axis=1, keepdims=True), np.array(_ICO_F, dtype=np.int64)


def geosphere(freq: int, radius: float = 1.0, noise: float = 0.0, seed: int = 0,
              center=(0.0, 0.0, 0.0)):
    """Class-I geodesic sphere: each icosahedron face split into freq^2 triangles.

    20 * freq^2 triangles and 10 * freq^2 + 2 vertices; freq = 2^s gives the
    counts of an s-times subdivided icosphere (s = 8: 1,310,720 triangles).
    Vertices are projected to the sphere, then moved radially by N(0, noise).
    """
    n = int(freq)
    assert n >= 1
    cv, cf = _icosahedron()
    # canonical edges (lo, hi) -> id, so that faces sharing an edge share its points
    edges = {}
    for f in cf:
        for k in range(3):
            a, b = int(f[k]), int(f[(k + 1) % 3])
            key = (min(a, b), max(a, b))
            if key not in edges:
                edges[key] = len(edges)
    ne = len(edges)
    nv_edge = n - 1
    nv_face = (n - 1) * (n - 2) // 2
    V = 12 + ne * nv_edge + 20 * nv_face
    pts = np.zeros((V, 3), dtype=np.float64)
    pts[:12] = cv
    s_ = np.arange(1, n, dtype=np.float64)[:, None] / n
    for (a, b), e in edges.items():
        pts[12 + e * nv_edge: 12 + (e + 1) * nv_edge] = cv[a] * (1 - s_) + cv[b] * s_
    face_base = 12 + ne * nv_edge
    # grid (i, j), i + j <= n: point = A + i/n (B - A) + j/n (C - A)
    I, J = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    inner = (I > 0) & (J > 0) & (I + J < n)
    ii_in, jj_in = I[inner], J[inner]  # row-major order of interior points
    tris = []
    for fi, (A, B, C) in enumerate(cf):
        A, B, C = int(A), int(B), int(C)
        idx = -np.ones((n + 1, n + 1), dtype=np.int64)

        def edge_run(a, b, k):
            # points k (1..n-1) from a toward b on the canonical edge
            e = edges[(min(a, b), max(a, b))]
            kk = k if a < b else n - k
            return 12 + e * nv_edge + (kk - 1)

        k = np.arange(1, n)
        idx[0, 0], idx[n, 0], idx[0, n] = A, B, C
        if n > 1:
            idx[k, 0] = edge_run(A, B, k)
            idx[0, k] = edge_run(A, C, k)
            idx[n - k, k] = edge_run(B, C, k)
        base = face_base + fi * nv_face
        idx[ii_in, jj_in] = base + np.arange(len(ii_in))
        pts[base: base + len(ii_in)] = (cv[A][None, :] + (ii_in[:, None] / n) * (cv[B] - cv[A])[None, :]
                                        + (jj_in[:, None] / n) * (cv[C] - cv[A])[None, :])
        ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        m = ii + jj <= n - 1
        i0, j0 = ii[m], jj[m]
        tris.append(np.stack([idx[i0, j0], idx[i0 + 1, j0], idx[i0, j0 + 1]], axis=1))
        m2 = ii + jj <= n - 2
        i1, j1 = ii[m2], jj[m2]
        tris.append(np.stack([idx[i1 + 1, j1], idx[i1 + 1, j1 + 1], idx[i1, j1 + 1]], axis=1))
    tris = np.concatenate(tris, axis=0)
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    rad = np.full(V, float(radius))
    if noise > 0:
        rad = rad + np.random.default_rng(seed).normal(0.0, noise, size=V)
    pts = pts * rad[:, None] + np.asarray(center, dtype=np.float64)[None, :]
    return _f32(pts), _i32(tris)


def gear(M: int = 2048, K: int = 24, teeth: int = 64, seed: int = 0,
         r_root: float = 0.9, tooth_h: float = 0.1, r_in: float = 0.4,
         thick: float = 0.2, noise_frac: float = 0.01, cap_rings: int = 1):
    """Annular gear extruded along z: 4*M*K + 4*M*cap_rings triangles.

    The outer profile has M points (M / teeth per tooth, trapezoidal teeth of
    height tooth_h, radial noise of noise_frac * tooth_h), the inner wall is a
    circle of M points, K layers of quads on both walls, and two annular caps
    of cap_rings rings of quads each (1: one quad from the outer profile
    straight to the inner circle).
    """
    rng = np.random.default_rng(seed)
    th = 2 * np.pi * np.arange(M) / M
    per = M // teeth
    ph = (np.arange(M) % per) / per
    prof = np.clip(np.minimum((ph - 0.0) / 0.125, (0.625 - ph) / 0.125), 0.0, 1.0)
    r_out = r_root + tooth_h * prof + rng.normal(0.0, noise_frac * tooth_h, size=M)
    z = np.linspace(0.0, thick, K + 1)
    outer = np.stack([
        (r_out[None, :] * np.cos(th)[None, :]) * np.ones((K + 1, 1)),
        (r_out[None, :] * np.sin(th)[None, :]) * np.ones((K + 1, 1)),
        z[:, None] * np.ones((1, M)),
    ], axis=-1).reshape(-1, 3)
    inner = np.stack([
        (r_in * np.cos(th)[None, :]) * np.ones((K + 1, 1)),
        (r_in * np.sin(th)[None, :]) * np.ones((K + 1, 1)),
        z[:, None] * np.ones((1, M)),
    ], axis=-1).reshape(-1, 3)
    verts = np.concatenate([outer, inner], axis=0)
    off_in = (K + 1) * M

    def wall(base, flip):
        k = np.arange(K)[:, None]
        m = np.arange(M)[None, :]
        a = base + k * M + m
        b = base + k * M + (m + 1) % M
        c = base + (k + 1) * M + (m + 1) % M
        d = base + (k + 1) * M + m
        if flip:
            t1, t2 = np.stack([a, c, b], -1), np.stack([a, d, c], -1)
        else:
            t1, t2 = np.stack([a, b, c], -1), np.stack([a, c, d], -1)
        return np.stack([t1.reshape(-1, 3), t2.reshape(-1, 3)], axis=1).reshape(-1, 3)

    extra = []  # intermediate cap rings (top then bottom), appended after the walls

    def ring_ids(layer, k):
        # vertex ids of ring k (0: outer profile, cap_rings: inner circle) of a cap
        if k == 0:
            return layer * M + np.arange(M)
        if k == cap_rings:
            return off_in + layer * M + np.arange(M)
        return ring_base[layer] + (k - 1) * M + np.arange(M)

    ring_base = {}
    nv = len(verts)
    for layer in (K, 0):
        ring_base[layer] = nv + sum(len(e) for e in extra)
        for k in range(1, cap_rings):
            f = k / cap_rings
            r = r_out + (r_in - r_out) * f
            extra.append(np.stack([r * np.cos(th), r * np.sin(th), np.full(M, z[layer])], axis=-1))
    if extra:
        verts = np.concatenate([verts] + extra, axis=0)

    def cap(layer, flip):
        out = []
        for k in range(cap_rings):
            o = ring_ids(layer, k)
            i = ring_ids(layer, k + 1)
            a, b = o, np.roll(o, -1)
            c, d = np.roll(i, -1), i
            if flip:
                t1, t2 = np.stack([a, c, b], -1), np.stack([a, d, c], -1)
            else:
                t1, t2 = np.stack([a, b, c], -1), np.stack([a, c, d], -1)
            out.append(np.stack([t1, t2], axis=1).reshape(-1, 3))
        return np.concatenate(out, axis=0)

    tris = np.concatenate([wall(0, False), wall(off_in, True), cap(K, False), cap(0, True)], axis=0)
    return _f32(verts), _i32(tris)


def box(lo, hi):
    """Closed axis-aligned box surface: 8 vertices, 12 triangles."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    v = np.array([[(hi if (m >> k) & 1 else lo)[k] for k in range(3)] for m in range(8)])
    f = [(0, 2, 3, 1), (4, 5, 7, 6), (0, 1, 5, 4), (2, 6, 7, 3), (0, 4, 6, 2), (1, 3, 7, 5)]
    t = []
    for a, b, c, d in f:
        t += [(a, b, c), (a, c, d)]
    return _f32(v), _i32(t)


def grid(n: int, size: float = 1.0, z: float = 0.0, x0: float = 0.0, y0: float = 0.0):
    """Flat square grid at height z: (n+1)^2 vertices, 2 n^2 triangles."""
    s = np.linspace(0.0, size, n + 1)
    X, Y = np.meshgrid(s + x0, s + y0, indexing="ij")
    v = np.stack([X, Y, np.full_like(X, z)], axis=-1).reshape(-1, 3)
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    a = i * (n + 1) + j
    b = (i + 1) * (n + 1) + j
    c = (i + 1) * (n + 1) + j + 1
    d = i * (n + 1) + j + 1
    t = np.stack([np.stack([a, b, c], -1).reshape(-1, 3), np.stack([a, c, d], -1).reshape(-1, 3)],
                 axis=1).reshape(-1, 3)
    return _f32(v), _i32(t)


# --------------------------------------------------------------------------
# workloads


def config_tori(seed: int = 0):
    """Two tori R=1, r=0.3, 32x32 quads (2,048 triangles each); B gets a seeded
    uniform rotation and an offset of 2.5 along x.  Returns (A, B, xa, xb)."""
    A = torus(1.0, 0.3, 32, 32)
    rng = np.random.default_rng(seed)
    xb = xform(random_rotation(rng), (2.5, 0.0, 0.0))
    return A, A, identity_xform(), xb


RING_GAP = 1e-3


def config_rings(frames: int = 100, seed: int = 0, nu: int = 2500, nv: int = 1500,
                 R: float = 1.0, r: float = 0.05, gap: float = RING_GAP):
    """Interlinked rings (the paper's teaser scene, Fig. 1): two tori of
    2 * nu * nv triangles (7.5 M at the default sizes).  A lies in the xy-plane
    at the origin; B lies in the xz-plane centred at (c, 0, 0) with
    c = 2 r + gap, so the core circles pass within c of each other at two
    sites and the surfaces within about `gap`.  Each frame spins B about its
    own symmetry axis by a seeded uniform angle.  Returns (A, B, xa, [xb...])."""
    A = torus(R, r, nu, nv)
    c = 2 * r + gap
    rng = np.random.default_rng(seed)
    to_xz = rot_axis((1, 0, 0), math.pi / 2)  # local z -> world -y
    xbs = []
    for _ in range(frames):
        ang = rng.uniform(0.0, 2 * math.pi)
        Rb = to_xz @ rot_axis((0, 0, 1), ang)
        xbs.append(xform(Rb, (c, 0.0, 0.0)))
    return A, A, identity_xform(), xbs


def warp(verts, amp: float, freq: float, phase: float):
    """Smooth non-rigid deformation of a vertex array (a deforming body for the
    paper's Deformable scene, Section 8): every vertex x moves by
    amp * (sin(2 pi f y + p), sin(2 pi f z + 1.3 p), sin(2 pi f x + 0.7 p)),
    at most amp * sqrt(3).  Connectivity is unchanged.  float64 arithmetic,
    rounded to float32."""
    v = np.asarray(verts, dtype=np.float64)
    w = 2.0 * math.pi * freq
    d = np.stack([np.sin(w * v[:, 1] + phase), np.sin(w * v[:, 2] + 1.3 * phase),
                  np.sin(w * v[:, 0] + 0.7 * phase)], axis=1)
    return _f32(v + amp * d)


def config_deforming_rings(frames: int = 8, seed: int = 0, nu: int = 2500, nv: int = 1500,
                           R: float = 1.0, r: float = 0.05, gap: float = RING_GAP, amp: float = 0.01):
    """The interlinked rings with a deforming B: each frame warps B's local
    vertices (warp with amplitude amp, one wave per unit length, a seeded
    phase) and spins B as in config_rings.  B's centre sits at
    c = 2 r + gap + 2 amp, so the warped surfaces stay apart (each vertex moves
    by at most amp * sqrt(3) < 2 amp).  Returns (A, tris_B, xa, [xb...],
    frame_verts) where frame_verts(i) gives B's float32 vertices of frame i."""
    A = torus(R, r, nu, nv)
    c = 2 * r + gap + 2 * amp
    rng = np.random.default_rng(seed)
    to_xz = rot_axis((1, 0, 0), math.pi / 2)
    xbs, phases = [], []
    for _ in range(frames):
        Rb = to_xz @ rot_axis((0, 0, 1), rng.uniform(0.0, 2 * math.pi))
        xbs.append(xform(Rb, (c, 0.0, 0.0)))
        phases.append(rng.uniform(0.0, 2 * math.pi))
    base = A[0]

    def frame_verts(i: int):
        return warp(base, amp, 1.0, phases[i])

    return A, A[1], identity_xform(), xbs, frame_verts


def config_icospheres(level: int = 8, seed: int = 0, noise: float = 1e-3, gap_frac: float = 1e-5):
    """Two noisy geodesic spheres of 20 * 4^level triangles, radius 1, radial
    noise N(0, noise) with seeds s and s+1.  B is shifted along +x so that the
    x-extents of the two vertex sets are separated by gap_frac times the world
    bounding-box diagonal of both meshes."""
    f = 2 ** level
    A = geosphere(f, 1.0, noise, seed)
    B = geosphere(f, 1.0, noise, seed + 1)
    va = A[0].astype(np.float64)
    vb = B[0].astype(np.float64)
    shift = va[:, 0].max() - vb[:, 0].min()
    for _ in range(3):
        lo = np.minimum(va.min(0), vb.min(0) + (shift, 0, 0))
        hi = np.maximum(va.max(0), vb.max(0) + (shift, 0, 0))
        diag = float(np.linalg.norm(hi - lo))
        shift = va[:, 0].max() - vb[:, 0].min() + gap_frac * diag
    return A, B, identity_xform(), xform(np.eye(3), (shift, 0.0, 0.0))


def config_icosphere_frames(frames: int = 100, level: int = 8, seed: int = 0, noise: float = 1e-3,
                            gap_frac: float = 1e-5):
    """The near-contact icospheres of config_icospheres as a frame sequence:
    frame 0 is that placement; frame f > 0 first spins B about its own x-axis
    by a seeded uniform angle.  The spin keeps every x-coordinate of B, so the
    x-extents stay gap_frac x diag apart while the noisy surfaces that face
    each other change from frame to frame.  Returns (A, B, xa, [xb...])."""
    A, B, xa, xb0 = config_icospheres(level, seed, noise, gap_frac)
    rng = np.random.default_rng(seed + 11)
    xbs = [xb0]
    for _ in range(frames - 1):
        xbs.append(compose(xb0, xform(rot_axis((1, 0, 0), rng.uniform(0.0, 2 * math.pi)), (0.0, 0.0, 0.0))))
    return A, B, xa, xbs


def config_gears(n: int = 4096, seed: int = 0, M: int = 2048, K: int = 24):
    """One gear pair (4*M*K + 4*M triangles each) under n seeded rigid
    transforms of B: uniform rotation, centre offset in a uniformly random
    direction at a distance uniform in [0.5, 1.5] x the outer diameter.
    Returns (A, B, xa, [xb...])."""
    A = gear(M, K, seed=seed)
    B = gear(M, K, seed=seed + 1)
    vb = B[0].astype(np.float64)
    diam = 2 * float(np.max(np.linalg.norm(vb[:, :2], axis=1)))
    rng = np.random.default_rng(seed + 2)
    xbs = []
    for _ in range(n):
        Rm = random_rotation(rng)
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        dist = rng.uniform(0.5, 1.5) * diam
        xbs.append(xform(Rm, d * dist))
    return A, B, identity_xform(), xbs


def mesh_pool(n: int = 64, seed: int = 0, tmin: float = 1e3, tmax: float = 4e6):
    """Pool of meshes of kinds {torus, geodesic sphere, gear} with triangle
    counts log-uniform in [tmin, tmax] (hit within a few percent)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n):
        kind = int(rng.integers(0, 3))
        T = float(math.exp(rng.uniform(math.log(tmin), math.log(tmax))))
        if kind == 0:
            nv = max(3, int(round(math.sqrt(T / 4))))
            nu = max(3, int(round(T / (2 * nv))))
            m = torus(1.0, 0.25, nu, nv)
        elif kind == 1:
            f = max(1, int(round(math.sqrt(T / 20))))
            m = geosphere(f, 1.0, 1e-3, seed * 1000 + k)
        else:
            # near-square cells: wall layers K ~ M (thickness / circumference),
            # cap rings ~ M (annulus width / circumference); T = 4 M K + 4 M rings
            teeth = 16
            M = max(teeth * 2, int(round(math.sqrt(T / 0.445) / teeth)) * teeth)
            Kl = max(1, int(round(0.2 * M / (2 * math.pi))))
            rings = max(1, int(round(0.5 * M / (2 * math.pi))))
            m = gear(M, Kl, teeth=teeth, seed=seed * 1000 + k, cap_rings=rings)
        out.append(m)
    return out
