"""FP64 CPU oracle for mesh-mesh min/max distance -- test infrastructure only.

Only `tests/`, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import this package.  It wraps `gd_oracle.c` (plain C, float64,
see that file's header for the definitions it follows: Section 3, Eqs. 1-2 of
the paper) through ctypes and shares nothing with the CUDA engine.

`bounds.py` next to this file restates the paper's AABB distance bounds
(Section 4, Eqs. 3-11) in numpy for the bound property tests.
"""

from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gd_oracle.c")
_LIB = os.path.join(_HERE, "_build", "liboracle.so")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction, so x86 and Arm agree)."""
    os.makedirs(os.path.dirname(_LIB), exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
            "-pthread", "-o", tmp, _SRC, "-lm",
        ])
        os.replace(tmp, _LIB)
    return _LIB


class Result(C.Structure):
    _fields_ = [("d", C.c_double), ("ta", C.c_int64), ("tb", C.c_int64),
                ("pa", C.c_double * 3), ("pb", C.c_double * 3)]


_dp = C.POINTER(C.c_double)
_fp = C.POINTER(C.c_float)
_ip = C.POINTER(C.c_int32)


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        for name in ("or_point_segment",):
            getattr(L, name).argtypes = [_dp, _dp, _dp, _dp]
        L.or_point_segment.restype = C.c_double
        L.or_point_triangle.argtypes = [_dp, _dp, _dp, _dp, _dp]
        L.or_point_triangle.restype = C.c_double
        L.or_segment_segment.argtypes = [_dp, _dp, _dp, _dp, _dp, _dp]
        L.or_segment_segment.restype = C.c_double
        L.or_tri_tri.argtypes = [_dp, _dp, _dp, _dp]
        L.or_tri_tri.restype = C.c_double
        L.or_tri_tri_max.argtypes = [_dp, _dp, _dp, _dp]
        L.or_tri_tri_max.restype = C.c_double
        L.or_brute.argtypes = [_fp, C.c_int64, _ip, C.c_int64, _dp, _fp, C.c_int64, _ip, C.c_int64, _dp,
                               C.c_int, C.c_int, C.POINTER(Result)]
        L.or_brute.restype = C.c_int
        L.or_bvh_build.argtypes = [_fp, C.c_int64, _ip, C.c_int64]
        L.or_bvh_build.restype = C.c_void_p
        L.or_bvh_free.argtypes = [C.c_void_p]
        L.or_bvh_free.restype = None
        L.or_bvh_nodes.argtypes = [C.c_void_p]
        L.or_bvh_nodes.restype = C.c_int32
        L.or_bvh_query.argtypes = [C.c_void_p, _dp, C.c_void_p, _dp, C.c_int, C.POINTER(Result),
                                   C.POINTER(C.c_int64)]
        L.or_bvh_query.restype = C.c_int
        L.or_bvh_query_batch.argtypes = [C.c_void_p, _dp, C.c_void_p, _dp, C.c_int64, C.c_int, C.c_int,
                                         C.POINTER(Result)]
        L.or_bvh_query_batch.restype = C.c_int
        L.or_tri_pair_world.argtypes = [_fp, _dp, _fp, _dp, C.c_int, _dp, _dp]
        L.or_tri_pair_world.restype = C.c_double
        L.or_point_mesh.argtypes = [_fp, C.c_int64, _ip, C.c_int64, _dp, _dp, C.c_int64, C.c_int, _dp,
                                    C.POINTER(C.c_int64), _dp]
        L.or_point_mesh.restype = C.c_int
        _lib = L
    return _lib


def _d(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if n is not None:
        assert a.size == n, (a.shape, n)
    return a


def _ptr(a, t):
    return a.ctypes.data_as(t)


@dataclass
class Answer:
    d: float
    ta: int
    tb: int
    pa: np.ndarray
    pb: np.ndarray


def _ans(r: Result) -> Answer:
    return Answer(r.d, int(r.ta), int(r.tb), np.array(r.pa[:]), np.array(r.pb[:]))


# ---------------------------------------------------------------- primitives

def point_segment(p, a, b):
    p, a, b = _d(p, 3), _d(a, 3), _d(b, 3)
    q = np.zeros(3)
    d = lib().or_point_segment(_ptr(p, _dp), _ptr(a, _dp), _ptr(b, _dp), _ptr(q, _dp))
    return d, q


def point_triangle(p, a, b, c):
    p, a, b, c = _d(p, 3), _d(a, 3), _d(b, 3), _d(c, 3)
    q = np.zeros(3)
    d = lib().or_point_triangle(_ptr(p, _dp), _ptr(a, _dp), _ptr(b, _dp), _ptr(c, _dp), _ptr(q, _dp))
    return d, q


def segment_segment(p0, p1, q0, q1):
    p0, p1, q0, q1 = _d(p0, 3), _d(p1, 3), _d(q0, 3), _d(q1, 3)
    cp, cq = np.zeros(3), np.zeros(3)
    d = lib().or_segment_segment(_ptr(p0, _dp), _ptr(p1, _dp), _ptr(q0, _dp), _ptr(q1, _dp),
                                 _ptr(cp, _dp), _ptr(cq, _dp))
    return d, cp, cq


def tri_tri(A, B):
    """Distance between closed triangles (3x3 arrays of vertices)."""
    A, B = _d(A, 9), _d(B, 9)
    pa, pb = np.zeros(3), np.zeros(3)
    d = lib().or_tri_tri(_ptr(A, _dp), _ptr(B, _dp), _ptr(pa, _dp), _ptr(pb, _dp))
    return d, pa, pb


def tri_tri_max(A, B):
    A, B = _d(A, 9), _d(B, 9)
    pa, pb = np.zeros(3), np.zeros(3)
    d = lib().or_tri_tri_max(_ptr(A, _dp), _ptr(B, _dp), _ptr(pa, _dp), _ptr(pb, _dp))
    return d, pa, pb


# ---------------------------------------------------------------- meshes

def _mesh(m):
    v, t = m
    v = np.ascontiguousarray(np.asarray(v, dtype=np.float32))
    t = np.ascontiguousarray(np.asarray(t, dtype=np.int32))
    return v, t


def brute(A, xa, B, xb, kind: str = "min", threads: int | None = None) -> Answer:
    """All-pairs triangle distance, float64 (kind 'min' or 'max')."""
    (va, ta), (vb, tb) = _mesh(A), _mesh(B)
    xa, xb = _d(xa, 12), _d(xb, 12)
    r = Result()
    rc = lib().or_brute(_ptr(va, _fp), len(va), _ptr(ta, _ip), len(ta), _ptr(xa, _dp),
                        _ptr(vb, _fp), len(vb), _ptr(tb, _ip), len(tb), _ptr(xb, _dp),
                        1 if kind == "max" else 0, int(threads or os.cpu_count() or 1), C.byref(r))
    if rc:
        raise RuntimeError(f"oracle brute force failed ({rc})")
    return _ans(r)


class Bvh:
    """The oracle's own float64 median-split AABB tree over one mesh (local frame)."""

    def __init__(self, mesh):
        self.v, self.t = _mesh(mesh)
        self.h = lib().or_bvh_build(_ptr(self.v, _fp), len(self.v), _ptr(self.t, _ip), len(self.t))
        if not self.h:
            raise RuntimeError("oracle BVH build failed")

    @property
    def nodes(self) -> int:
        return lib().or_bvh_nodes(self.h)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_bvh_free(self.h)
            self.h = None


def bvh_query(A: Bvh, xa, B: Bvh, xb, kind: str = "min", with_visits: bool = False):
    xa, xb = _d(xa, 12), _d(xb, 12)
    r = Result()
    nv = C.c_int64(0)
    rc = lib().or_bvh_query(A.h, _ptr(xa, _dp), B.h, _ptr(xb, _dp), 1 if kind == "max" else 0,
                            C.byref(r), C.byref(nv))
    if rc:
        raise RuntimeError(f"oracle BVH query failed ({rc})")
    return (_ans(r), nv.value) if with_visits else _ans(r)


def bvh_query_batch(A: Bvh, xa, B: Bvh, xbs, kind: str = "min", threads: int | None = None):
    """Many queries of the same mesh pair; xa may be one transform or one per query."""
    xbs = np.ascontiguousarray(np.asarray(xbs, dtype=np.float64).reshape(-1, 12))
    n = len(xbs)
    xa = np.asarray(xa, dtype=np.float64).reshape(-1, 12)
    if len(xa) == 1:
        xa = np.repeat(xa, n, axis=0)
    xa = np.ascontiguousarray(xa)
    out = (Result * n)()
    rc = lib().or_bvh_query_batch(A.h, _ptr(xa, _dp), B.h, _ptr(xbs, _dp), n, 1 if kind == "max" else 0,
                                  int(threads or os.cpu_count() or 1), out)
    if rc:
        raise RuntimeError(f"oracle batch query failed ({rc})")
    return [_ans(out[i]) for i in range(n)]


def point_mesh(mesh, x, points, threads: int | None = None):
    """Distance from each world point to the mesh placed by x (Eq. 1 with one
    side a single point), brute force: (d[n], tri[n], closest[n, 3])."""
    v, t = _mesh(mesh)
    x = _d(x, 12)
    P = np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, 3))
    n = len(P)
    d = np.zeros(n)
    tri = np.zeros(n, dtype=np.int64)
    q = np.zeros((n, 3))
    rc = lib().or_point_mesh(_ptr(v, _fp), len(v), _ptr(t, _ip), len(t), _ptr(x, _dp), _ptr(P, _dp), n,
                             threads or os.cpu_count() or 1, _ptr(d, _dp),
                             tri.ctypes.data_as(C.POINTER(C.c_int64)), _ptr(q, _dp))
    if rc != 0:
        raise RuntimeError(f"or_point_mesh failed ({rc})")
    return d, tri, q


def world_vertices(mesh, x):
    """float64 world coordinates of a mesh's vertices under [R|t]."""
    v = np.asarray(mesh[0], dtype=np.float64)
    X = np.asarray(x, dtype=np.float64).reshape(3, 4)
    return v @ X[:, :3].T + X[:, 3]


def diag(A, xa, B, xb) -> float:
    """Diagonal of the world bounding box of both meshes' referenced vertices."""
    pts = []
    for m, x in ((A, xa), (B, xb)):
        w = world_vertices(m, x)
        used = np.unique(np.asarray(m[1]).reshape(-1))
        pts.append(w[used])
    p = np.concatenate(pts)
    return float(np.linalg.norm(p.max(0) - p.min(0)))


def witness_distance(A, xa, B, xb, ta, tb, kind: str = "min"):
    """The oracle's float64 distance of one triangle pair (a witness check),
    with the world mapping done exactly as in the mesh queries.
    Returns (d, pa, pb)."""
    a9 = np.ascontiguousarray(np.asarray(A[0], dtype=np.float32)[np.asarray(A[1])[int(ta)]].reshape(9))
    b9 = np.ascontiguousarray(np.asarray(B[0], dtype=np.float32)[np.asarray(B[1])[int(tb)]].reshape(9))
    xa, xb = _d(xa, 12), _d(xb, 12)
    pa, pb = np.zeros(3), np.zeros(3)
    d = lib().or_tri_pair_world(_ptr(a9, _fp), _ptr(xa, _dp), _ptr(b9, _fp), _ptr(xb, _dp),
                                1 if kind == "max" else 0, _ptr(pa, _dp), _ptr(pb, _dp))
    return d, pa, pb
