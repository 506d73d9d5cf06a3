"""ctypes binding of the engine's C ABI (include/gdist.h).

Argument marshalling only: every function forwards to the function of the same
name in libgdist.so, and every step of the computation runs in the library's
CUDA kernels.  There is no CPU fallback: if the library is missing or no CUDA
device is present, the calls raise.
"""

from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libgdist.so")

GD_OK, GD_ERR_INVALID_ARG, GD_ERR_OOM, GD_ERR_CUDA, GD_ERR_NOT_BUILT = 0, 1, 2, 3, 4
GD_ERR_OVERFLOW, GD_ERR_TIMEOUT, GD_ERR_BUSY, GD_ERR_NOT_READY = 5, 6, 7, 8
GD_MIN, GD_MAX = 0, 1
STATUS_NAMES = {
    0: "GD_OK", 1: "GD_ERR_INVALID_ARG", 2: "GD_ERR_OOM", 3: "GD_ERR_CUDA", 4: "GD_ERR_NOT_BUILT",
    5: "GD_ERR_OVERFLOW", 6: "GD_ERR_TIMEOUT", 7: "GD_ERR_BUSY", 8: "GD_ERR_NOT_READY",
}

# every symbol include/gdist.h declares
EXPORTS = [
    "gd_ctx_create", "gd_ctx_destroy", "gd_last_error", "gd_ctx_set_tunables", "gd_ctx_get_tunables",
    "gd_get_stats", "gd_ctx_stream", "gd_mesh_create", "gd_bvh_build", "gd_mesh_update", "gd_mesh_destroy", "gd_mesh_info",
    "gd_mesh_download", "gd_min_distance", "gd_max_distance", "gd_naive_query", "gd_point_distance", "gd_point_stats", "gd_query_device", "gd_query_device_noalloc",
    "gd_batch_query", "gd_batch_times", "gd_autotune", "gd_graph_create", "gd_graph_launch", "gd_graph_destroy",
    "gd_mesh_build_time", "gd_query_footprint",
    "gd_serve_start", "gd_serve_submit", "gd_serve_poll", "gd_serve_drain", "gd_serve_stop",
]


class gd_point_result(C.Structure):
    _fields_ = [("d", C.c_double), ("tri", C.c_int64), ("p", C.c_double * 3), ("status", C.c_uint32),
                ("pad", C.c_uint32)]


class gd_naive_result(C.Structure):
    _fields_ = [("d", C.c_double), ("node_tests", C.c_uint64), ("leaf_tests", C.c_uint64),
                ("max_thread_tests", C.c_uint64), ("status", C.c_uint32), ("pad", C.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad"}


class gd_result(C.Structure):
    _fields_ = [("d", C.c_double), ("tri_a", C.c_int64), ("tri_b", C.c_int64), ("pa", C.c_double * 3),
                ("pb", C.c_double * 3), ("status", C.c_uint32), ("flags", C.c_uint32)]

    def as_dict(self):
        return {"d": self.d, "tri_a": self.tri_a, "tri_b": self.tri_b, "pa": list(self.pa), "pb": list(self.pb),
                "status": self.status, "flags": self.flags}


class gd_query(C.Structure):
    _fields_ = [("a", C.c_void_p), ("b", C.c_void_p), ("xa", C.c_double * 12), ("xb", C.c_double * 12),
                ("kind", C.c_int), ("user_tag", C.c_uint64)]


class gd_build_opts(C.Structure):
    _fields_ = [("morton_bits", C.c_int)]


class gd_tunables(C.Structure):
    _fields_ = [("work_target", C.c_int64), ("k_max", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("front_capacity", C.c_int64), ("leaf_capacity", C.c_int64), ("cand_capacity", C.c_int64),
                ("max_capacity", C.c_int64), ("timeout_ns", C.c_int64), ("refit_mode", C.c_int32),
                ("refit_slots", C.c_int32), ("probes", C.c_int32), ("batch_budget", C.c_int64),
                ("bounds_mode", C.c_int32)]


class gd_stats(C.Structure):
    _fields_ = [("levels", C.c_uint32), ("front", C.c_uint32 * 32), ("slots", C.c_uint32 * 32),
                ("pairs_tested", C.c_uint64), ("leaf_pairs", C.c_uint32), ("tri_pairs", C.c_uint32),
                ("candidates", C.c_uint32), ("refined", C.c_uint32), ("alg_bytes", C.c_uint64),
                ("retries", C.c_uint32), ("blocks", C.c_uint32), ("level_ns", C.c_uint32 * 32),
                ("phase_ns", C.c_uint32 * 12), ("probes", C.c_uint32), ("u_level", C.c_float * 32),
                ("u_probe", C.c_float), ("refits", C.c_uint32)]

    PHASES = ("setup", "refit", "probe", "levels", "leaf", "refine", "tail_wait", "select", "finalize", "total")

    def as_dict(self):
        n = self.levels
        return {"levels": n, "front": list(self.front[:min(n, 32)]), "slots": list(self.slots[:min(n, 32)]),
                "pairs_tested": self.pairs_tested, "leaf_pairs": self.leaf_pairs, "tri_pairs": self.tri_pairs,
                "candidates": self.candidates, "refined": self.refined, "alg_bytes": self.alg_bytes,
                "retries": self.retries, "blocks": self.blocks,
                "level_us": [x / 1000.0 for x in self.level_ns[:min(n, 32)]],
                "phase_us": {k: self.phase_ns[i] / 1000.0 for i, k in enumerate(self.PHASES)},
                "probes": self.probes, "u_level": list(self.u_level[:min(n, 32)]), "u_probe": self.u_probe,
                "refits": self.refits}


class gd_serve_opts(C.Structure):
    _fields_ = [("slots", C.c_int32), ("max_batch", C.c_int32), ("memory_budget", C.c_int64),
                ("linger_us", C.c_int32)]


_lib = None
_vp = C.c_void_p
_dp = C.POINTER(C.c_double)


def load(path: str = LIB_PATH):
    """Load libgdist.so (raises if it was not built: run __graft_entry__.build())."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA engine library missing: {path} (build it with __graft_entry__.build())")
    L = C.CDLL(path)
    sig = {
        "gd_ctx_create": (C.c_int, [C.c_int, C.POINTER(_vp)]),
        "gd_ctx_destroy": (None, [_vp]),
        "gd_last_error": (C.c_char_p, [_vp]),
        "gd_ctx_set_tunables": (C.c_int, [_vp, C.POINTER(gd_tunables)]),
        "gd_ctx_get_tunables": (C.c_int, [_vp, C.POINTER(gd_tunables)]),
        "gd_get_stats": (C.c_int, [_vp, C.POINTER(gd_stats)]),
        "gd_ctx_stream": (_vp, [_vp]),
        "gd_mesh_create": (C.c_int, [_vp, C.POINTER(C.c_float), C.c_int64, C.POINTER(C.c_int32), C.c_int64,
                                     C.POINTER(_vp)]),
        "gd_bvh_build": (C.c_int, [_vp, C.POINTER(gd_build_opts)]),
        "gd_mesh_update": (C.c_int, [_vp, _vp, C.c_int64]),
        "gd_mesh_destroy": (None, [_vp]),
        "gd_mesh_info": (C.c_int, [_vp, C.POINTER(C.c_int32), C.POINTER(C.c_int64)]),
        "gd_mesh_download": (C.c_int, [_vp, C.POINTER(C.c_float), C.POINTER(C.c_int32)]),
        "gd_min_distance": (C.c_int, [_vp, _vp, _vp, _dp, _dp, C.POINTER(gd_result)]),
        "gd_max_distance": (C.c_int, [_vp, _vp, _vp, _dp, _dp, C.POINTER(gd_result)]),
        "gd_point_distance": (C.c_int, [_vp, _vp, _dp, _vp, C.c_int64, _vp]),
        "gd_point_stats": (C.c_int, [_vp, C.POINTER(C.c_uint64), C.POINTER(C.c_uint64)]),
        "gd_naive_query": (C.c_int, [_vp, _vp, _vp, C.c_int, _dp, _dp, C.c_int64, C.POINTER(gd_naive_result)]),
        "gd_query_device": (C.c_int, [_vp, _vp, _vp, C.c_int, _vp, _vp, _vp, _vp]),
        "gd_query_device_noalloc": (C.c_int, [_vp, _vp, C.c_int, _vp, _vp, _vp, _vp]),
        "gd_batch_query": (C.c_int, [_vp, C.POINTER(gd_query), C.c_int64, C.POINTER(gd_result)]),
        "gd_batch_times": (C.c_int, [_vp, C.c_int64, C.POINTER(C.c_int64)]),
        "gd_query_footprint": (C.c_int, [C.POINTER(gd_query), C.POINTER(C.c_int64)]),
        "gd_mesh_build_time": (C.c_int, [_vp, C.POINTER(C.c_double)]),
        "gd_autotune": (C.c_int, [_vp, C.POINTER(gd_query), C.c_int64, C.c_int32, C.POINTER(gd_tunables)]),
        "gd_graph_create": (C.c_int, [_vp, _vp, _vp, C.c_int, _vp, _vp, _vp, C.POINTER(_vp)]),
        "gd_graph_launch": (C.c_int, [_vp, _vp]),
        "gd_graph_destroy": (C.c_int, [_vp]),
        "gd_serve_start": (C.c_int, [_vp, C.POINTER(gd_serve_opts), C.POINTER(_vp)]),
        "gd_serve_submit": (C.c_int, [_vp, C.POINTER(gd_query), C.POINTER(C.c_uint64)]),
        "gd_serve_poll": (C.c_int, [_vp, C.c_uint64, C.POINTER(gd_result)]),
        "gd_serve_drain": (C.c_int, [_vp, C.POINTER(C.c_uint64), C.POINTER(gd_result), C.c_int64,
                                     C.POINTER(C.c_int64)]),
        "gd_serve_stop": (C.c_int, [_vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class GdError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(rc, ctx=None):
    if rc != GD_OK:
        msg = load().gd_last_error(ctx).decode() if ctx else ""
        raise GdError(rc, msg)


def _x(a):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(12))
    return a


# ------------------------------------------------------------- same-name wrappers

def gd_ctx_create(device: int = 0):
    h = _vp()
    _check(load().gd_ctx_create(device, C.byref(h)))
    return h.value


def gd_ctx_destroy(ctx):
    load().gd_ctx_destroy(ctx)


def gd_last_error(ctx) -> str:
    return load().gd_last_error(ctx).decode()


def gd_ctx_set_tunables(ctx, **kw):
    t = gd_tunables()
    for k, v in kw.items():
        setattr(t, k, int(v))
    _check(load().gd_ctx_set_tunables(ctx, C.byref(t)), ctx)


def gd_ctx_get_tunables(ctx) -> dict:
    t = gd_tunables()
    _check(load().gd_ctx_get_tunables(ctx, C.byref(t)), ctx)
    return {f: getattr(t, f) for f, _ in gd_tunables._fields_}


def gd_get_stats(ctx) -> dict:
    s = gd_stats()
    _check(load().gd_get_stats(ctx, C.byref(s)), ctx)
    return s.as_dict()


def gd_ctx_stream(ctx) -> int:
    return load().gd_ctx_stream(ctx) or 0


def gd_mesh_create(ctx, verts, tris):
    v = np.ascontiguousarray(np.asarray(verts, dtype=np.float32).reshape(-1, 3))
    t = np.ascontiguousarray(np.asarray(tris, dtype=np.int32).reshape(-1, 3))
    h = _vp()
    rc = load().gd_mesh_create(ctx, v.ctypes.data_as(C.POINTER(C.c_float)), len(v),
                               t.ctypes.data_as(C.POINTER(C.c_int32)), len(t), C.byref(h))
    _check(rc, ctx)
    return h.value


def gd_bvh_build(mesh, morton_bits: int | None = None, ctx=None):
    o = None
    if morton_bits is not None:
        o = C.byref(gd_build_opts(int(morton_bits)))
    _check(load().gd_bvh_build(mesh, o), ctx)


def gd_mesh_update(mesh, verts, ctx=None):
    """New vertex positions for a built mesh, then a device refit of its BVH.
    verts: an (nv, 3) float32 array on the host, or a contiguous float32 CUDA
    tensor (its device pointer is passed through)."""
    if hasattr(verts, "is_cuda") and verts.is_cuda:
        if str(verts.dtype) != "torch.float32" or not verts.is_contiguous() or verts.numel() % 3:
            raise ValueError("device vertices must be a contiguous float32 tensor of nv x 3 values")
        _check(load().gd_mesh_update(mesh, _vp(verts.data_ptr()), verts.numel() // 3), ctx)
        return
    v = np.ascontiguousarray(np.asarray(verts, dtype=np.float32).reshape(-1, 3))
    _check(load().gd_mesh_update(mesh, _vp(v.ctypes.data), len(v)), ctx)


def gd_mesh_destroy(mesh):
    load().gd_mesh_destroy(mesh)


def gd_mesh_info(mesh):
    L = C.c_int32()
    T = C.c_int64()
    _check(load().gd_mesh_info(mesh, C.byref(L), C.byref(T)))
    return L.value, T.value


def gd_mesh_build_time(mesh) -> float:
    """Device ms of the kernels of the mesh's last BVH build."""
    t = C.c_double()
    _check(load().gd_mesh_build_time(mesh, C.byref(t)))
    return t.value


def gd_mesh_download(mesh):
    L, T = gd_mesh_info(mesh)
    boxes = np.zeros((2 << L, 6), dtype=np.float32)
    order = np.zeros(T, dtype=np.int32)
    _check(load().gd_mesh_download(mesh, boxes.ctypes.data_as(C.POINTER(C.c_float)),
                                   order.ctypes.data_as(C.POINTER(C.c_int32))))
    return boxes, order


_tls = threading.local()


def _xbufs():
    """Per-thread ctypes arrays for two transforms and numpy views of them
    (numpy's .ctypes.data_as costs microseconds per call; filling a
    preallocated array does not)."""
    b = getattr(_tls, "x", None)
    if b is None:
        ba, bb = (C.c_double * 12)(), (C.c_double * 12)()
        b = _tls.x = (ba, bb, np.frombuffer(ba, dtype=np.float64), np.frombuffer(bb, dtype=np.float64))
    return b


def _query(fn, ctx, A, B, xa, xb):
    ba, bb, va, vb = _xbufs()
    va[:] = np.asarray(xa, dtype=np.float64).reshape(12)
    vb[:] = np.asarray(xb, dtype=np.float64).reshape(12)
    r = gd_result()
    rc = fn(ctx, A, B, ba, bb, C.byref(r))
    _check(rc, ctx)
    return r


def gd_min_distance(ctx, A, B, xa, xb) -> gd_result:
    return _query(load().gd_min_distance, ctx, A, B, xa, xb)


def gd_max_distance(ctx, A, B, xa, xb) -> gd_result:
    return _query(load().gd_max_distance, ctx, A, B, xa, xb)


def gd_point_distance(ctx, M, x, points):
    """Distances from world points to mesh M placed by x.  points: an (n, 3)
    float64 array on the host, or a contiguous float64 CUDA tensor.  Returns a
    structured numpy array with fields d, tri, p, status (host), or, for a
    CUDA tensor input, a CUDA tensor of n x 6 float64 holding the raw
    gd_point_result records."""
    x = _x(x)
    if hasattr(points, "is_cuda") and points.is_cuda:
        import torch
        if points.dtype != torch.float64 or not points.is_contiguous() or points.numel() % 3:
            raise ValueError("device points must be a contiguous float64 tensor of n x 3 values")
        n = points.numel() // 3
        out = torch.empty((n, C.sizeof(gd_point_result) // 8), dtype=torch.float64, device=points.device)
        _check(load().gd_point_distance(ctx, M, x.ctypes.data_as(_dp), _vp(points.data_ptr()), n,
                                        _vp(out.data_ptr())), ctx)
        return out
    P = np.ascontiguousarray(np.asarray(points, dtype=np.float64).reshape(-1, 3))
    n = len(P)
    out = (gd_point_result * max(n, 1))()
    _check(load().gd_point_distance(ctx, M, x.ctypes.data_as(_dp), _vp(P.ctypes.data), n,
                                    C.cast(out, _vp)), ctx)
    dt = np.dtype([("d", np.float64), ("tri", np.int64), ("p", np.float64, 3), ("status", np.uint32),
                   ("pad", np.uint32)])
    return np.frombuffer(bytes(out), dtype=dt, count=n).copy()


def gd_point_records(raw):
    """View raw gd_point_result records (a CPU copy of the tensor that
    gd_point_distance returns for device points) as a structured array."""
    dt = np.dtype([("d", np.float64), ("tri", np.int64), ("p", np.float64, 3), ("status", np.uint32),
                   ("pad", np.uint32)])
    return np.frombuffer(np.ascontiguousarray(raw).tobytes(), dtype=dt).copy()


def gd_point_stats(ctx):
    a, b = C.c_uint64(), C.c_uint64()
    _check(load().gd_point_stats(ctx, C.byref(a), C.byref(b)), ctx)
    return {"node_tests": a.value, "exact_tests": b.value}


def gd_naive_query(ctx, A, B, kind: int, xa, xb, timeout_ns: int = 0) -> dict:
    """The naive comparator; a timeout is reported in the result's status
    (with partial counts) instead of raising."""
    xa, xb = _x(xa), _x(xb)
    r = gd_naive_result()
    rc = load().gd_naive_query(ctx, A, B, int(kind), xa.ctypes.data_as(_dp), xb.ctypes.data_as(_dp),
                               int(timeout_ns), C.byref(r))
    if rc not in (GD_OK, GD_ERR_TIMEOUT):
        _check(rc, ctx)
    return r.as_dict()


def gd_query_device(ctx, A, B, kind: int, d_xa: int, d_xb: int, d_out: int, stream: int = 0):
    """Device-resident query: d_xa, d_xb, d_out are device addresses (ints)."""
    _check(load().gd_query_device(ctx, A, B, int(kind), d_xa, d_xb, d_out, stream or None), ctx)


def gd_query_device_noalloc(A, B, kind: int, d_xa: int, d_xb: int, d_out: int, stream: int = 0):
    """Device-resident query whose work buffers come from a fixed array inside
    the library (no allocation); device addresses as ints."""
    _check(load().gd_query_device_noalloc(A, B, int(kind), d_xa, d_xb, d_out, stream or None))


def make_queries(items):
    """items: iterable of (meshA, meshB, xa, xb, kind[, tag]) -> ctypes array of gd_query."""
    items = list(items)
    arr = (gd_query * len(items))()
    for i, it in enumerate(items):
        a, b, xa, xb, kind = it[:5]
        arr[i].a = a
        arr[i].b = b
        arr[i].xa[:] = list(_x(xa))
        arr[i].xb[:] = list(_x(xb))
        arr[i].kind = int(kind)
        arr[i].user_tag = int(it[5]) if len(it) > 5 else i
    return arr


def gd_graph_create(ctx, A, B, kind, d_xa, d_xb, d_out):
    """Graph of one device-resident query (device pointers as ints)."""
    g = _vp()
    _check(load().gd_graph_create(ctx, A, B, int(kind), d_xa, d_xb, d_out, C.byref(g)), ctx)
    return g.value


def gd_graph_launch(graph, stream=None, ctx=None):
    _check(load().gd_graph_launch(graph, stream or None), ctx)


def gd_graph_destroy(graph):
    _check(load().gd_graph_destroy(graph))


def gd_autotune(ctx, sample, reps=3) -> dict:
    """Tune ctx's traversal tunables on a sample of queries; returns them."""
    if not isinstance(sample, C.Array):
        sample = make_queries(sample)
    t = gd_tunables()
    _check(load().gd_autotune(ctx, sample, len(sample), int(reps), C.byref(t)), ctx)
    return {f: getattr(t, f) for f, _ in gd_tunables._fields_}


def gd_batch_query(ctx, queries):
    if not isinstance(queries, C.Array):
        queries = make_queries(queries)
    n = len(queries)
    out = (gd_result * n)()
    _check(load().gd_batch_query(ctx, queries, n, out), ctx)
    return out


def gd_batch_times(ctx, n: int) -> np.ndarray:
    """Per-query completion times of the last gd_batch_query (device ns since
    the start of that call's first launch)."""
    out = np.zeros(n, dtype=np.int64)
    _check(load().gd_batch_times(ctx, n, out.ctypes.data_as(C.POINTER(C.c_int64))), ctx)
    return out


def gd_query_footprint(query) -> int:
    """Predicted work-buffer bytes of one query (the server's admission model)."""
    if not isinstance(query, gd_query):
        query = make_queries([query])[0]
    b = C.c_int64()
    _check(load().gd_query_footprint(C.byref(query), C.byref(b)))
    return b.value


def gd_serve_start(ctx, slots=0, max_batch=0, memory_budget=0, linger_us=0):
    o = gd_serve_opts(int(slots), int(max_batch), int(memory_budget), int(linger_us))
    h = _vp()
    _check(load().gd_serve_start(ctx, C.byref(o), C.byref(h)), ctx)
    return h.value


def gd_serve_submit(srv, query: gd_query):
    t = C.c_uint64()
    rc = load().gd_serve_submit(srv, C.byref(query), C.byref(t))
    return rc, t.value


def gd_serve_poll(srv, ticket):
    r = gd_result()
    rc = load().gd_serve_poll(srv, C.c_uint64(ticket), C.byref(r))
    return rc, r


_drain_bufs = {}


def gd_serve_drain(srv, max_n=256):
    """Finished requests as a list of (ticket, gd_result), at most max_n."""
    if max_n not in _drain_bufs:
        _drain_bufs[max_n] = ((C.c_uint64 * max_n)(), (gd_result * max_n)())
    tk, rs = _drain_bufs[max_n]
    n = C.c_int64()
    rc = load().gd_serve_drain(srv, tk, rs, max_n, C.byref(n))
    if rc != GD_OK:
        raise GdError(rc, "gd_serve_drain")
    return [(tk[i], gd_result.from_buffer_copy(rs[i])) for i in range(n.value)]


def gd_serve_stop(srv):
    _check(load().gd_serve_stop(srv))
