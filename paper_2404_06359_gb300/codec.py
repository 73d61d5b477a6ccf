"""Python binding of ``libmeshletcodec.so`` (argument marshalling only).

Every function named ``mc_*`` is the C entry point of the same name in
``include/meshlet_codec.h``; PyTorch tensors supply device memory and CUDA
streams.  All computation happens in the library: there is no Python or CPU
fallback, and importing this module fails loudly if the library cannot be
built or loaded.
"""
from __future__ import annotations

import ctypes as C
import threading

import numpy as np

from . import build as _build

u8, u16, u32, u64 = C.c_uint8, C.c_uint16, C.c_uint32, C.c_uint64
P = C.c_void_p


class mc_limits(C.Structure):
    _fields_ = [("max_verts", u32), ("max_tris", u32)]


class mc_encode_params(C.Structure):
    _fields_ = [("pos_bits", u32), ("pos_bits_per_meshlet", P), ("reuse_mode", u32),
                ("order", P), ("mesh_id", u32), ("n_threads", u32), ("attrs", P),
                ("n_attr", u32), ("attr_bits", u32), ("strip_search_nodes", u32)]


class mc_mesh_info(C.Structure):
    _fields_ = [("first_meshlet", u32), ("n_meshlets", u32), ("tri_base", u64), ("n_tris", u64),
                ("vertex_base", u64), ("n_verts", u64), ("input_tris", u64)]


class mc_blob_view_t(C.Structure):
    _fields_ = [("desc", P), ("n_meshlets", u32), ("payload", P), ("payload_bytes", u64),
                ("grids", P), ("n_grids", u32), ("meshes", C.POINTER(mc_mesh_info)),
                ("n_meshes", u32), ("vertex_map", P), ("total_tris", u64), ("total_verts", u64),
                ("input_tris", u64), ("restarts", u64), ("split_meshlets", u64),
                ("conn_bits", u64), ("pos_bits_total", u64), ("max_block_words", u32),
                ("max_tris", u32), ("cones", P), ("n_attr", u32), ("attr_bits", u32),
                ("attr_desc", P), ("attr_grids", P), ("n_attr_grids", u32), ("max_verts", u32)]


class mc_device_batch(C.Structure):
    _fields_ = [("desc", P), ("payload", P), ("grids", P), ("n_meshlets", u32), ("n_grids", u32),
                ("payload_bytes", u64), ("total_tris", u64), ("total_verts", u64),
                ("max_block_words", u32), ("max_tris", u32), ("cones", P),
                ("n_attr", u32), ("attr_bits", u32), ("attr_desc", P), ("attr_grids", P),
                ("n_attr_grids", u32), ("max_verts", u32)]


class mc_request(C.Structure):
    _fields_ = [("first_meshlet", u32), ("n_meshlets", u32), ("work_start", u32),
                ("reserved0", u32), ("tri_base", u32), ("vertex_base", u32), ("tri_count", u32),
                ("vert_count", u32), ("d_local", P), ("d_global", P), ("d_pos", P),
                ("reserved1", P)]


class mc_tuning(C.Structure):
    _fields_ = [("warps_per_cta", u32), ("ctas_per_sm", u32), ("meshlets_per_grab", u32),
                ("checked", u32), ("wait_cycles", u32), ("lanes_per_meshlet", u32)]


STATUS = {0: "MC_OK", 1: "MC_ERR_INVALID_ARG", 2: "MC_ERR_LIMIT", 3: "MC_ERR_CORRUPT",
          4: "MC_ERR_CUDA", 5: "MC_ERR_OOM", 6: "MC_ERR_TIMEOUT"}
MC_ERR_CORRUPT = 3
MC_ERR_TIMEOUT = 6

# every entry point of include/meshlet_codec.h: (name, restype, argtypes)
_SIGS = [
    ("mc_status_string", C.c_char_p, [C.c_int]),
    ("mc_version", C.c_char_p, []),
    ("mc_meshletize", C.c_int, [P, u32, u32, P, C.POINTER(mc_limits), u32, u32, C.POINTER(P)]),
    ("mc_meshlets_count", u32, [P]),
    ("mc_meshlets_get", C.c_int, [P, P, P]),
    ("mc_meshlets_free", None, [P]),
    ("mc_encode", C.c_int, [P, P, u32, C.POINTER(mc_encode_params), C.POINTER(P)]),
    ("mc_blob_concat", C.c_int, [C.POINTER(P), u32, C.POINTER(P)]),
    ("mc_blob_view", C.c_int, [P, C.POINTER(mc_blob_view_t)]),
    ("mc_blob_free", None, [P]),
    ("mc_scratch_bytes", C.c_size_t, []),
    ("mc_decode_plain", C.c_int, [C.POINTER(mc_device_batch), u32, u32, P, P, P, P,
                                  C.POINTER(mc_tuning), P]),
    ("mc_decode_batch", C.c_int, [C.POINTER(mc_device_batch), P, P, P, P, P,
                                  C.POINTER(mc_tuning), P]),
    ("mc_decode_batch_vertices", C.c_int, [C.POINTER(mc_device_batch), P, P, P, P, P,
                                           C.POINTER(mc_tuning), P]),
    ("mc_decode_batch_noalloc", C.c_int, [C.POINTER(mc_device_batch), P, P, P, P,
                                          C.POINTER(mc_tuning), P]),
    ("mc_decode_cull", C.c_int, [C.POINTER(mc_device_batch), P, P, P, P, P, P,
                                 C.POINTER(mc_tuning), P]),
    ("mc_decode_cull_views", C.c_int, [C.POINTER(mc_device_batch), P, u32, P, u64, P, P, P, P,
                                       C.POINTER(mc_tuning), P]),
    ("mc_cull_order_bytes", C.c_size_t, [C.POINTER(mc_device_batch)]),
    ("mc_decode_cull_ordered", C.c_int, [C.POINTER(mc_device_batch), P, P, P, P, P, P, P,
                                         C.POINTER(mc_tuning), P]),
    ("mc_decode_requests", C.c_int, [C.POINTER(mc_device_batch), P, u32, u32, P, P,
                                     C.POINTER(mc_tuning), P]),
    ("mc_autotune", C.c_int, [C.POINTER(mc_device_batch), P, P, P, P, P, P,
                              C.POINTER(mc_tuning), C.POINTER(C.c_float)]),
    ("mc_graph_capture_batch", C.c_int, [C.POINTER(mc_device_batch), P, P, P, P, P,
                                         C.POINTER(mc_tuning), P, C.POINTER(P)]),
    ("mc_graph_capture_cull", C.c_int, [C.POINTER(mc_device_batch), P, u32, P, P, P, P, P,
                                        C.POINTER(mc_tuning), P, C.POINTER(P)]),
    ("mc_graph_capture_cull_views", C.c_int, [C.POINTER(mc_device_batch), P, u32, P, u64, P, P,
                                              P, P, C.POINTER(mc_tuning), P, C.POINTER(P)]),
    ("mc_graph_launch", C.c_int, [P, P]),
    ("mc_graph_free", None, [P]),
    ("mc_decode_batch_host", C.c_int, [C.POINTER(mc_blob_view_t), P, P, P, P, P, P, P, P,
                                       P, P, P, C.POINTER(mc_tuning), P]),
    ("mc_launch_count", u64, []),
]

_lock = threading.Lock()
_lib = None


def lib():
    """The loaded library (built on first use if needed)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = C.CDLL(path)
            for name, res, args in _SIGS:
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
        return _lib


def exported_names() -> list[str]:
    return [s[0] for s in _SIGS]


class CodecError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {STATUS.get(status, status)}")
        self.status = status


def _check(st: int, what: str):
    if st != 0:
        raise CodecError(st, what)


def _np_ptr(a):
    return None if a is None else a.ctypes.data_as(P)


def _tptr(t):
    return None if t is None else P(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return P(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return P(stream)
    return P(stream.cuda_stream)


def _tuning(t):
    if t is None:
        return None
    if isinstance(t, mc_tuning):
        return C.byref(t)
    return C.byref(mc_tuning(**t))


def mc_status_string(st: int) -> str:
    return lib().mc_status_string(st).decode()


def mc_version() -> str:
    return lib().mc_version().decode()


def mc_scratch_bytes() -> int:
    return int(lib().mc_scratch_bytes())


def mc_launch_count() -> int:
    return int(lib().mc_launch_count())


# ------------------------------------------------------------------- host
class Meshlets:
    """Owns an ``mc_meshlets*``."""

    def __init__(self, handle, n_tris):
        self._h = handle
        self.n_tris = n_tris

    @property
    def count(self) -> int:
        return int(lib().mc_meshlets_count(self._h))

    def get(self):
        tri = np.zeros(self.n_tris, np.uint32)
        start = np.zeros(self.count + 1, np.uint32)
        _check(lib().mc_meshlets_get(self._h, _np_ptr(tri), _np_ptr(start)), "mc_meshlets_get")
        return tri, start

    def __del__(self):
        if getattr(self, "_h", None):
            lib().mc_meshlets_free(self._h)
            self._h = None


def mc_meshletize(tris: np.ndarray, n_verts: int, limits=((64, 126),), tri_class=None,
                  n_threads: int = 0) -> Meshlets:
    tris = np.ascontiguousarray(tris, np.uint32)
    lim = np.asarray(limits, np.uint32).reshape(-1, 2)
    arr = (mc_limits * lim.shape[0])(*[mc_limits(int(a), int(b)) for a, b in lim])
    cls = None if tri_class is None else np.ascontiguousarray(tri_class, np.uint8)
    h = P()
    _check(lib().mc_meshletize(_np_ptr(tris), tris.shape[0], n_verts, _np_ptr(cls), arr,
                               lim.shape[0], n_threads, C.byref(h)), "mc_meshletize")
    return Meshlets(h, tris.shape[0])


class Blob:
    """Owns an ``mc_blob*``; ``view()`` exposes its arrays as numpy views."""

    def __init__(self, handle):
        self._h = handle
        self._view = None

    def view(self) -> mc_blob_view_t:
        if self._view is None:
            v = mc_blob_view_t()
            _check(lib().mc_blob_view(self._h, C.byref(v)), "mc_blob_view")
            self._view = v
        return self._view

    def arrays(self) -> dict:
        """Copies of desc (uint8 [M,32]), payload, grids (uint8 [G,32]),
        cones (uint8 [M,32], mc_cone records), vertex_map and the per-mesh
        table."""
        v = self.view()

        def grab(ptr, n, dt):
            if n == 0:
                return np.zeros(0, dt)
            return np.ctypeslib.as_array(C.cast(ptr, C.POINTER(np.ctypeslib.as_ctypes_type(dt))),
                                         (n,)).copy()
        meshes = [{k: int(getattr(v.meshes[i], k)) for k, _ in mc_mesh_info._fields_}
                  for i in range(v.n_meshes)]
        return {
            "desc": grab(v.desc, 32 * v.n_meshlets, np.uint8).reshape(-1, 32),
            "payload": grab(v.payload, v.payload_bytes, np.uint8),
            "grids": grab(v.grids, 32 * v.n_grids, np.uint8).reshape(-1, 32),
            "cones": grab(v.cones, 32 * v.n_meshlets, np.uint8).reshape(-1, 32),
            "attr_desc": grab(v.attr_desc, 32 * v.n_meshlets if v.n_attr else 0,
                              np.uint8).reshape(-1, 32),
            "attr_grids": grab(v.attr_grids, 48 * v.n_attr_grids, np.uint8).reshape(-1, 48),
            "vertex_map": grab(v.vertex_map, v.total_verts, np.uint32),
            "meshes": meshes,
        }

    def stats(self) -> dict:
        v = self.view()
        keys = ("n_meshlets", "payload_bytes", "n_grids", "n_meshes", "total_tris", "total_verts",
                "input_tris", "restarts", "split_meshlets", "conn_bits", "pos_bits_total",
                "max_block_words", "max_tris", "max_verts", "n_attr", "attr_bits")
        return {k: int(getattr(v, k)) for k in keys}

    def __del__(self):
        if getattr(self, "_h", None):
            lib().mc_blob_free(self._h)
            self._h = None


def mc_encode(meshlets: Meshlets, pos: np.ndarray, pos_bits=16, reuse_mode: int = 0, order=None,
              mesh_id: int = 0, n_threads: int = 0, attrs: np.ndarray | None = None,
              attr_bits: int = 16, strip_search_nodes: int = 0) -> Blob:
    """attrs: optional float32 [n_verts, n_attr] extra attribute channels (n_attr <= 5);
    strip_search_nodes: node budget of the fewest-strips search per meshlet
    (0 = the greedy strips)."""
    pos = np.ascontiguousarray(pos, np.float32)
    per = None
    if np.ndim(pos_bits) > 0:
        per = np.ascontiguousarray(pos_bits, np.uint8)
    order = None if order is None else np.ascontiguousarray(order, np.uint32)
    at = None if attrs is None else np.ascontiguousarray(attrs, np.float32).reshape(pos.shape[0], -1)
    n_attr = 0 if at is None else at.shape[1]
    p = mc_encode_params(int(pos_bits) if per is None else 0, _np_ptr(per), reuse_mode,
                         _np_ptr(order), mesh_id, n_threads, _np_ptr(at), n_attr,
                         attr_bits if n_attr else 0, strip_search_nodes)
    h = P()
    _check(lib().mc_encode(meshlets._h, _np_ptr(pos), pos.shape[0], C.byref(p), C.byref(h)),
           "mc_encode")
    return Blob(h)


def mc_blob_concat(blobs: list[Blob]) -> Blob:
    arr = (P * len(blobs))(*[b._h for b in blobs])
    h = P()
    _check(lib().mc_blob_concat(arr, len(blobs), C.byref(h)), "mc_blob_concat")
    return Blob(h)


# ----------------------------------------------------------------- device
class DeviceBatch:
    """A blob copied into device memory (torch uint8 tensors) plus the
    ``mc_device_batch`` that points at it."""

    def __init__(self, blob: Blob, device="cuda", cones: bool = False, attrs: bool = False):
        """cones: also copy the normal cones (enables the cone test of the
        fused cull); attrs: also copy the attribute records and grids (for
        mc_decode_batch_vertices)."""
        a = blob.arrays()
        self._init(a["desc"], a["payload"], a["grids"], blob.stats(), device,
                   a["cones"] if cones else None,
                   (a["attr_desc"], a["attr_grids"]) if attrs else None)
        self.meshes = a["meshes"]

    @classmethod
    def from_arrays(cls, desc, payload, grids, total_tris, total_verts, max_block_words,
                    max_tris=256, device="cuda", cones=None, attrs: dict | None = None,
                    max_verts: int = 0):
        """Wrap blob arrays that did not come from ``mc_encode`` (e.g. a
        hand-packed stream); sizes are the caller's; cones (uint8 [M,32])
        optional; attrs: {"n_attr", "attr_bits", "adesc", "agrids"} of a blob
        with attribute channels (optional); max_verts: largest V (0 = bounded
        by max_tris + 2)."""
        self = cls.__new__(cls)
        stats = {"n_meshlets": desc.shape[0], "n_grids": grids.shape[0],
                 "payload_bytes": payload.size, "total_tris": total_tris,
                 "total_verts": total_verts, "max_block_words": max_block_words,
                 "max_tris": max_tris, "max_verts": max_verts,
                 "n_attr": attrs["n_attr"] if attrs else 0,
                 "attr_bits": attrs["attr_bits"] if attrs else 0}
        self._init(np.asarray(desc, np.uint8), np.asarray(payload, np.uint8),
                   np.asarray(grids, np.uint8), stats, device,
                   None if cones is None else np.asarray(cones, np.uint8),
                   (attrs["adesc"], attrs["agrids"]) if attrs else None)
        self.meshes = []
        return self

    def _init(self, desc, payload, grids, stats, device, cones=None, attr_arrays=None):
        import torch
        self.stats = stats
        self.desc = torch.from_numpy(np.ascontiguousarray(desc).reshape(-1)).to(device)
        self.payload = torch.from_numpy(np.ascontiguousarray(payload) if payload.size
                                        else np.zeros(16, np.uint8)).to(device)
        self.grids = torch.from_numpy(np.ascontiguousarray(grids).reshape(-1)).to(device)
        self.cones = None if cones is None or cones.size == 0 else \
            torch.from_numpy(np.ascontiguousarray(cones).reshape(-1)).to(device)
        self.attr_desc = self.attr_grids = None
        if attr_arrays is not None and attr_arrays[0].size:
            self.attr_desc = torch.from_numpy(np.ascontiguousarray(attr_arrays[0]).reshape(-1)).to(device)
            self.attr_grids = torch.from_numpy(np.ascontiguousarray(attr_arrays[1]).reshape(-1)).to(device)
        s = self.stats
        self.c = mc_device_batch(self.desc.data_ptr(), self.payload.data_ptr(), self.grids.data_ptr(),
                                 s["n_meshlets"], s["n_grids"], s["payload_bytes"], s["total_tris"],
                                 s["total_verts"], max(1, s["max_block_words"]),
                                 s.get("max_tris", 256),
                                 None if self.cones is None else self.cones.data_ptr(),
                                 s.get("n_attr", 0), s.get("attr_bits", 0),
                                 None if self.attr_desc is None else self.attr_desc.data_ptr(),
                                 None if self.attr_grids is None else self.attr_grids.data_ptr(),
                                 0 if self.attr_grids is None else self.attr_grids.numel() // 48,
                                 s.get("max_verts", 0))

    def outputs(self, local=True, global_=True, device="cuda"):
        import torch
        T, V = self.stats["total_tris"], self.stats["total_verts"]
        return {
            "local": torch.empty(3 * T, dtype=torch.uint8, device=device) if local else None,
            "global": torch.empty(3 * T, dtype=torch.int32, device=device) if global_ else None,
            "pos": torch.empty(3 * V, dtype=torch.float32, device=device),
            "status": torch.zeros(1, dtype=torch.int32, device=device),
        }


def new_scratch(device="cuda"):
    import torch
    return torch.zeros(mc_scratch_bytes() // 4, dtype=torch.int32, device=device)


def mc_decode_plain(db: DeviceBatch, first, count, d_local, d_global, d_pos, d_status,
                    tuning=None, stream=None):
    _check(lib().mc_decode_plain(C.byref(db.c), first, count, _tptr(d_local), _tptr(d_global),
                                 _tptr(d_pos), _tptr(d_status), _tuning(tuning), _stream(stream)),
           "mc_decode_plain")


def mc_decode_batch(db: DeviceBatch, d_local, d_global, d_pos, d_status, d_scratch, tuning=None,
                    stream=None):
    _check(lib().mc_decode_batch(C.byref(db.c), _tptr(d_local), _tptr(d_global), _tptr(d_pos),
                                 _tptr(d_status), _tptr(d_scratch), _tuning(tuning), _stream(stream)),
           "mc_decode_batch")


def mc_decode_cull_ordered(db: DeviceBatch, d_view_proj, d_tri_out, d_tri_count, d_pos, d_status,
                           d_scratch, d_order=None, tuning=None, stream=None):
    """Fused cull with the survivors in meshlet order, then triangle order.
    d_order: uint8 device buffer of mc_cull_order_bytes bytes (allocated here
    when None)."""
    if d_order is None:
        import torch
        d_order = torch.empty(int(lib().mc_cull_order_bytes(C.byref(db.c))), dtype=torch.uint8,
                              device="cuda")
    _check(lib().mc_decode_cull_ordered(C.byref(db.c), _tptr(d_view_proj), _tptr(d_tri_out),
                                        _tptr(d_tri_count), _tptr(d_pos), _tptr(d_status),
                                        _tptr(d_scratch), _tptr(d_order), _tuning(tuning),
                                        _stream(stream)),
           "mc_decode_cull_ordered")


def mc_decode_batch_vertices(db: DeviceBatch, d_local, d_global, d_vertex, d_status, d_scratch,
                             tuning=None, stream=None):
    """Batched decode writing full 32-byte vertices (x, y, z, attribute
    channels, zero padding) into d_vertex (float32 [8 * total_verts])."""
    _check(lib().mc_decode_batch_vertices(C.byref(db.c), _tptr(d_local), _tptr(d_global),
                                          _tptr(d_vertex), _tptr(d_status), _tptr(d_scratch),
                                          _tuning(tuning), _stream(stream)),
           "mc_decode_batch_vertices")


def mc_decode_batch_noalloc(db: DeviceBatch, d_local, d_global, d_pos, d_status, tuning=None,
                            stream=None):
    """mc_decode_batch without a scratch argument (the library's own static
    device array holds the work-queue counters; nothing is allocated)."""
    _check(lib().mc_decode_batch_noalloc(C.byref(db.c), _tptr(d_local), _tptr(d_global),
                                         _tptr(d_pos), _tptr(d_status), _tuning(tuning),
                                         _stream(stream)), "mc_decode_batch_noalloc")


def mc_decode_cull_views(db: DeviceBatch, d_view_projs, n_views, d_tri_out, tri_stride, d_tri_counts,
                         d_pos, d_status, d_scratch, tuning=None, stream=None):
    """Fused cull against n_views (1..8) matrices in one launch: view v's
    survivors at d_tri_out[v * tri_stride:], its count in d_tri_counts[v]."""
    _check(lib().mc_decode_cull_views(C.byref(db.c), _tptr(d_view_projs), n_views, _tptr(d_tri_out),
                                      tri_stride, _tptr(d_tri_counts), _tptr(d_pos),
                                      _tptr(d_status), _tptr(d_scratch), _tuning(tuning),
                                      _stream(stream)), "mc_decode_cull_views")


def mc_decode_cull(db: DeviceBatch, d_view_proj, d_tri_out, d_tri_count, d_pos, d_status, d_scratch,
                   tuning=None, stream=None):
    _check(lib().mc_decode_cull(C.byref(db.c), _tptr(d_view_proj), _tptr(d_tri_out),
                                _tptr(d_tri_count), _tptr(d_pos), _tptr(d_status), _tptr(d_scratch),
                                _tuning(tuning), _stream(stream)), "mc_decode_cull")


REQUEST_DTYPE = np.dtype([("first_meshlet", "<u4"), ("n_meshlets", "<u4"), ("work_start", "<u4"),
                          ("reserved0", "<u4"), ("tri_base", "<u4"), ("vertex_base", "<u4"),
                          ("tri_count", "<u4"), ("vert_count", "<u4"), ("d_local", "<u8"),
                          ("d_global", "<u8"), ("d_pos", "<u8"), ("reserved1", "<u8")])
assert REQUEST_DTYPE.itemsize == C.sizeof(mc_request) == 64


def mc_decode_requests(db: DeviceBatch, d_reqs, n_reqs: int, total_work: int, d_status, d_scratch,
                       tuning=None, stream=None):
    """d_reqs: a device tensor holding n_reqs mc_request records (REQUEST_DTYPE)."""
    _check(lib().mc_decode_requests(C.byref(db.c), _tptr(d_reqs), n_reqs, total_work,
                                    _tptr(d_status), _tptr(d_scratch), _tuning(tuning),
                                    _stream(stream)), "mc_decode_requests")


def mc_autotune(db: DeviceBatch, d_local, d_global, d_pos, d_status, d_scratch, stream=None):
    best = mc_tuning()
    ms = C.c_float()
    _check(lib().mc_autotune(C.byref(db.c), _tptr(d_local), _tptr(d_global), _tptr(d_pos),
                             _tptr(d_status), _tptr(d_scratch), _stream(stream), C.byref(best),
                             C.byref(ms)), "mc_autotune")
    return best, float(ms.value)


class Graph:
    def __init__(self, h):
        self._h = h

    def launch(self, stream=None):
        mc_graph_launch(self, stream)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().mc_graph_free(self._h)
            self._h = None


def mc_graph_capture_batch(db: DeviceBatch, d_local, d_global, d_pos, d_status, d_scratch,
                           tuning=None, stream=None) -> Graph:
    h = P()
    _check(lib().mc_graph_capture_batch(C.byref(db.c), _tptr(d_local), _tptr(d_global), _tptr(d_pos),
                                        _tptr(d_status), _tptr(d_scratch), _tuning(tuning),
                                        _stream(stream), C.byref(h)), "mc_graph_capture_batch")
    return Graph(h)


def mc_graph_capture_cull(db: DeviceBatch, d_view_projs, n_views, d_tri_out, d_tri_count, d_pos,
                          d_status, d_scratch, tuning=None, stream=None) -> Graph:
    h = P()
    _check(lib().mc_graph_capture_cull(C.byref(db.c), _tptr(d_view_projs), n_views, _tptr(d_tri_out),
                                       _tptr(d_tri_count), _tptr(d_pos), _tptr(d_status),
                                       _tptr(d_scratch), _tuning(tuning), _stream(stream), C.byref(h)),
           "mc_graph_capture_cull")
    return Graph(h)


def mc_graph_capture_cull_views(db: DeviceBatch, d_view_projs, n_views, d_tri_out, tri_stride,
                                d_tri_counts, d_pos, d_status, d_scratch, tuning=None,
                                stream=None) -> Graph:
    """Graph of ceil(n_views / 8) multi-view cull launches; view v writes
    region v % 8 of d_tri_out (tri_stride words each) and d_tri_counts[v]."""
    h = P()
    _check(lib().mc_graph_capture_cull_views(C.byref(db.c), _tptr(d_view_projs), n_views,
                                             _tptr(d_tri_out), tri_stride, _tptr(d_tri_counts),
                                             _tptr(d_pos), _tptr(d_status), _tptr(d_scratch),
                                             _tuning(tuning), _stream(stream), C.byref(h)),
           "mc_graph_capture_cull_views")
    return Graph(h)


def mc_graph_launch(g: Graph, stream=None):
    _check(lib().mc_graph_launch(g._h, _stream(stream)), "mc_graph_launch")


def pinned_inputs(blob: Blob) -> dict:
    """Page-locked host copies of the blob's descriptor, payload and grid
    arrays (for mc_decode_batch_host's asynchronous input copies)."""
    import torch
    a = blob.arrays()
    return {k: torch.from_numpy(np.ascontiguousarray(a[k]).reshape(-1)).pin_memory()
            for k in ("desc", "payload", "grids")}


def mc_decode_batch_host(blob: Blob, d_desc, d_payload, d_grids, d_local, d_global, d_pos, d_status,
                         d_scratch, h_local, h_global, h_pos, tuning=None, stream=None,
                         host_inputs: dict | None = None):
    """host_inputs: optional pinned copies of the blob arrays (pinned_inputs)
    used as the copy sources instead of the blob's own (pageable) arrays."""
    v = blob.view()
    if host_inputs is not None:
        v = mc_blob_view_t.from_buffer_copy(v)
        for k in ("desc", "payload", "grids"):
            setattr(v, k, host_inputs[k].data_ptr())
    _check(lib().mc_decode_batch_host(C.byref(v), _tptr(d_desc), _tptr(d_payload), _tptr(d_grids),
                                      _tptr(d_local), _tptr(d_global), _tptr(d_pos), _tptr(d_status),
                                      _tptr(d_scratch), _tptr(h_local), _tptr(h_global), _tptr(h_pos),
                                      _tuning(tuning), _stream(stream)), "mc_decode_batch_host")
