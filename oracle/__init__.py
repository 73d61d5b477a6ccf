"""CPU oracle for GTS-Reuse meshlet compression -- TEST INFRASTRUCTURE ONLY.

A plain, slow, sequential restatement of Kuth et al., "Towards Practical
Meshlet Compression" (VMV 2024), written in C (``oracle/*.c``, see
``oracle.h`` for the format and the section each step follows) and wrapped
here with ctypes.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package.  It shares no code with
the library in ``paper_2404_06359_gb300``; the two meet only in the seeded
input generators (``paper_2404_06359_gb300.meshgen``) and in the blob format.

Pinned by ``tests/test_oracle_*.py`` against textbook strip/fan definitions,
brute-force enumeration, round trips to the input mesh, the paper's
degenerate-per-restart ratio (Tab. 1), exact size accounting and the
quantisation bounds of Sec. 4.4.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["meshletize.c", "stripify.c", "encode.c", "decode.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (no FP contraction, portable flags)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES] + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_LIB_PATH):
        if os.path.getmtime(_LIB_PATH) >= max(os.path.getmtime(s) for s in srcs):
            return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-o", tmp] + [os.path.join(_HERE, s) for s in _SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Blob(C.Structure):
    _fields_ = [("n_meshlets", C.c_uint32), ("n_grids", C.c_uint32),
                ("payload_bytes", C.c_uint64), ("total_tris", C.c_uint64),
                ("total_verts", C.c_uint64), ("restarts", C.c_uint64),
                ("degenerates", C.c_uint64), ("conn_bits", C.c_uint64),
                ("reuse_entries", C.c_uint64), ("desc", C.POINTER(C.c_uint8)),
                ("payload", C.POINTER(C.c_uint8)), ("grids", C.POINTER(C.c_uint8)),
                ("vmap", C.POINTER(C.c_uint32)), ("cones", C.POINTER(C.c_uint8)),
                ("n_attr", C.c_uint32), ("attr_bits", C.c_uint32),
                ("adesc", C.POINTER(C.c_uint8)), ("agrids", C.POINTER(C.c_uint8))]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            P = C.c_void_p
            u32, u64 = C.c_uint32, C.c_uint64
            L.orc_meshletize.argtypes = [u32, P, u32, P, P, u32, P, P, P, P]
            L.orc_stripify.argtypes = [P, P, u32, u32, P, P, P, P, P]
            L.orc_min_strips.argtypes = [P, P, u32, u32, u32, P, P, P]
            L.orc_encode.argtypes = [P, u32, P, P, P, u32, P, u32, P, u32, P, u32, u32, u32,
                                     C.POINTER(C.POINTER(_Blob))]
            L.orc_decode_attrs.argtypes = [P, P, u32, P, u64, P, u32, u32, u32, u32, u32, P]
            L.orc_blob_free.argtypes = [C.POINTER(_Blob)]
            L.orc_blob_free.restype = None
            L.orc_dequant32.argtypes = [u32, C.c_float, C.c_float]
            L.orc_dequant32.restype = C.c_float
            L.orc_decode_meshlet.argtypes = [P, P, u64, P, u32, P, P, P]
            L.orc_decode.argtypes = [P, u32, P, u64, P, u32, u32, u32, P, P, P, P]
            L.orc_decode_cull.argtypes = [P, u32, P, u64, P, u32, u32, u32, P, P, P, P, P, P]
            L.orc_view_eye.argtypes = [P, P]
            L.orc_cone_test.argtypes = [P, P]
            _lib = L
        return _lib


class OracleError(RuntimeError):
    pass


def _check(rc: int, what: str):
    if rc != 0:
        raise OracleError(f"{what} failed with status {rc}")


def _p(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


# --------------------------------------------------------------------------
# blob container (the oracle's own; the library has a separate one)
# --------------------------------------------------------------------------
@dataclass
class Blob:
    desc: np.ndarray      # uint8 [M, 32]
    payload: np.ndarray   # uint8 [bytes]
    grids: np.ndarray     # uint8 [G, 32]
    stats: dict = field(default_factory=dict)
    cones: np.ndarray | None = None  # uint8 [M, 32] normal cones (format in oracle.h)
    # extra attribute channels: {"n_attr", "attr_bits", "adesc" uint8 [M,32], "agrids" uint8 [A,48]}
    attrs: dict | None = None

    @property
    def n_meshlets(self) -> int:
        return int(self.desc.shape[0])

    @property
    def n_grids(self) -> int:
        return int(self.grids.shape[0])

    def fields(self) -> dict:
        """Descriptor fields as numpy arrays (format in oracle.h)."""
        w = self.desc.view(np.uint32).reshape(-1, 8)
        return {
            "off16": w[:, 0], "vertex_base": w[:, 1], "tri_base": w[:, 2],
            "V": w[:, 3] & 0xFFFF, "Tp": w[:, 3] >> 16,
            "w": w[:, 4] & 0xFF, "b": (w[:, 4] >> 8) & 0xFF, "grid": w[:, 4] >> 16,
            "L": w[:, 5:8],
        }

    @property
    def total_tris(self) -> int:
        return int(self.fields()["Tp"].astype(np.int64).sum())

    @property
    def total_verts(self) -> int:
        return int(self.fields()["V"].astype(np.int64).sum())


def meshletize(tris: np.ndarray, n_verts: int, limits, tri_class: np.ndarray | None = None):
    """Greedy meshlets; returns (mtri uint32[T], mstart uint32[M+1], n_grown)."""
    tris = np.ascontiguousarray(tris, np.uint32)
    lim = np.ascontiguousarray(np.asarray(limits, np.uint32).reshape(-1))
    nt = tris.shape[0]
    cls = None if tri_class is None else np.ascontiguousarray(tri_class, np.uint8)
    mtri = np.zeros(nt, np.uint32)
    mstart = np.zeros(nt + 1, np.uint32)
    nm, ng = C.c_uint32(0), C.c_uint32(0)
    _check(lib().orc_meshletize(n_verts, _p(tris), nt, _p(cls), _p(lim), lim.size // 2,
                                _p(mtri), _p(mstart), C.byref(nm), C.byref(ng)), "orc_meshletize")
    return mtri, mstart[: nm.value + 1].copy(), ng.value


def stripify(tris: np.ndarray, ids: np.ndarray, search_nodes: int = 0):
    """Strip of tris[ids] (greedy; with search_nodes > 0, the fewest-strips
    cover found within that budget when it is better); returns (stream,
    flags, order, T', strips)."""
    tris = np.ascontiguousarray(tris, np.uint32)
    ids = np.ascontiguousarray(ids, np.uint32)
    T = ids.size
    stream = np.zeros(5 * T + 8, np.uint32)
    flags = np.zeros(5 * T + 8, np.uint8)
    order = np.zeros(T, np.uint32)
    tp, ns = C.c_uint32(0), C.c_uint32(0)
    _check(lib().orc_stripify(_p(tris), _p(ids), T, search_nodes, _p(stream), _p(flags), _p(order),
                              C.byref(tp), C.byref(ns)), "orc_stripify")
    return stream[: tp.value + 2].copy(), flags[: tp.value].copy(), order, tp.value, ns.value


def min_strips(tris: np.ndarray, ids: np.ndarray, greedy_strips: int, max_nodes: int = 2_000_000,
               best_found: bool = False):
    """(fewest strips or 0 when the search gave up after max_nodes nodes,
    lower bound[, fewest found within the budget]) for the triangles
    tris[ids] (orc_min_strips)."""
    tris = np.ascontiguousarray(tris, np.uint32)
    ids = np.ascontiguousarray(ids, np.uint32)
    mn, lo, bf = C.c_uint32(0), C.c_uint32(0), C.c_uint32(0)
    _check(lib().orc_min_strips(_p(tris), _p(ids), ids.size, greedy_strips, max_nodes,
                                C.byref(mn), C.byref(lo), C.byref(bf)), "orc_min_strips")
    return (mn.value, lo.value, bf.value) if best_found else (mn.value, lo.value)


def encode(pos: np.ndarray, tris: np.ndarray, mtri: np.ndarray, mstart: np.ndarray,
           bits, reuse_mode: int = 0, perm: np.ndarray | None = None, mesh_id: int = 0,
           attrs: np.ndarray | None = None, attr_bits: int = 16, search_nodes: int = 0) -> Blob:
    """attrs: optional float32 [n_verts, n_attr] extra attribute channels (n_attr <= 5);
    search_nodes: node budget of the fewest-strips search per meshlet (0 = greedy)."""
    pos = np.ascontiguousarray(pos, np.float32)
    at = None if attrs is None else np.ascontiguousarray(attrs, np.float32).reshape(pos.shape[0], -1)
    n_attr = 0 if at is None else at.shape[1]
    tris = np.ascontiguousarray(tris, np.uint32)
    nm = mstart.size - 1
    bits = np.ascontiguousarray(np.broadcast_to(np.asarray(bits, np.uint8), (nm,)))
    perm = None if perm is None else np.ascontiguousarray(perm, np.uint32)
    out = C.POINTER(_Blob)()
    _check(lib().orc_encode(_p(pos), pos.shape[0], _p(tris), _p(np.ascontiguousarray(mtri, np.uint32)),
                            _p(np.ascontiguousarray(mstart, np.uint32)), nm, _p(bits), reuse_mode,
                            _p(perm), mesh_id, _p(at), n_attr, attr_bits if n_attr else 0,
                            search_nodes, C.byref(out)), "orc_encode")
    b = out.contents
    try:
        desc = np.ctypeslib.as_array(b.desc, (b.n_meshlets * 32,)).copy().reshape(-1, 32) \
            if b.n_meshlets else np.zeros((0, 32), np.uint8)
        payload = np.ctypeslib.as_array(b.payload, (b.payload_bytes,)).copy() \
            if b.payload_bytes else np.zeros(0, np.uint8)
        grids = np.ctypeslib.as_array(b.grids, (b.n_grids * 32,)).copy().reshape(-1, 32) \
            if b.n_grids else np.zeros((0, 32), np.uint8)
        stats = {k: int(getattr(b, k)) for k in ("total_tris", "total_verts", "restarts",
                                                  "degenerates", "conn_bits", "reuse_entries")}
        stats["vmap"] = np.ctypeslib.as_array(b.vmap, (b.total_verts,)).copy() \
            if b.total_verts else np.zeros(0, np.uint32)
        cones = np.ctypeslib.as_array(b.cones, (b.n_meshlets * 32,)).copy().reshape(-1, 32) \
            if b.n_meshlets else np.zeros((0, 32), np.uint8)
        attr = None
        if b.n_attr:
            attr = {"n_attr": int(b.n_attr), "attr_bits": int(b.attr_bits),
                    "adesc": np.ctypeslib.as_array(b.adesc, (b.n_meshlets * 32,)).copy().reshape(-1, 32),
                    "agrids": np.ctypeslib.as_array(b.agrids, (48,)).copy().reshape(1, 48)}
    finally:
        lib().orc_blob_free(out)
    return Blob(desc, payload, grids, stats, cones, attr)


def encode_mesh(mesh, limits=(64, 126), bits=16, reuse_mode: int = 0, perm=None,
                mesh_id: int = 0, attrs: np.ndarray | None = None, attr_bits: int = 16,
                search_nodes: int = 0) -> Blob:
    """meshletize + encode of a ``meshgen.Mesh``; ``bits`` scalar or callable(n)->array."""
    lim = np.asarray(limits, np.uint32).reshape(-1)
    mtri, mstart, ng = meshletize(mesh.tris, mesh.n_verts, lim, mesh.tri_class)
    nm = mstart.size - 1
    b = bits(nm) if callable(bits) else np.full(nm, bits, np.uint8)
    p = perm(nm) if callable(perm) else perm
    blob = encode(mesh.pos, mesh.tris, mtri, mstart, b, reuse_mode, p, mesh_id, attrs, attr_bits,
                  search_nodes)
    blob.stats["grown_meshlets"] = ng
    blob.stats["input_tris"] = mesh.n_tris
    blob.stats["mtri"], blob.stats["mstart"] = mtri, mstart
    return blob


def concat(blobs: list[Blob]) -> Blob:
    """One batch from several single-mesh blobs (offsets rebased, mesh ids
    renumbered in list order)."""
    descs, pays, grids = [], [], []
    off16 = vb = tb = gb = 0
    stats = {k: 0 for k in ("total_tris", "total_verts", "restarts", "degenerates",
                            "conn_bits", "reuse_entries", "input_tris")}
    vmaps = []
    for i, b in enumerate(blobs):
        d = b.desc.copy().view(np.uint32).reshape(-1, 8)
        d[:, 0] += off16
        d[:, 1] += vb
        d[:, 2] += tb
        d[:, 4] = (d[:, 4] & 0xFFFF) | (((d[:, 4] >> 16) + gb) << 16)
        g = b.grids.copy().view(np.uint32).reshape(-1, 8)
        g[:, 7] = i
        descs.append(d.view(np.uint8).reshape(-1, 32))
        pays.append(b.payload)
        grids.append(g.view(np.uint8).reshape(-1, 32))
        f = b.fields()
        off16 += b.payload.size // 16
        vb += int(f["V"].astype(np.int64).sum())
        tb += int(f["Tp"].astype(np.int64).sum())
        gb += b.n_grids
        for k in stats:
            stats[k] += int(b.stats.get(k, 0))
        if "vmap" in b.stats:
            vmaps.append(b.stats["vmap"])
    if len(vmaps) == len(blobs):
        stats["vmap_per_mesh"] = vmaps
    cones = np.concatenate([b.cones for b in blobs]) \
        if all(b.cones is not None for b in blobs) else None
    attr = None
    if all(b.attrs is not None for b in blobs) and \
            len({(b.attrs["n_attr"], b.attrs["attr_bits"]) for b in blobs}) == 1:
        adescs, agrids, ag = [], [], 0
        for i, b in enumerate(blobs):
            a = b.attrs["adesc"].copy()
            gid = a[:, 20].astype(np.uint32) | (a[:, 21].astype(np.uint32) << 8)
            gid += ag
            a[:, 20], a[:, 21] = gid & 0xFF, gid >> 8
            g = b.attrs["agrids"].copy()
            g.view(np.uint32).reshape(-1, 12)[:, 11] = i
            adescs.append(a)
            agrids.append(g)
            ag += g.shape[0]
        attr = {"n_attr": blobs[0].attrs["n_attr"], "attr_bits": blobs[0].attrs["attr_bits"],
                "adesc": np.concatenate(adescs), "agrids": np.concatenate(agrids)}
    return Blob(np.concatenate(descs), np.concatenate(pays), np.concatenate(grids), stats, cones, attr)


def dequant32(g: int, G: float, D: float) -> float:
    return float(lib().orc_dequant32(int(g), float(np.float32(G)), float(np.float32(D))))


def decode_meshlet(blob: Blob, m: int):
    """(local uint8 [T',3], pos float32 [V,3], pos64 float64 [V,3]) of meshlet m."""
    f = blob.fields()
    tp, V = int(f["Tp"][m]), int(f["V"][m])
    loc = np.zeros(3 * 256, np.uint8)
    pos = np.zeros(3 * 256, np.float32)
    pos64 = np.zeros(3 * 256, np.float64)
    d = np.ascontiguousarray(blob.desc[m])
    _check(lib().orc_decode_meshlet(_p(d), _p(blob.payload), blob.payload.size, _p(blob.grids),
                                    blob.n_grids, _p(loc), _p(pos), _p(pos64)), "orc_decode_meshlet")
    return loc[: 3 * tp].reshape(-1, 3), pos[: 3 * V].reshape(-1, 3), pos64[: 3 * V].reshape(-1, 3)


def decode(blob: Blob, first: int = 0, count: int | None = None, want_pos64: bool = True):
    """Whole-batch outputs: local uint8 [T'_total,3], global uint32 [T'_total,3],
    pos float32 [V_total,3], pos64 float64 [V_total,3] (meshlets outside the
    range are left zero)."""
    if count is None:
        count = blob.n_meshlets - first
    T, V = blob.total_tris, blob.total_verts
    loc = np.zeros(3 * T, np.uint8)
    glob = np.zeros(3 * T, np.uint32)
    pos = np.zeros(3 * V, np.float32)
    pos64 = np.zeros(3 * V, np.float64) if want_pos64 else None
    _check(lib().orc_decode(_p(blob.desc), blob.n_meshlets, _p(blob.payload), blob.payload.size,
                            _p(blob.grids), blob.n_grids, first, count, _p(loc), _p(glob),
                            _p(pos), _p(pos64)), "orc_decode")
    return (loc.reshape(-1, 3), glob.reshape(-1, 3), pos.reshape(-1, 3),
            None if pos64 is None else pos64.reshape(-1, 3))


def decode_into(blob: Blob, first: int, count: int, loc: np.ndarray, glob: np.ndarray,
                pos: np.ndarray) -> None:
    """orc_decode of meshlets [first, first + count) into caller-owned
    whole-batch arrays (uint8 [3 T'_total], uint32 [3 T'_total], float32
    [3 V_total]).  ctypes releases the GIL during the call, so disjoint
    ranges may be decoded from several threads at once."""
    _check(lib().orc_decode(_p(blob.desc), blob.n_meshlets, _p(blob.payload), blob.payload.size,
                            _p(blob.grids), blob.n_grids, first, count, _p(loc), _p(glob),
                            _p(pos), None), "orc_decode")


def decode_cull_into(blob: Blob, vp: np.ndarray, first: int, count: int, cones, out: np.ndarray,
                     pos: np.ndarray, passed: np.ndarray | None = None) -> int:
    """orc_decode_cull of meshlets [first, first + count): survivors from
    out[0] (uint32, room for 3 T' of the range), positions into the
    whole-batch pos (float32 [3 V_total]), and, when given, passed[m] (uint8
    [M]) = 1 for each meshlet of the range that passes the meshlet tests;
    returns the survivor count.  Like decode_into, callable from several
    threads on disjoint ranges."""
    cnt = C.c_uint64(0)
    vp = np.ascontiguousarray(np.asarray(vp, np.float32).reshape(16))
    cn = None if cones is None else np.ascontiguousarray(np.asarray(cones, np.uint8).reshape(-1, 32))
    _check(lib().orc_decode_cull(_p(blob.desc), blob.n_meshlets, _p(blob.payload),
                                 blob.payload.size, _p(blob.grids), blob.n_grids, first, count,
                                 _p(vp), _p(cn), _p(out), C.byref(cnt), _p(pos), _p(passed)),
           "orc_decode_cull")
    return int(cnt.value)


def decode_attrs(blob: Blob, first: int = 0, count: int | None = None) -> np.ndarray:
    """float32 [V_total, n_attr] decoded attribute channels (meshlets outside
    the range left zero)."""
    a = blob.attrs
    if count is None:
        count = blob.n_meshlets - first
    out = np.zeros(blob.total_verts * a["n_attr"], np.float32)
    _check(lib().orc_decode_attrs(_p(blob.desc), _p(a["adesc"]), blob.n_meshlets, _p(blob.payload),
                                  blob.payload.size, _p(a["agrids"]), a["agrids"].shape[0],
                                  a["n_attr"], a["attr_bits"], first, count, _p(out)),
           "orc_decode_attrs")
    return out.reshape(-1, a["n_attr"])


def view_eye(vp: np.ndarray):
    """Camera position (float32 [3]) of a clip matrix, or None (orc_view_eye)."""
    vp = np.ascontiguousarray(np.asarray(vp, np.float32).reshape(16))
    eye = np.zeros(3, np.float32)
    return eye if lib().orc_view_eye(_p(vp), _p(eye)) else None


def cone_test(cone32: np.ndarray, eye: np.ndarray) -> bool:
    """True when the normal-cone record rejects its meshlet seen from eye."""
    c = np.ascontiguousarray(np.asarray(cone32, np.uint8).reshape(32))
    e = np.ascontiguousarray(np.asarray(eye, np.float32).reshape(3))
    return bool(lib().orc_cone_test(_p(c), _p(e)))


def decode_cull(blob: Blob, vp: np.ndarray, first: int = 0, count: int | None = None,
                cones: np.ndarray | None = None):
    """(survivor triples uint32 [n,3] in meshlet order, pos float32 [V_total,3],
    pass flags uint8 [M]).  cones (uint8 [M,32], e.g. blob.cones): also drop
    meshlets the normal-cone test rejects."""
    if count is None:
        count = blob.n_meshlets - first
    T, V = blob.total_tris, blob.total_verts
    out = np.zeros(3 * T + 3, np.uint32)
    pos = np.zeros(3 * V, np.float32)
    passed = np.zeros(blob.n_meshlets, np.uint8)
    cnt = C.c_uint64(0)
    vp = np.ascontiguousarray(np.asarray(vp, np.float32).reshape(16))
    cn = None if cones is None else np.ascontiguousarray(np.asarray(cones, np.uint8).reshape(-1, 32))
    if cn is not None and cn.shape[0] != blob.n_meshlets:
        raise ValueError("one cone record per meshlet expected")
    _check(lib().orc_decode_cull(_p(blob.desc), blob.n_meshlets, _p(blob.payload),
                                 blob.payload.size, _p(blob.grids), blob.n_grids, first, count,
                                 _p(vp), _p(cn), _p(out), C.byref(cnt), _p(pos), _p(passed)),
           "orc_decode_cull")
    return out[: 3 * cnt.value].reshape(-1, 3), pos.reshape(-1, 3), passed
