"""The benchmark workloads, built through the library's own host encoder.

  cfg1  64x64-quad jittered grid, 8,192 triangles; meshlets 64/126; b = 16,
        w = 8; u8 local indices + FP32 positions; plain one-launch decode.
  cfg2  256 UV-spheres / tori, triangles log-uniform in [10k, 200k]
        (~16 M total), 1% normal noise; meshlets 64/126; b = 16, w = 8;
        u8 + u32 + FP32; one persistent launch.
  cfg3  disc height field of ~50 M triangles (4-octave value noise), three
        120-degree sectors meshletized at 64/126, 128/128 and 256/256;
        w = ceil(log2 V); b drawn from {12, 16, 20} per meshlet; meshlets
        shuffled; one persistent launch.
  cfg4  cfg2's generator grown to >= 50 M triangles on a 3-D lattice, fused
        decode + per-meshlet frustum / normal-cone and per-triangle back-face
        cull + compaction under 64 camera poses (60 degree FOV), one CUDA
        graph.
All inputs are seeded; see meshgen for the recipes.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import codec as mc
from . import meshgen as G

SEEDS = {1: G.SEED_BASE + 1, 2: G.SEED_BASE + 2, 3: G.SEED_BASE + 3, 4: G.SEED_BASE + 4}


def _threads():
    return os.cpu_count() or 4


def encode_meshes(meshes, limits=((64, 126),), pos_bits=16, reuse_mode=0, attrs=False,
                  strip_search_nodes: int = 0):
    """Encode each mesh (in parallel, one thread per mesh) and concatenate.
    attrs: also encode normals and texture coordinates (5 channels at 16
    bits, the rest of an 8-channel attribute vector); strip_search_nodes:
    node budget of the fewest-strips search per meshlet (0 = greedy strips)."""
    def enc(i):
        m = meshes[i]
        ml = mc.mc_meshletize(m.tris, m.n_verts, limits, m.tri_class, n_threads=1)
        at = G.vertex_attributes(m) if attrs else None
        return mc.mc_encode(ml, m.pos, pos_bits, reuse_mode, mesh_id=i, n_threads=1, attrs=at,
                            attr_bits=16, strip_search_nodes=strip_search_nodes)
    with ThreadPoolExecutor(_threads()) as ex:
        blobs = list(ex.map(enc, range(len(meshes))))
    return mc.mc_blob_concat(blobs)


def cfg1():
    mesh = G.grid_mesh(64, 0.25, SEEDS[1])
    ml = mc.mc_meshletize(mesh.tris, mesh.n_verts, [(64, 126)])
    return mc.mc_encode(ml, mesh.pos, 16, 0), [mesh]


def cfg2(rank: int = 0, plain_gts: bool = False, attrs: bool = False, strip_search_nodes: int = 0):
    """plain_gts: store every strip entry at 8 bits (Sec. 4.2) instead of the
    GTS-Reuse packing; attrs: 8-channel vertices (position, normal, texture
    coordinate); strip_search_nodes: fewest-strips search budget per meshlet."""
    meshes = G.surface_batch(256, 10_000, 200_000, SEEDS[2] + 1000 * rank)
    return encode_meshes(meshes, reuse_mode=2 if plain_gts else 0, attrs=attrs,
                         strip_search_nodes=strip_search_nodes), meshes


def cfg3(rank: int = 0, total_tris: int = 50_000_000, plain_gts: bool = False):
    seed = SEEDS[3] + 1000 * rank
    mesh = G.height_field_disc(total_tris, seed)
    ml = mc.mc_meshletize(mesh.tris, mesh.n_verts, list(G.SECTOR_LIMITS), mesh.tri_class)
    n = ml.count
    bits = G.meshlet_bits(n, seed + 1)
    order = G.meshlet_permutation(n, seed + 2)
    return mc.mc_encode(ml, mesh.pos, bits, 2 if plain_gts else 1, order), [mesh]


def cfg4(rank: int = 0, min_tris: int = 50_000_000, n_views: int = 64):
    meshes = G.surface_batch(256, 10_000, 200_000, SEEDS[2] + 1000 * rank, min_total_tris=min_tris)
    blob = encode_meshes(meshes)
    return blob, meshes, G.scene_views(meshes, n_views, SEEDS[4] + rank)


def _block_words(T, V, w, b):
    """Unpadded payload words per meshlet: L/R words, then increment and
    reuse words (GTS-Reuse) or one byte per triangle k >= 1 (plain GTS,
    w = 0), then the position words."""
    nw = (T + 31) // 32
    conn = np.where(w == 0, nw + (T + 2) // 4, 2 * nw + ((T + 2 - V) * w + 31) // 32)
    return conn + (3 * V * b + 31) // 32


def algorithmic_bytes(stats: dict, desc: np.ndarray, local=True, global_=True,
                      vertices: bool = False) -> dict:
    """Bytes one decode must move: compressed input read (descriptors, payload
    without block padding, grids; with attribute channels their words,
    records and grids) and decoded output written (vertices: 32 B per vertex
    instead of 12)."""
    w = desc.view(np.uint32).reshape(-1, 8)
    V = (w[:, 3] & 0xFFFF).astype(np.int64)
    T = (w[:, 3] >> 16).astype(np.int64)
    rw = (w[:, 4] & 0xFF).astype(np.int64)
    b = ((w[:, 4] >> 8) & 0xFF).astype(np.int64)
    n_attr, abits = int(stats.get("n_attr", 0)), int(stats.get("attr_bits", 0))
    words = _block_words(T, V, rw, b) + (n_attr * V * abits + 31) // 32
    read = 32 * w.shape[0] + 4 * int(words.sum()) + 32 * stats["n_grids"]
    if vertices:
        read += 32 * w.shape[0] + 48 * int(stats.get("n_meshes", 1))
    Tt, Vt = int(T.sum()), int(V.sum())
    write = (3 * Tt if local else 0) + (12 * Tt if global_ else 0) + (32 if vertices else 12) * Vt
    return {"read": read, "write": write, "total": read + write,
            "padding": 4 * int(((words + 3) // 4 * 4 - words).sum())}


def _eye64(vp: np.ndarray):
    """Camera position of a clip matrix (the point with clip x = y = w = 0),
    FP64, or None for an affine projection."""
    m = np.asarray(vp, np.float64).reshape(4, 4)
    a = m[[0, 1, 3], :3]
    if abs(np.linalg.det(a)) == 0.0:
        return None
    return np.linalg.solve(a, -m[[0, 1, 3], 3])


def _meshlet_passes(arrays: dict, vps: np.ndarray, cones: bool):
    """Per view, the meshlets that pass the meshlet tests -- quantisation box
    not wholly outside one clip plane, normal cone not facing away (both in
    FP64: exact decisions near a boundary do not matter for a byte count) --
    and each meshlet's payload words and vertex count."""
    w = arrays["desc"].view(np.uint32).reshape(-1, 8)
    V = (w[:, 3] & 0xFFFF).astype(np.int64)
    T = (w[:, 3] >> 16).astype(np.int64)
    rw = (w[:, 4] & 0xFF).astype(np.int64)
    b = ((w[:, 4] >> 8) & 0xFF).astype(np.int64)
    words = _block_words(T, V, rw, b)
    g = arrays["grids"].view(np.float32).reshape(-1, 8).astype(np.float64)
    gid = (w[:, 4] >> 16).astype(np.int64)
    L = w[:, 5:8].astype(np.float64)
    lo = g[gid, 0:3] + L * g[gid, 4:7]
    hi = g[gid, 0:3] + (L + (2.0 ** b - 1)[:, None]) * g[gid, 4:7]
    corners = np.stack([np.where(np.array([(k >> c) & 1 for c in range(3)], bool), hi, lo)
                        for k in range(8)], 1)                      # [M, 8, 3]
    ch = np.concatenate([corners, np.ones(corners.shape[:2] + (1,))], 2)
    if cones:
        cn = arrays["cones"].view(np.float32).reshape(-1, 8).astype(np.float64)
    keeps = []
    for vp in vps:
        clip = ch @ vp.reshape(4, 4).astype(np.float64).T           # [M, 8, 4]
        wv = clip[..., 3]
        out = np.zeros(w.shape[0], bool)
        for c in range(3):
            out |= (clip[..., c] > wv).all(1) | (clip[..., c] < -wv).all(1)
        eye = _eye64(vp) if cones else None
        if eye is not None:
            v = cn[:, 0:3] - eye
            d = (cn[:, 4:7] * v).sum(1)
            out |= (cn[:, 7] < 1) & (d >= cn[:, 7] * np.linalg.norm(v, axis=1) + cn[:, 3])
        keeps.append(~out)
    return keeps, words, V


def cull_bytes(stats: dict, arrays: dict, vps: np.ndarray, counts: np.ndarray,
               cones: bool = False, views_per_launch: int = 1) -> int:
    """Mean algorithmic bytes of one fused decode+cull launch over
    views_per_launch consecutive views: every descriptor and grid entry (and
    cone record, with cones), the payload and positions of the meshlets that
    pass the meshlet tests of at least one of the launch's views, and the
    surviving triangles of each view (12 B each)."""
    keeps, words, V = _meshlet_passes(arrays, vps, cones)
    M = words.size
    per_meshlet = 64 if cones else 32
    launches = []
    for v0 in range(0, len(vps), views_per_launch):
        k = np.zeros(M, bool)
        for kk in keeps[v0:v0 + views_per_launch]:
            k |= kk
        n = int(np.sum(np.asarray(counts[v0:v0 + views_per_launch], np.int64)))
        launches.append(4 * words[k].sum() + 12 * V[k].sum() + 12 * n)
    return int(per_meshlet * M + 32 * stats["n_grids"] + float(np.mean(launches)))
