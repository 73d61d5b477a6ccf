"""Seeded synthetic inputs: meshes, per-meshlet draws, camera poses, arrival times.

This module holds no part of the codec. It only makes the inputs that the
encoder, the decoder and the test oracle all consume, so it is the one module
shared by the product path and the tests. Every function is deterministic in
its seed (numpy PCG64).

Workloads (the paper's scanned meshes are not available; these stand in for
them, with the shapes the paper assumes: closed 2-manifold surfaces and
height-field scans, Sec. 5):

* ``grid_mesh``            64x64 quads -> 8,192 triangles, xyz jittered by
                           +-0.25 cell.
* ``surface_batch``        UV-spheres and tori, triangle counts log-uniform,
                           Gaussian noise along the normal (sigma = 1% of the
                           sphere radius or of the torus tube radius).
* ``height_field_disc``    jittered grid clipped to a disc, each quad split
                           along its Delaunay diagonal, heights from 4-octave
                           value noise, triangles tagged with one of three
                           120-degree sectors (meshlet-limit classes).
* ``vertex_attributes``    normals and texture coordinates (the rest of an
                           8-channel attribute vector).
* ``camera_poses``         row-major float32 view-projection matrices (OpenGL
                           clip conventions, 60 degree vertical FOV).
* ``poisson_arrivals``     request arrival times and mesh choices.

All meshes are wound counter-clockwise seen from outside (from +z for the
planar meshes).
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 20240406


@dataclass
class Mesh:
    """A triangle mesh: float32 positions [V,3], uint32 triangles [T,3]."""

    pos: np.ndarray
    tris: np.ndarray
    tri_class: np.ndarray | None = None  # uint8 [T] or None (one class)
    kind: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])

    @property
    def n_verts(self) -> int:
        return int(self.pos.shape[0])


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _orient_outward(pos: np.ndarray, tris: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Swap the last two corners of triangles whose normal points toward ``ref``
    (a per-triangle reference point inside the surface)."""
    a = pos[tris[:, 0]].astype(np.float64)
    b = pos[tris[:, 1]].astype(np.float64)
    c = pos[tris[:, 2]].astype(np.float64)
    n = np.cross(b - a, c - a)
    cen = (a + b + c) / 3.0
    flip = np.einsum("ij,ij->i", n, cen - ref) < 0
    out = tris.copy()
    out[flip, 1], out[flip, 2] = tris[flip, 2], tris[flip, 1]
    return out


def grid_mesh(n_quads: int = 64, jitter: float = 0.25, seed: int = SEED_BASE + 1) -> Mesh:
    """(n+1)^2 vertices on a unit-spaced grid, every quad split by the same
    diagonal, x/y/z each jittered uniformly by +-jitter cells."""
    rng = _rng(seed)
    n1 = n_quads + 1
    iy, ix = np.meshgrid(np.arange(n1), np.arange(n1), indexing="ij")
    pos = np.stack([ix, iy, np.zeros_like(ix)], -1).reshape(-1, 3).astype(np.float64)
    pos += rng.uniform(-jitter, jitter, size=pos.shape)
    qy, qx = np.meshgrid(np.arange(n_quads), np.arange(n_quads), indexing="ij")
    v00 = (qy * n1 + qx).reshape(-1)
    v10 = v00 + 1
    v01 = v00 + n1
    v11 = v01 + 1
    t = np.empty((n_quads * n_quads * 2, 3), np.uint32)
    t[0::2] = np.stack([v00, v10, v11], -1)
    t[1::2] = np.stack([v00, v11, v01], -1)
    return Mesh(pos.astype(np.float32), t, None, "grid", {"n_quads": n_quads, "seed": seed})


def uv_sphere(t_target: int, rng: np.random.Generator, radius: float = 1.0,
              noise: float = 0.01, center=(0.0, 0.0, 0.0)) -> Mesh:
    """UV-sphere with fan-capped poles: T = 2 * n_u * n_r exactly, where n_u
    is the number of segments and n_r the number of vertex rings."""
    n_u = max(3, int(round(math.sqrt(t_target))))
    n_r = max(2, int(round(t_target / (2 * n_u))))
    theta = np.pi * np.arange(1, n_r + 1) / (n_r + 1)
    phi = 2 * np.pi * np.arange(n_u) / n_u
    st, ct = np.sin(theta)[:, None], np.cos(theta)[:, None]
    ring = np.stack([st * np.cos(phi)[None, :], st * np.sin(phi)[None, :],
                     np.broadcast_to(ct, (n_r, n_u))], -1).reshape(-1, 3)
    unit = np.concatenate([[[0, 0, 1]], ring, [[0, 0, -1]]], 0)
    south = 1 + n_r * n_u
    j = np.arange(n_u)
    jn = (j + 1) % n_u

    def idx(i, jj):
        return 1 + i * n_u + jj

    parts = [np.stack([np.zeros(n_u, np.int64), idx(0, j), idx(0, jn)], -1)]
    if n_r > 1:
        i = np.arange(n_r - 1)[:, None]
        a, b = idx(i, j[None, :]), idx(i, jn[None, :])
        c, d = idx(i + 1, jn[None, :]), idx(i + 1, j[None, :])
        q = np.empty((n_r - 1, n_u, 2, 3), np.int64)
        q[:, :, 0] = np.stack([a, d, c], -1)
        q[:, :, 1] = np.stack([a, c, b], -1)
        parts.append(q.reshape(-1, 3))
    parts.append(np.stack([np.full(n_u, south), idx(n_r - 1, jn), idx(n_r - 1, j)], -1))
    tris = np.concatenate(parts, 0).astype(np.uint32)
    r = radius + rng.normal(0.0, noise * radius, size=unit.shape[0])
    pos = unit * r[:, None] + np.asarray(center, np.float64)[None, :]
    tris = _orient_outward(pos, tris, np.asarray(center, np.float64)[None, :])
    return Mesh(pos.astype(np.float32), tris, None, "sphere",
                {"n_u": n_u, "n_r": n_r, "radius": radius, "center": tuple(center)})


def torus(t_target: int, rng: np.random.Generator, major: float = 1.0, minor: float = 1.0 / 3.0,
          noise: float = 0.01, center=(0.0, 0.0, 0.0)) -> Mesh:
    """Torus around the z axis: T = 2 * n_u * n_v exactly."""
    n_u = max(3, int(round(math.sqrt(1.5 * t_target))))
    n_v = max(3, int(round(t_target / (2 * n_u))))
    phi = 2 * np.pi * np.arange(n_u) / n_u
    psi = 2 * np.pi * np.arange(n_v) / n_v
    P, S = np.meshgrid(phi, psi, indexing="ij")
    nrm = np.stack([np.cos(S) * np.cos(P), np.cos(S) * np.sin(P), np.sin(S)], -1).reshape(-1, 3)
    axis = np.stack([np.cos(P), np.sin(P), np.zeros_like(P)], -1).reshape(-1, 3) * major
    rr = minor + rng.normal(0.0, noise * minor, size=nrm.shape[0])
    cen = np.asarray(center, np.float64)[None, :]
    pos = axis + nrm * rr[:, None] + cen
    i = np.arange(n_u)[:, None]
    jj = np.arange(n_v)[None, :]
    a = i * n_v + jj
    b = ((i + 1) % n_u) * n_v + jj
    c = ((i + 1) % n_u) * n_v + (jj + 1) % n_v
    d = i * n_v + (jj + 1) % n_v
    q = np.empty((n_u, n_v, 2, 3), np.int64)
    q[:, :, 0] = np.stack([a, b, c], -1)
    q[:, :, 1] = np.stack([a, c, d], -1)
    tris = q.reshape(-1, 3).astype(np.uint32)
    # reference point for orientation: the tube centre nearest to each triangle
    cenv = pos[tris].mean(1) - cen
    ang = np.arctan2(cenv[:, 1], cenv[:, 0])
    ref = np.stack([np.cos(ang), np.sin(ang), np.zeros_like(ang)], -1) * major + cen
    tris = _orient_outward(pos, tris, ref)
    return Mesh(pos.astype(np.float32), tris, None, "torus",
                {"n_u": n_u, "n_v": n_v, "major": major, "minor": minor, "center": tuple(center)})


def _lattice_center(i: int, side: int, spacing: float):
    x, y, z = i % side, (i // side) % side, i // (side * side)
    return (x * spacing, y * spacing, z * spacing)


def surface_batch(n_meshes: int = 256, t_lo: int = 10_000, t_hi: int = 200_000,
                  seed: int = SEED_BASE + 2, min_total_tris: int = 0,
                  spacing: float = 3.0, side: int | None = None) -> list[Mesh]:
    """Alternating UV-spheres (even index) and tori (odd index) with triangle
    counts log-uniform in [t_lo, t_hi], placed on a cubic lattice.

    With ``min_total_tris`` > 0 meshes keep being added (same seed stream) until
    the total triangle count reaches it, even past ``n_meshes``."""
    rng = _rng(seed)
    if side is None:
        est = max(n_meshes, 1)
        if min_total_tris:
            est = max(est, int(min_total_tris / (0.5 * (t_lo + t_hi) / math.log(t_hi / t_lo))) + 8)
        side = max(1, int(math.ceil(est ** (1.0 / 3.0))))
    out: list[Mesh] = []
    total = 0
    i = 0
    while i < n_meshes or total < min_total_tris:
        t = int(round(math.exp(rng.uniform(math.log(t_lo), math.log(t_hi)))))
        c = _lattice_center(i, side, spacing)
        m = uv_sphere(t, rng, center=c) if i % 2 == 0 else torus(t, rng, center=c)
        m.meta["index"] = i
        out.append(m)
        total += m.n_tris
        i += 1
    return out


def _hash32(ix: np.ndarray, iy: np.ndarray, octave: int, seed: int) -> np.ndarray:
    """32-bit lattice hash (xor-shift-multiply mixer) -> uint32."""
    h = (ix.astype(np.uint32) * np.uint32(0x8DA6B343)) ^ (iy.astype(np.uint32) * np.uint32(0xD8163841))
    h ^= np.uint32((octave * 0xCB1AB31F + seed) & 0xFFFFFFFF)
    h ^= h >> np.uint32(16)
    h *= np.uint32(0x7FEB352D)
    h ^= h >> np.uint32(15)
    h *= np.uint32(0x846CA68B)
    h ^= h >> np.uint32(16)
    return h


def value_noise(x: np.ndarray, y: np.ndarray, seed: int, octaves: int = 4,
                base_period: float = 512.0, amplitude: float = 64.0) -> np.ndarray:
    """Sum of ``octaves`` layers of lattice value noise with smoothstep
    interpolation; each octave doubles the frequency and halves the amplitude.
    Evaluated in parallel chunks (pointwise, so the result does not depend on
    the chunking)."""
    n = x.shape[0]
    chunk = 1 << 20
    if n <= chunk:
        return _value_noise(x, y, seed, octaves, base_period, amplitude)
    out = np.empty(n, np.float64)

    def run(i):
        sl = slice(i, min(n, i + chunk))
        out[sl] = _value_noise(x[sl], y[sl], seed, octaves, base_period, amplitude)
    with ThreadPoolExecutor(os.cpu_count() or 4) as ex:
        list(ex.map(run, range(0, n, chunk)))
    return out


def _value_noise(x, y, seed, octaves, base_period, amplitude):
    out = np.zeros(x.shape, np.float64)
    freq, amp = 1.0 / base_period, amplitude
    with np.errstate(over="ignore"):
        for o in range(octaves):
            X, Y = x * freq, y * freq
            x0, y0 = np.floor(X), np.floor(Y)
            fx, fy = X - x0, Y - y0
            sx, sy = fx * fx * (3 - 2 * fx), fy * fy * (3 - 2 * fy)
            x0i, y0i = x0.astype(np.int64), y0.astype(np.int64)
            inv = 1.0 / 4294967296.0
            v00 = _hash32(x0i, y0i, o, seed) * inv
            v10 = _hash32(x0i + 1, y0i, o, seed) * inv
            v01 = _hash32(x0i, y0i + 1, o, seed) * inv
            v11 = _hash32(x0i + 1, y0i + 1, o, seed) * inv
            top = v00 + (v10 - v00) * sx
            bot = v01 + (v11 - v01) * sx
            out += amp * (top + (bot - top) * sy)
            freq *= 2.0
            amp *= 0.5
    return out


SECTOR_LIMITS = ((64, 126), (128, 128), (256, 256))


def height_field_disc(total_tris: int = 50_000_000, seed: int = SEED_BASE + 3,
                      jitter: float = 0.25) -> Mesh:
    """Jittered unit grid clipped to a disc (quads whose four corners lie in
    the disc), each quad split along its Delaunay diagonal, z from 4-octave
    value noise. ``tri_class`` = 120-degree sector of the quad centre (0,1,2).

    The diagonal v00-v11 is taken unless v01 lies strictly inside the
    circumcircle of (v00, v10, v11) (the in-circle determinant, in FP64 on the
    FP32 xy positions, relative to v01).  With jitter <= 0.25 no other point
    comes inside those circles, so the triangles are exactly the Delaunay
    triangles of the point set that fall in the clipped region (up to the
    rounding of quads within about 1e-12 of cocircular, where either diagonal
    is Delaunay to that precision)."""
    rng = _rng(seed)
    radius = math.sqrt(total_tris / (2.0 * math.pi))
    rc = int(math.ceil(radius)) + 1
    n1 = 2 * rc + 1
    g = np.arange(-rc, rc + 1)
    inside = (g[:, None] ** 2 + g[None, :] ** 2) <= radius * radius  # [iy, ix]
    q_ok = inside[:-1, :-1] & inside[:-1, 1:] & inside[1:, :-1] & inside[1:, 1:]
    used = np.zeros_like(inside)
    used[:-1, :-1] |= q_ok
    used[:-1, 1:] |= q_ok
    used[1:, :-1] |= q_ok
    used[1:, 1:] |= q_ok
    vid = np.full(inside.shape, -1, np.int64)
    uy, ux = np.nonzero(used)
    nv = uy.shape[0]
    vid[uy, ux] = np.arange(nv)
    px = g[ux].astype(np.float64) + rng.uniform(-jitter, jitter, nv)
    py = g[uy].astype(np.float64) + rng.uniform(-jitter, jitter, nv)
    pz = value_noise(px, py, seed)
    pos = np.stack([px, py, pz], -1).astype(np.float32)
    del px, py, pz
    qy, qx = np.nonzero(q_ok)
    v00 = vid[qy, qx]
    v10 = vid[qy, qx + 1]
    v01 = vid[qy + 1, qx]
    v11 = vid[qy + 1, qx + 1]
    p = pos[:, :2].astype(np.float64)
    d = p[v01]
    ax, ay = p[v00, 0] - d[:, 0], p[v00, 1] - d[:, 1]
    bx, by = p[v10, 0] - d[:, 0], p[v10, 1] - d[:, 1]
    cx, cy = p[v11, 0] - d[:, 0], p[v11, 1] - d[:, 1]
    incircle = ((ax * ax + ay * ay) * (bx * cy - cx * by) - (bx * bx + by * by) * (ax * cy - cx * ay)
                + (cx * cx + cy * cy) * (ax * by - bx * ay))
    main = incircle <= 0.0  # v01 not inside the circle of the counter-clockwise (v00, v10, v11)
    del p, d, ax, ay, bx, by, cx, cy, incircle
    nq = qy.shape[0]
    t = np.empty((nq, 2, 3), np.int64)
    t[:, 0] = np.where(main[:, None], np.stack([v00, v10, v11], -1), np.stack([v00, v10, v01], -1))
    t[:, 1] = np.where(main[:, None], np.stack([v00, v11, v01], -1), np.stack([v10, v11, v01], -1))
    tris = t.reshape(-1, 3).astype(np.uint32)
    ang = np.arctan2(g[qy] + 0.5, g[qx] + 0.5) + np.pi
    sector = np.minimum((ang / (2 * np.pi / 3)).astype(np.int64), 2).astype(np.uint8)
    tri_class = np.repeat(sector, 2)
    return Mesh(pos, tris, tri_class, "height_field",
                {"radius": radius, "seed": seed, "limits": SECTOR_LIMITS})


def vertex_attributes(mesh: Mesh) -> np.ndarray:
    """float32 [V, 5] per-vertex attributes beyond the position, the rest of
    an 8-channel attribute vector (position, normal, texture coordinate):
    unit normal (area-weighted sum of the incident triangle normals) and a
    texture coordinate -- spherical about the mesh's bounding-box centre for
    spheres and tori, planar (x, y scaled to [0, 1]) otherwise."""
    p = mesh.pos.astype(np.float64)
    t = mesh.tris.astype(np.int64)
    fn = np.cross(p[t[:, 1]] - p[t[:, 0]], p[t[:, 2]] - p[t[:, 0]])
    n = np.zeros_like(p)
    for c in range(3):
        np.add.at(n, t[:, c], fn)
    ln = np.linalg.norm(n, axis=1)
    n = np.where(ln[:, None] > 0, n / np.maximum(ln, 1e-300)[:, None], np.array([0.0, 0.0, 1.0]))
    lo, hi = p.min(0), p.max(0)
    if mesh.kind in ("sphere", "torus"):
        d = p - 0.5 * (lo + hi)
        u = np.arctan2(d[:, 1], d[:, 0]) / (2 * np.pi) + 0.5
        v = np.arccos(np.clip(d[:, 2] / np.maximum(np.linalg.norm(d, axis=1), 1e-300), -1, 1)) / np.pi
    else:
        ext = np.maximum(hi - lo, 1e-300)
        u, v = (p[:, 0] - lo[0]) / ext[0], (p[:, 1] - lo[1]) / ext[1]
    return np.concatenate([n, u[:, None], v[:, None]], 1).astype(np.float32)


def meshlet_bits(n: int, seed: int, choices=(12, 16, 20)) -> np.ndarray:
    """Position bit width per meshlet, drawn uniformly from ``choices``."""
    return np.asarray(choices, np.uint8)[_rng(seed).integers(0, len(choices), n)]


def meshlet_permutation(n: int, seed: int) -> np.ndarray:
    """A seeded permutation used to shuffle meshlets inside a batch."""
    return _rng(seed).permutation(n).astype(np.uint32)


def _look_at(eye, target, up):
    f = target - eye
    f /= np.linalg.norm(f)
    if abs(np.dot(f, up)) > 0.99:
        up = np.array([0.0, 1.0, 0.0])
    s = np.cross(f, up)
    s /= np.linalg.norm(s)
    u = np.cross(s, f)
    m = np.eye(4)
    m[0, :3], m[1, :3], m[2, :3] = s, u, -f
    m[0, 3], m[1, 3], m[2, 3] = -np.dot(s, eye), -np.dot(u, eye), np.dot(f, eye)
    return m


def _perspective(fovy_deg, aspect, near, far):
    f = 1.0 / math.tan(math.radians(fovy_deg) / 2.0)
    m = np.zeros((4, 4))
    m[0, 0] = f / aspect
    m[1, 1] = f
    m[2, 2] = (far + near) / (near - far)
    m[2, 3] = 2 * far * near / (near - far)
    m[3, 2] = -1.0
    return m


def camera_poses(n: int, center, radius: float, seed: int = SEED_BASE + 4,
                 fovy_deg: float = 60.0, distance: float = 1.5, jitter: float = 0.1) -> np.ndarray:
    """``n`` row-major float32 view-projection matrices [n,16]: eye uniformly on
    a sphere of ``distance * radius`` around ``center``, look-at point jittered
    by N(0, jitter * radius), aspect 1, near 0.01 R, far 4 R, clip = M [x y z 1]^T."""
    rng = _rng(seed)
    center = np.asarray(center, np.float64)
    out = np.empty((n, 16), np.float32)
    proj = _perspective(fovy_deg, 1.0, 0.01 * radius, 4.0 * radius)
    for i in range(n):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        eye = center + distance * radius * d
        tgt = center + rng.normal(0.0, jitter * radius, 3)
        out[i] = (proj @ _look_at(eye, tgt, np.array([0.0, 0.0, 1.0]))).reshape(-1)
    return out


def scene_views(meshes, n_views: int, seed: int) -> np.ndarray:
    """n_views camera poses around a batch of meshes: the eye on a sphere of
    1.5 times the radius of the batch's bounding box around its centre
    (camera_poses)."""
    lo = np.min([m.pos.min(0) for m in meshes], 0).astype(np.float64)
    hi = np.max([m.pos.max(0) for m in meshes], 0).astype(np.float64)
    center = 0.5 * (lo + hi)
    radius = float(np.linalg.norm(hi - lo) / 2)
    return camera_poses(n_views, center, radius, seed)


def poisson_arrivals(rate: float, duration: float, n_choices: int, seed: int):
    """Arrival times (s) of a Poisson process of ``rate`` per second over
    ``duration`` seconds, and a uniformly drawn mesh index per arrival."""
    rng = _rng(seed)
    n_est = int(rate * duration * 1.2 + 100)
    t = np.cumsum(rng.exponential(1.0 / rate, n_est))
    while t[-1] < duration:
        t = np.concatenate([t, t[-1] + np.cumsum(rng.exponential(1.0 / rate, n_est))])
    t = t[t < duration]
    return t, rng.integers(0, n_choices, t.shape[0]).astype(np.int64)
