"""The byte counts behind the bench's roofline (workloads.algorithmic_bytes,
workloads.cull_bytes), pinned on CPU against quantities fixed elsewhere: the
encoder's payload size and padding, the descriptor totals, and views whose
meshlet tests are known in advance (everything inside / everything outside
the frustum)."""
import numpy as np

from paper_2404_06359_gb300 import meshgen as G
from paper_2404_06359_gb300 import workloads as W


def _blob():
    rng = np.random.Generator(np.random.PCG64(123))
    meshes = [G.uv_sphere(6_000, rng), G.torus(4_000, rng)]
    return W.encode_meshes(meshes), meshes


def test_algorithmic_bytes_matches_the_blob():
    blob, _ = _blob()
    s, a = blob.stats(), blob.arrays()
    b = W.algorithmic_bytes(s, a["desc"])
    M = s["n_meshlets"]
    # payload words without block padding = payload bytes - padding
    assert b["read"] == 32 * M + s["payload_bytes"] - b["padding"] + 32 * s["n_grids"]
    assert b["write"] == 15 * s["total_tris"] + 12 * s["total_verts"]
    assert W.algorithmic_bytes(s, a["desc"], global_=False)["write"] == 3 * s["total_tris"] + 12 * s["total_verts"]


def _ortho(scale, shift):
    m = np.eye(4, dtype=np.float32) * np.float32(scale)
    m[3, 3] = 1.0
    m[:3, 3] = shift
    return m.reshape(16)


def test_cull_bytes_all_in_and_all_out():
    blob, meshes = _blob()
    s, a = blob.stats(), blob.arrays()
    pts = np.concatenate([m.pos for m in meshes]).astype(np.float64)
    c = 0.5 * (pts.min(0) + pts.max(0))
    r = float(np.abs(pts - c).max())
    inside = _ortho(0.5 / r, -0.5 / r * c)          # every point within |x|, |y|, |z| <= 0.5 w
    outside = _ortho(0.5 / r, -0.5 / r * c + 10.0)  # every point beyond x = w
    fixed = 64 * s["n_meshlets"] + 32 * s["n_grids"]
    payload = s["payload_bytes"] - W.algorithmic_bytes(s, a["desc"])["padding"]
    every = payload + 12 * s["total_verts"]
    n_kept = 1000
    assert W.cull_bytes(s, a, np.stack([outside]), np.array([0]), cones=True) == fixed
    assert W.cull_bytes(s, a, np.stack([inside]), np.array([n_kept]), cones=True) == fixed + every + 12 * n_kept
    # two views per launch: the input is counted once, each view's survivors apart
    two = W.cull_bytes(s, a, np.stack([inside, outside]), np.array([n_kept, 0]), cones=True,
                       views_per_launch=2)
    assert two == fixed + every + 12 * n_kept
    # one view per launch: the mean of the two launches
    one = W.cull_bytes(s, a, np.stack([inside, outside]), np.array([n_kept, 0]), cones=True)
    assert one == fixed + (every + 12 * n_kept) // 2
