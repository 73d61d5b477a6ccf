"""Pins of the oracle's plain GTS mode (Sec. 4.2: one L/R bit and one stored
8-bit index per triangle, before the reuse packing of Sec. 4.3).

The two modes share the strips and the first-appearance numbering, so a
plain-GTS blob must decode to exactly what the GTS-Reuse blob of the same
meshlets decodes to (and the Reuse decode is pinned elsewhere by round trips
and brute force); its size follows from one bit plus one byte per triangle.
"""
import numpy as np
import pytest

import oracle as O
from paper_2404_06359_gb300 import meshgen as G


@pytest.fixture(scope="module")
def meshes():
    rng = np.random.Generator(np.random.PCG64(77))
    hf = G.height_field_disc(8_000, 123)
    hf.tri_class = None  # one meshlet class: the limits under test apply everywhere
    return [G.torus(12_000, rng), G.grid_mesh(32), G.uv_sphere(6_000, rng), hf]


@pytest.mark.parametrize("limits", [(64, 126), (128, 128), (256, 256)])
def test_plain_gts_decodes_like_reuse(meshes, limits):
    for mesh in meshes:
        a = O.encode_mesh(mesh, limits, 16, 0)
        b = O.encode_mesh(mesh, limits, 16, 2)
        assert np.all(b.fields()["w"] == 0)
        for x, y in zip(O.decode(a)[:3], O.decode(b)[:3]):
            assert np.array_equal(x, y)


def test_plain_gts_size_accounting(meshes):
    for mesh in meshes:
        b = O.encode_mesh(mesh, (64, 126), 16, 2)
        f = b.fields()
        tp, V = f["Tp"].astype(np.int64), f["V"].astype(np.int64)
        assert b.stats["conn_bits"] == int((tp + 8 * (tp - 1)).sum())
        nw = (tp + 31) // 32
        words = nw + (tp - 1 + 3) // 4 + (3 * V * 16 + 31) // 32
        assert b.payload.size == int(16 * ((words + 3) // 4).sum())
        # block offsets are the running sum of the padded blocks
        off = np.concatenate([[0], np.cumsum((words + 3) // 4)])[:-1]
        assert np.array_equal(f["off16"].astype(np.int64), off)
        # the paper's band for plain GTS is 9.4-9.6 bits per triangle
        assert 9.0 < b.stats["conn_bits"] / mesh.n_tris < 10.5


def test_plain_gts_rejects_an_entry_that_skips_a_vertex(meshes):
    b = O.encode_mesh(meshes[0], (64, 126), 16, 2)
    f = b.fields()
    m = int(np.argmax(f["Tp"]))
    tp = int(f["Tp"][m])
    nw = (tp + 31) // 32
    start = 16 * int(f["off16"][m]) + 4 * nw
    ent = b.payload[start:start + tp - 1]
    k = int(np.argmax(ent == ent.max()))       # first appearance of the largest vertex id
    bad = b.payload.copy()
    bad[start + k] = min(255, int(ent.max()) + 1)  # an id that was never introduced
    broken = O.Blob(b.desc, bad, b.grids)
    with pytest.raises(O.OracleError):
        O.decode_meshlet(broken, m)
