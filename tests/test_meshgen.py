"""Pins of the synthetic input generators against independent references."""
import numpy as np
import pytest

from paper_2404_06359_gb300 import meshgen as G


def test_height_field_is_delaunay():
    """The height field's triangulation (its xy projection) is a subset of the
    Delaunay triangulation of its points computed by Qhull; what Qhull adds
    lies along the convex hull, outside the clipped disc of quads."""
    sp = pytest.importorskip("scipy.spatial")
    for seed in (1, 2):
        m = G.height_field_disc(30_000, seed=seed)
        d = sp.Delaunay(m.pos[:, :2].astype(np.float64))
        ref = set(map(tuple, np.sort(d.simplices, 1)))
        ours = set(map(tuple, np.sort(m.tris.astype(np.int64), 1)))
        assert ours <= ref, len(ours - ref)
        assert len(ours) > 0.95 * len(ref)


def test_height_field_winding_is_counter_clockwise():
    m = G.height_field_disc(20_000, seed=3)
    p = m.pos[:, :2].astype(np.float64)
    t = m.tris.astype(np.int64)
    a, b, c = p[t[:, 0]], p[t[:, 1]], p[t[:, 2]]
    cross = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    assert np.all(cross > 0)


def test_meshletizer_leaves_few_stranded_triangles():
    """The shared-edge pick of the greedy meshletizer keeps one- and
    two-triangle meshlets (triangles enclosed by full meshlets) rare, in the
    oracle and in the library alike; meshlets stay within their limits."""
    import oracle as O
    from paper_2404_06359_gb300 import codec as mc
    rng = np.random.Generator(np.random.PCG64(21))
    for mesh in (G.torus(40_000, rng), G.uv_sphere(60_000, rng)):
        ob = O.encode_mesh(mesh, (64, 126), 16, 0)
        f = ob.fields()
        T, V = f["Tp"].astype(np.int64), f["V"].astype(np.int64)
        assert np.mean(T <= 2) < 0.01, np.mean(T <= 2)
        assert V.max() <= 64 and T.max() <= 126
        ml = mc.mc_meshletize(mesh.tris, mesh.n_verts, [(64, 126)])
        lb = mc.mc_encode(ml, mesh.pos, 16, 0)
        assert lb.stats()["n_meshlets"] == ob.n_meshlets
