"""The library's host encoder (C++, multithreaded) against the oracle's plain C
encoder: both follow the same documented greedy rules, so for every input the
meshlet grouping and every byte of the blob must agree.  Also checks the C ABI
exports and argument errors (no GPU needed)."""
import re
import os

import numpy as np
import pytest

import oracle as O
from paper_2404_06359_gb300 import codec as mc
from paper_2404_06359_gb300 import meshgen as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cases():
    rng = np.random.Generator(np.random.PCG64(31))
    return {
        "grid_64_126": (G.grid_mesh(), [(64, 126)], 16, 0, False),
        "sphere_64_126": (G.uv_sphere(15_000, rng), [(64, 126)], 16, 0, False),
        "torus_128_128": (G.torus(12_000, rng), [(128, 128)], 16, 0, False),
        "sphere_256_256_log2": (G.uv_sphere(30_000, rng), [(256, 256)], 12, 1, False),
        "torus_3_8_b7": (G.torus(3_000, rng), [(8, 3)], 7, 1, False),
        "hf_mixed": (G.height_field_disc(40_000, seed=5), list(G.SECTOR_LIMITS), "mixed", 1, True),
        "torus_64_126_plain_gts": (G.torus(10_000, rng), [(64, 126)], 16, 2, False),
        "hf_mixed_plain_gts": (G.height_field_disc(20_000, seed=6), list(G.SECTOR_LIMITS), "mixed",
                               2, True),
    }


CASES = _cases()


@pytest.fixture(scope="module", params=list(CASES))
def both(request):
    mesh, lim, bits, mode, shuffle = CASES[request.param]
    m = mc.mc_meshletize(mesh.tris, mesh.n_verts, lim, mesh.tri_class, n_threads=4)
    n = m.count
    b = G.meshlet_bits(n, 9) if bits == "mixed" else bits
    order = G.meshlet_permutation(n, 10) if shuffle else None
    blob = mc.mc_encode(m, mesh.pos, b, mode, order, n_threads=4)
    mtri, mstart, ng = O.meshletize(mesh.tris, mesh.n_verts, np.asarray(lim).reshape(-1), mesh.tri_class)
    ob = O.encode(mesh.pos, mesh.tris, mtri, mstart, b if np.ndim(b) else np.full(mstart.size - 1, b),
                  mode, order)
    return request.param, mesh, m, blob, (mtri, mstart, ng), ob


def test_meshlet_grouping_identical(both):
    name, mesh, m, blob, (mtri, mstart, ng), ob = both
    tri, start = m.get()
    assert np.array_equal(start, mstart)
    assert np.array_equal(tri, mtri)


def test_blob_bytes_identical(both):
    name, mesh, m, blob, (mtri, mstart, ng), ob = both
    a = blob.arrays()
    assert np.array_equal(a["desc"], ob.desc)
    assert np.array_equal(a["grids"], ob.grids)
    assert a["payload"].size == ob.payload.size
    assert np.array_equal(a["payload"], ob.payload)
    assert np.array_equal(a["vertex_map"], ob.stats["vmap"])
    assert np.array_equal(a["cones"], ob.cones)
    s = blob.stats()
    assert s["restarts"] == ob.stats["restarts"]
    assert s["conn_bits"] == ob.stats["conn_bits"]
    assert s["total_tris"] == ob.stats["total_tris"] and s["total_verts"] == ob.stats["total_verts"]
    assert s["split_meshlets"] == s["n_meshlets"] - ng
    assert s["input_tris"] == mesh.n_tris


@pytest.mark.parametrize("mode,bits,abits", [(0, 16, 16), (1, 12, 10), (2, 16, 20)])
def test_attribute_channels_identical(mode, bits, abits):
    """Blocks with attribute words, records and grids: library == oracle,
    byte for byte, alone and concatenated."""
    rng = np.random.Generator(np.random.PCG64(8 + mode))
    meshes = [G.uv_sphere(6_000, rng), G.torus(5_000, rng), G.grid_mesh(12)]
    blobs, oblobs = [], []
    for i, mesh in enumerate(meshes):
        at = G.vertex_attributes(mesh)
        m = mc.mc_meshletize(mesh.tris, mesh.n_verts, [(64, 126)])
        blobs.append(mc.mc_encode(m, mesh.pos, bits, mode, mesh_id=i, attrs=at, attr_bits=abits))
        oblobs.append(O.encode_mesh(mesh, (64, 126), bits, mode, mesh_id=i, attrs=at, attr_bits=abits))
        a = blobs[-1].arrays()
        assert np.array_equal(a["payload"], oblobs[-1].payload)
        assert np.array_equal(a["attr_desc"], oblobs[-1].attrs["adesc"])
        assert np.array_equal(a["attr_grids"], oblobs[-1].attrs["agrids"])
        assert blobs[-1].stats()["n_attr"] == 5 and blobs[-1].stats()["attr_bits"] == abits
    a = mc.mc_blob_concat(blobs).arrays()
    ocat = O.concat(oblobs)
    assert np.array_equal(a["desc"], ocat.desc)
    assert np.array_equal(a["payload"], ocat.payload)
    assert np.array_equal(a["attr_desc"], ocat.attrs["adesc"])
    assert np.array_equal(a["attr_grids"], ocat.attrs["agrids"])


def test_concat_matches_oracle_concat():
    rng = np.random.Generator(np.random.PCG64(2))
    meshes = [G.uv_sphere(3000, rng), G.torus(2500, rng), G.grid_mesh(16)]
    blobs, oblobs = [], []
    for i, mesh in enumerate(meshes):
        m = mc.mc_meshletize(mesh.tris, mesh.n_verts, [(64, 126)])
        blobs.append(mc.mc_encode(m, mesh.pos, 16, 0, mesh_id=i))
        oblobs.append(O.encode_mesh(mesh, (64, 126), 16, 0, mesh_id=i))
    cat = mc.mc_blob_concat(blobs)
    ocat = O.concat(oblobs)
    a = cat.arrays()
    assert np.array_equal(a["desc"], ocat.desc)
    assert np.array_equal(a["payload"], ocat.payload)
    assert np.array_equal(a["grids"], ocat.grids)
    assert np.array_equal(a["cones"], ocat.cones)
    meshes_t = a["meshes"]
    assert [x["n_meshlets"] for x in meshes_t] == [b.n_meshlets for b in oblobs]
    assert meshes_t[1]["first_meshlet"] == oblobs[0].n_meshlets


def _header_functions():
    src = open(os.path.join(ROOT, "include", "meshlet_codec.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(mc_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_library_exports_every_header_function():
    lib = mc.lib()
    names = _header_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(mc.exported_names()) == names


def test_argument_errors_are_synchronous():
    tris = np.array([[0, 1, 2], [0, 0, 1]], np.uint32)       # repeated vertex
    with pytest.raises(mc.CodecError) as e:
        mc.mc_meshletize(tris, 3, [(64, 126)])
    assert e.value.status == 1
    with pytest.raises(mc.CodecError):
        mc.mc_meshletize(np.array([[0, 1, 5]], np.uint32), 3, [(64, 126)])   # index >= n_verts
    with pytest.raises(mc.CodecError):
        mc.mc_meshletize(np.array([[0, 1, 2]], np.uint32), 3, [(2, 126)])    # V~ < 3
    m = mc.mc_meshletize(np.array([[0, 1, 2]], np.uint32), 3, [(64, 126)])
    with pytest.raises(mc.CodecError):
        mc.mc_encode(m, np.zeros((3, 3), np.float32), 33)                     # b > 32
    with pytest.raises(mc.CodecError):
        mc.mc_encode(m, np.zeros((3, 3), np.float32), 16, order=np.array([1], np.uint32))
    assert mc.mc_status_string(3) == "MC_ERR_CORRUPT"
    assert mc.mc_scratch_bytes() >= 12


def _canon(t: np.ndarray) -> np.ndarray:
    """Each triangle rotated so that its smallest index comes first (winding
    kept), rows sorted."""
    t = np.asarray(t, np.int64).reshape(-1, 3)
    r = np.argmin(t, 1)
    rot = np.stack([t[np.arange(len(t)), (r + k) % 3] for k in range(3)], 1)
    return rot[np.lexsort(rot.T[::-1])]


@pytest.mark.parametrize("name", ["sphere_64_126", "torus_128_128", "hf_mixed", "torus_64_126_plain_gts"])
def test_strip_search_bytes_identical_and_round_trip(name):
    """With the fewest-strips search on, both encoders still produce the same
    bytes, never more restarts than the greedy strips, and every meshlet still
    decodes to exactly its input triangles with their winding."""
    mesh, lim, bits, mode, shuffle = CASES[name]
    nodes = 50_000
    m = mc.mc_meshletize(mesh.tris, mesh.n_verts, lim, mesh.tri_class, n_threads=4)
    n = m.count
    b = G.meshlet_bits(n, 9) if bits == "mixed" else bits
    order = G.meshlet_permutation(n, 10) if shuffle else None
    blob = mc.mc_encode(m, mesh.pos, b, mode, order, n_threads=4, strip_search_nodes=nodes)
    greedy = mc.mc_encode(m, mesh.pos, b, mode, order, n_threads=4)
    mtri, mstart, _ = O.meshletize(mesh.tris, mesh.n_verts, np.asarray(lim).reshape(-1), mesh.tri_class)
    bb = b if np.ndim(b) else np.full(mstart.size - 1, b)
    ob = O.encode(mesh.pos, mesh.tris, mtri, mstart, bb, mode, order, search_nodes=nodes)
    a = blob.arrays()
    assert np.array_equal(a["desc"], ob.desc)
    assert np.array_equal(a["payload"], ob.payload)
    s, g = blob.stats(), greedy.stats()
    assert s["restarts"] == ob.stats["restarts"] <= g["restarts"]
    assert s["restarts"] < g["restarts"]  # the search improves some meshlets here
    loc, glob, _, _ = O.decode(ob, want_pos64=False)
    vmap = ob.stats["vmap"].astype(np.int64)
    tri = vmap[glob.astype(np.int64)]
    keep = (tri[:, 0] != tri[:, 1]) & (tri[:, 1] != tri[:, 2]) & (tri[:, 0] != tri[:, 2])
    assert np.array_equal(_canon(tri[keep]), _canon(mesh.tris))
    print(f"\n{name}: restarts {g['restarts']} -> {s['restarts']} with {nodes} search nodes per meshlet")
