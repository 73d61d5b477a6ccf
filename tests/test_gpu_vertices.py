"""GPU parity of the full-vertex decode (positions + attribute channels,
8 FP32 per vertex) against the oracle, and of the other decode paths on
blobs whose payload blocks carry attribute words."""
import numpy as np
import pytest

import oracle as O
from paper_2404_06359_gb300 import codec as mc
from paper_2404_06359_gb300 import meshgen as G
from tests.gpu_util import assert_same_decode, device_batch_from_oracle, run_decode

pytestmark = pytest.mark.gpu


def _blob(n_attr: int, attr_bits: int, seed: int):
    rng = np.random.Generator(np.random.PCG64(seed))
    hf = G.height_field_disc(15_000, seed=seed)
    parts = []
    for i, (mesh, lim, bits, mode) in enumerate([
            (G.uv_sphere(8_000, rng), (64, 126), 16, 0),
            (G.torus(6_000, rng), (128, 128), 12, 1),
            (hf, np.array(G.SECTOR_LIMITS).reshape(-1), 20, 2),
            (G.grid_mesh(6), (8, 5), 7, 1)]):
        at = G.vertex_attributes(mesh)[:, 5 - n_attr:]  # the last n_attr channels
        parts.append(O.encode_mesh(mesh, lim, bits, mode, mesh_id=i, attrs=at, attr_bits=attr_bits))
    return O.concat(parts)


@pytest.fixture(scope="module", params=[(5, 16), (2, 10), (3, 24)])
def attr_blob(request):
    n_attr, bits = request.param
    return _blob(n_attr, bits, 90 + n_attr)


def _vertices(db, tuning=None):
    import torch
    T, V = db.stats["total_tris"], db.stats["total_verts"]
    loc = torch.full((3 * T,), 0xEE, dtype=torch.uint8, device="cuda")
    glob = torch.full((3 * T,), -1, dtype=torch.int32, device="cuda")
    vtx = torch.full((8 * V,), float("nan"), dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    scratch = mc.new_scratch()
    mc.mc_decode_batch_vertices(db, loc, glob, vtx, st, scratch, tuning)
    torch.cuda.synchronize()
    assert int(scratch.abs().sum()) == 0
    return loc.cpu().numpy(), glob.cpu().numpy(), vtx.cpu().numpy().reshape(-1, 8), int(st.item())


@pytest.mark.parametrize("tuning", [None, {"warps_per_cta": 4, "meshlets_per_grab": 1},
                                    {"warps_per_cta": 16, "meshlets_per_grab": 8},
                                    {"warps_per_cta": 8, "checked": 1}])
def test_vertices_vs_oracle(attr_blob, tuning):
    loc_ref, glob_ref, pos_ref, _ = O.decode(attr_blob)
    attr_ref = O.decode_attrs(attr_blob)
    n = attr_ref.shape[1]
    db = device_batch_from_oracle(attr_blob)
    loc, glob, vtx, st = _vertices(db, tuning)
    assert st == 0
    assert np.array_equal(loc.reshape(-1, 3), loc_ref)
    assert np.array_equal(glob.view(np.uint32).reshape(-1, 3), glob_ref)
    assert np.array_equal(vtx[:, :3].view(np.uint32), pos_ref.view(np.uint32))
    assert np.array_equal(vtx[:, 3:3 + n].view(np.uint32), attr_ref.view(np.uint32))
    assert np.all(vtx[:, 3 + n:] == 0.0)


def test_position_decode_skips_attribute_words(attr_blob):
    ref = O.decode(attr_blob)
    db = device_batch_from_oracle(attr_blob)
    for mode, tuning in (("batch", None), ("batch", {"checked": 1}), ("plain", {"checked": 1})):
        assert_same_decode(run_decode(db, mode, tuning), ref, f"{mode} {tuning}")


def test_cull_on_attribute_blob(attr_blob):
    import torch
    db = device_batch_from_oracle(attr_blob, cones=True)
    T, V = db.stats["total_tris"], db.stats["total_verts"]
    pts = O.decode(attr_blob)[2]
    c = 0.5 * (pts.min(0) + pts.max(0))
    r = float(np.linalg.norm(pts - c, axis=1).max())
    for vp in G.camera_poses(3, c, r, seed=93, distance=2.0):
        ref, _, _ = O.decode_cull(attr_blob, vp, cones=attr_blob.cones)
        tri = torch.zeros(3 * T + 3, dtype=torch.int32, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
        pos = torch.zeros(3 * V, dtype=torch.float32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        d_vp = torch.from_numpy(np.ascontiguousarray(vp, np.float32)).cuda()
        mc.mc_decode_cull(db, d_vp, tri, cnt, pos, st, mc.new_scratch())
        torch.cuda.synchronize()
        got = tri[: 3 * int(cnt.item())].cpu().numpy().view(np.uint32).reshape(-1, 3)
        assert int(st.item()) == 0
        assert np.array_equal(got[np.lexsort(got.T[::-1])], ref[np.lexsort(ref.T[::-1])])


def test_bad_attribute_grid_index_is_reported():
    blob = _blob(5, 16, 97)
    bad = dict(blob.attrs)
    bad["adesc"] = blob.attrs["adesc"].copy()
    bad["adesc"][3, 20] = 200  # grid id far beyond the grids
    broken = O.Blob(blob.desc, blob.payload, blob.grids, blob.stats, blob.cones, bad)
    db = device_batch_from_oracle(broken)
    _, _, _, st = _vertices(db)
    assert st & (1 << 3)


def test_vertices_need_attribute_channels():
    blob = O.encode_mesh(G.grid_mesh(8), (64, 126), 16, 0)
    db = device_batch_from_oracle(blob)
    with pytest.raises(mc.CodecError) as e:
        _vertices(db)
    assert e.value.status == 1
