"""GPU parity of the multi-view fused cull on the other payload block forms:
12-bit positions with narrow reuse entries (the generic extraction path) and
plain GTS blocks with normal cones."""
import numpy as np
import pytest

import oracle as O
from paper_2404_06359_gb300 import codec as mc
from paper_2404_06359_gb300 import meshgen as G
from tests.gpu_util import device_batch_from_oracle
from tests.test_gpu_cull import _run_views, _sorted_rows

pytestmark = pytest.mark.gpu


def _generic_blob():
    meshes = G.surface_batch(n_meshes=6, t_lo=500, t_hi=3_000, seed=21)
    blob = O.concat([O.encode_mesh(m, (8, 8), 12, 1, mesh_id=i) for i, m in enumerate(meshes)])
    return blob, np.concatenate([m.pos for m in meshes])


def _plain_gts_blob():
    rng = np.random.Generator(np.random.PCG64(61))
    meshes = [G.uv_sphere(15_000, rng, noise=0.0), G.torus(12_000, rng, center=(2.5, 0, 0))]
    blob = O.concat([O.encode_mesh(m, (64, 126), 16, 2, mesh_id=i) for i, m in enumerate(meshes)])
    return blob, np.concatenate([m.pos for m in meshes])


@pytest.mark.parametrize("kind", ["generic", "plain_gts"])
def test_cull_views_other_block_forms(kind):
    """The multi-view cull on 12-bit positions with 3-bit reuse entries (the
    generic extraction path) and on plain GTS blocks with cones: per view the
    oracle's survivors, positions of meshlets passing any view to 0 ulp."""
    from tests.gpu_util import block_words_max
    blob, pts = _generic_blob() if kind == "generic" else _plain_gts_blob()
    f = blob.fields()
    cones = kind == "plain_gts"
    if kind == "generic":
        assert int(f["w"].max()) < 8 and int(f["b"].max()) == 12
        db = mc.DeviceBatch.from_arrays(blob.desc, blob.payload, blob.grids, blob.total_tris,
                                        blob.total_verts, block_words_max(blob.desc), 256)
    else:
        db = device_batch_from_oracle(blob, cones=True)
    c = 0.5 * (pts.min(0) + pts.max(0))
    r = float(np.linalg.norm(pts - c, axis=1).max())
    views = G.camera_poses(5, c, r, seed=63, distance=2.0)
    ref_pos = O.decode(blob)[2]
    for tuning in (None, {"warps_per_cta": 8, "meshlets_per_grab": 1, "checked": 1}):
        outs, pos, st = _run_views(db, views, tuning)
        assert st == 0
        any_pass = np.zeros(f["V"].size, bool)
        for v in range(len(views)):
            ref, _, passed = O.decode_cull(blob, views[v], cones=blob.cones if cones else None)
            assert np.array_equal(_sorted_rows(outs[v]), _sorted_rows(ref)), (kind, v)
            any_pass |= passed.astype(bool)
        vm = np.repeat(any_pass, f["V"].astype(np.int64))
        assert np.array_equal(pos.reshape(-1, 3)[vm].view(np.uint32), ref_pos[vm].view(np.uint32))
