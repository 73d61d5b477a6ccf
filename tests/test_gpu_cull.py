"""GPU parity of the fused decode + cull + compaction kernel against the
oracle's sequential decode_cull, without and with the normal-cone meshlet
test: the surviving triangles are the same multiset (their order across
warps is not fixed), the count is exact and the positions of meshlets that
pass the meshlet tests match to 0 ulp."""
import numpy as np
import pytest

import oracle as O
from paper_2404_06359_gb300 import codec as mc
from paper_2404_06359_gb300 import meshgen as G
from tests.gpu_util import assert_same_decode, device_batch_from_oracle, run_decode

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scene():
    meshes = G.surface_batch(n_meshes=27, t_lo=2_000, t_hi=20_000, seed=7)
    blob = O.concat([O.encode_mesh(m, (64, 126), 16, 0, mesh_id=i) for i, m in enumerate(meshes)])
    pts = np.concatenate([m.pos for m in meshes])
    c = 0.5 * (pts.min(0) + pts.max(0))
    r = float(np.linalg.norm(pts - c, axis=1).max())
    vps = G.camera_poses(6, c, r, seed=8)
    return blob, vps


def _sorted_rows(t):
    t = np.asarray(t, np.int64).reshape(-1, 3)
    return t[np.lexsort(t.T[::-1])]


def _run(db, vp, tuning=None):
    import torch
    T, V = db.stats["total_tris"], db.stats["total_verts"]
    tri = torch.full((3 * T + 3,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    pos = torch.zeros(3 * V, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    scratch = mc.new_scratch()
    d_vp = torch.from_numpy(np.ascontiguousarray(vp, np.float32)).cuda()
    mc.mc_decode_cull(db, d_vp, tri, cnt, pos, st, scratch, tuning)
    torch.cuda.synchronize()
    assert int(scratch.abs().sum()) == 0
    n = int(cnt.item())
    return tri[: 3 * n].cpu().numpy().view(np.uint32), pos.cpu().numpy(), int(st.item())


@pytest.mark.parametrize("tuning", [None, {"warps_per_cta": 4}, {"warps_per_cta": 16, "checked": 1}])
def test_cull_vs_oracle(scene, tuning):
    blob, vps = scene
    db = device_batch_from_oracle(blob)
    f = blob.fields()
    frac = []
    for vp in vps:
        ref_tri, ref_pos, passed = O.decode_cull(blob, vp)
        tri, pos, st = _run(db, vp, tuning)
        assert st == 0
        assert tri.size == ref_tri.size, (tri.size // 3, ref_tri.shape[0])
        assert np.array_equal(_sorted_rows(tri), _sorted_rows(ref_tri))
        vm = np.repeat(passed, f["V"].astype(np.int64)).astype(bool)
        p = pos.reshape(-1, 3)[vm]
        assert np.array_equal(p.view(np.uint32), ref_pos[vm].view(np.uint32))
        frac.append(ref_tri.shape[0] / blob.stats["input_tris"])
    print("kept fraction per view", np.round(frac, 3))


def test_cull_graph_many_views(scene):
    import torch
    blob, vps = scene
    db = device_batch_from_oracle(blob)
    T, V = db.stats["total_tris"], db.stats["total_verts"]
    tri = torch.zeros(3 * T + 3, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(len(vps), dtype=torch.int32, device="cuda")
    pos = torch.zeros(3 * V, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    scratch = mc.new_scratch()
    d_vps = torch.from_numpy(np.ascontiguousarray(vps, np.float32)).cuda()
    g = mc.mc_graph_capture_cull(db, d_vps, len(vps), tri, cnt, pos, st, scratch)
    g.launch()
    torch.cuda.synchronize()
    counts = cnt.cpu().numpy()
    for i, vp in enumerate(vps):
        ref_tri, _, _ = O.decode_cull(blob, vp)
        assert counts[i] == ref_tri.shape[0]
    last_ref, _, _ = O.decode_cull(blob, vps[-1])
    got = tri[: 3 * counts[-1]].cpu().numpy().view(np.uint32)
    assert np.array_equal(_sorted_rows(got), _sorted_rows(last_ref))
    assert int(st.item()) == 0 and int(scratch.abs().sum()) == 0


@pytest.mark.parametrize("tuning", [None, {"meshlets_per_grab": 1}, {"warps_per_cta": 8, "meshlets_per_grab": 16}])
def test_cull_small_meshlets_generic_path(tuning):
    """Meshlets of at most 8 vertices / 8 triangles with 12-bit positions and
    3-bit reuse entries (the kernel's generic bit-extraction path), declared
    against a 256-triangle bound: a warp's survivor buffer then fills up by
    its meshlet count (32 sources) rather than by its triangle capacity."""
    import torch
    meshes = G.surface_batch(n_meshes=6, t_lo=500, t_hi=3_000, seed=21)
    blob = O.concat([O.encode_mesh(m, (8, 8), 12, 1, mesh_id=i) for i, m in enumerate(meshes)])
    f = blob.fields()
    assert int(f["w"].max()) < 8 and int(f["b"].max()) == 12
    from tests.gpu_util import block_words_max
    db = mc.DeviceBatch.from_arrays(blob.desc, blob.payload, blob.grids, blob.total_tris,
                                    blob.total_verts, block_words_max(blob.desc), 256)
    pts = np.concatenate([m.pos for m in meshes])
    c = 0.5 * (pts.min(0) + pts.max(0))
    r = float(np.linalg.norm(pts - c, axis=1).max())
    for vp in G.camera_poses(3, c, r, seed=22):
        ref_tri, ref_pos, passed = O.decode_cull(blob, vp)
        tri, pos, st = _run(db, vp, tuning)
        assert st == 0
        assert np.array_equal(_sorted_rows(tri), _sorted_rows(ref_tri))
        vm = np.repeat(passed, f["V"].astype(np.int64)).astype(bool)
        assert np.array_equal(pos.reshape(-1, 3)[vm].view(np.uint32), ref_pos[vm].view(np.uint32))
    torch.cuda.synchronize()


@pytest.fixture(scope="module")
def smooth_scene():
    """Noise-free spheres and tori: narrow normal cones, so the cone test
    drops a large share of the meshlets."""
    rng = np.random.Generator(np.random.PCG64(31))
    meshes = []
    for i in range(12):
        c = (3.0 * (i % 3), 3.0 * ((i // 3) % 2), 3.0 * (i // 6))
        t = int(rng.integers(5_000, 40_000))
        meshes.append(G.uv_sphere(t, rng, noise=0.0, center=c) if i % 2 == 0
                      else G.torus(t, rng, noise=0.0, center=c))
    blob = O.concat([O.encode_mesh(m, (64, 126), 16, 0, mesh_id=i) for i, m in enumerate(meshes)])
    pts = np.concatenate([m.pos for m in meshes])
    c = 0.5 * (pts.min(0) + pts.max(0))
    r = float(np.linalg.norm(pts - c, axis=1).max())
    return blob, G.camera_poses(5, c, r, seed=32, distance=2.0)


@pytest.mark.parametrize("tuning", [None, {"warps_per_cta": 8, "meshlets_per_grab": 16},
                                    {"warps_per_cta": 4, "meshlets_per_grab": 3, "checked": 1}])
@pytest.mark.parametrize("which", ["scene", "smooth_scene"])
def test_cull_with_cones_vs_oracle(request, which, tuning):
    blob, vps = request.getfixturevalue(which)
    db = device_batch_from_oracle(blob, cones=True)
    f = blob.fields()
    rejected = 0
    for vp in vps:
        ref_tri, ref_pos, passed = O.decode_cull(blob, vp, cones=blob.cones)
        _, _, passed_plain = O.decode_cull(blob, vp)
        tri, pos, st = _run(db, vp, tuning)
        assert st == 0
        assert np.array_equal(_sorted_rows(tri), _sorted_rows(ref_tri))
        vm = np.repeat(passed, f["V"].astype(np.int64)).astype(bool)
        assert np.array_equal(pos.reshape(-1, 3)[vm].view(np.uint32), ref_pos[vm].view(np.uint32))
        rejected += int((passed_plain.astype(bool) & ~passed.astype(bool)).sum())
    if which == "smooth_scene":  # the cone test did drop meshlets here
        assert rejected > 0.2 * blob.n_meshlets * len(vps)


def test_cull_cones_ignored_without_a_camera(smooth_scene):
    """An affine projection has no camera position: the cone test is off and
    the result equals the cone-free cull."""
    blob, _ = smooth_scene
    pts_lo = blob.grids.view(np.float32).reshape(-1, 8)[:, :3].min(0)
    vp = np.eye(4, dtype=np.float32) * np.float32(0.02)
    vp[3, 3] = 1.0
    vp[:3, 3] = -0.02 * (pts_lo + 4.0)
    assert O.view_eye(vp) is None
    db = device_batch_from_oracle(blob, cones=True)
    ref_tri, _, _ = O.decode_cull(blob, vp)
    tri, _, st = _run(db, vp)
    assert st == 0 and np.array_equal(_sorted_rows(tri), _sorted_rows(ref_tri))


def test_cull_graph_many_views_with_cones(smooth_scene):
    import torch
    blob, vps = smooth_scene
    db = device_batch_from_oracle(blob, cones=True)
    T, V = db.stats["total_tris"], db.stats["total_verts"]
    tri = torch.zeros(3 * T + 3, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(len(vps), dtype=torch.int32, device="cuda")
    pos = torch.zeros(3 * V, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    scratch = mc.new_scratch()
    d_vps = torch.from_numpy(np.ascontiguousarray(vps, np.float32)).cuda()
    g = mc.mc_graph_capture_cull(db, d_vps, len(vps), tri, cnt, pos, st, scratch)
    g.launch()
    torch.cuda.synchronize()
    counts = cnt.cpu().numpy()
    for i, vp in enumerate(vps):
        ref_tri, _, _ = O.decode_cull(blob, vp, cones=blob.cones)
        assert counts[i] == ref_tri.shape[0]
    assert int(st.item()) == 0 and int(scratch.abs().sum()) == 0


def test_cull_plain_gts_vs_oracle(smooth_scene):
    """The fused cull on plain GTS blocks (with cones) against the oracle."""
    _, vps = smooth_scene
    rng = np.random.Generator(np.random.PCG64(61))
    meshes = [G.uv_sphere(15_000, rng, noise=0.0), G.torus(12_000, rng, center=(2.5, 0, 0))]
    blob = O.concat([O.encode_mesh(m, (64, 126), 16, 2, mesh_id=i) for i, m in enumerate(meshes)])
    pts = np.concatenate([m.pos for m in meshes])
    c = 0.5 * (pts.min(0) + pts.max(0))
    r = float(np.linalg.norm(pts - c, axis=1).max())
    db = device_batch_from_oracle(blob, cones=True)
    f = blob.fields()
    for vp in G.camera_poses(4, c, r, seed=62, distance=2.0):
        ref_tri, ref_pos, passed = O.decode_cull(blob, vp, cones=blob.cones)
        for tuning in (None, {"warps_per_cta": 8, "checked": 1}):
            tri, pos, st = _run(db, vp, tuning)
            assert st == 0
            assert np.array_equal(_sorted_rows(tri), _sorted_rows(ref_tri))
            vm = np.repeat(passed, f["V"].astype(np.int64)).astype(bool)
            assert np.array_equal(pos.reshape(-1, 3)[vm].view(np.uint32), ref_pos[vm].view(np.uint32))


def _run_ordered(db, vp, tuning=None, cones=None):
    import torch
    T, V = db.stats["total_tris"], db.stats["total_verts"]
    tri = torch.full((3 * T + 3,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    pos = torch.zeros(3 * V, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    scratch = mc.new_scratch()
    d_vp = torch.from_numpy(np.ascontiguousarray(vp, np.float32)).cuda()
    mc.mc_decode_cull_ordered(db, d_vp, tri, cnt, pos, st, scratch, None, tuning)
    torch.cuda.synchronize()
    assert int(scratch.abs().sum()) == 0
    n = int(cnt.item())
    return tri[: 3 * n].cpu().numpy().view(np.uint32).reshape(-1, 3), pos.cpu().numpy(), int(st.item())


@pytest.mark.parametrize("tuning", [None, {"warps_per_cta": 8, "meshlets_per_grab": 16},
                                    {"warps_per_cta": 4, "meshlets_per_grab": 1, "checked": 1},
                                    {"warps_per_cta": 16, "meshlets_per_grab": 5}])
@pytest.mark.parametrize("which", ["scene", "smooth_scene"])
def test_cull_ordered_is_the_sequential_order(request, which, tuning):
    """The ordered mode returns exactly the oracle's survivor array (meshlet
    order, then triangle order), with and without cones."""
    blob, vps = request.getfixturevalue(which)
    f = blob.fields()
    for use_cones in (False, True):
        db = device_batch_from_oracle(blob, cones=use_cones)
        for vp in vps[:3]:
            ref, ref_pos, passed = O.decode_cull(blob, vp, cones=blob.cones if use_cones else None)
            tri, pos, st = _run_ordered(db, vp, tuning)
            assert st == 0
            assert np.array_equal(tri, ref)
            vm = np.repeat(passed, f["V"].astype(np.int64)).astype(bool)
            assert np.array_equal(pos.reshape(-1, 3)[vm].view(np.uint32), ref_pos[vm].view(np.uint32))


def _affine_view(blob):
    lo = blob.grids.view(np.float32).reshape(-1, 8)[:, :3].min(0)
    vp = np.eye(4, dtype=np.float32) * np.float32(0.02)
    vp[3, 3] = 1.0
    vp[:3, 3] = -0.02 * (lo + 4.0)
    return vp.reshape(16)


def _views_of(blob, vps, n):
    """n matrices: the fixture's views, an affine one (no camera), repeats."""
    pool = [np.asarray(v, np.float32).reshape(16) for v in vps] + [_affine_view(blob)]
    pool += pool[::-1]
    return np.stack(pool[:n])


def _run_views(db, vps, tuning=None):
    import torch
    T, V = db.stats["total_tris"], db.stats["total_verts"]
    n = len(vps)
    stride = 3 * T + 5
    tri = torch.full((n * stride,), -1, dtype=torch.int32, device="cuda")
    cnt = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    pos = torch.zeros(3 * V, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    scratch = mc.new_scratch()
    d_vps = torch.from_numpy(np.ascontiguousarray(vps, np.float32)).cuda()
    mc.mc_decode_cull_views(db, d_vps, n, tri, stride, cnt, pos, st, scratch, tuning)
    torch.cuda.synchronize()
    assert int(scratch.abs().sum()) == 0
    t = tri.cpu().numpy().view(np.uint32)
    c = cnt.cpu().numpy()
    outs = [t[v * stride: v * stride + 3 * int(c[v])].reshape(-1, 3) for v in range(n)]
    # nothing past each view's survivors is written
    for v in range(n):
        assert np.all(t[v * stride + 3 * int(c[v]): (v + 1) * stride] == 0xFFFFFFFF)
    return outs, pos.cpu().numpy(), int(st.item())


@pytest.mark.parametrize("tuning", [None, {"warps_per_cta": 8, "meshlets_per_grab": 16},
                                    {"warps_per_cta": 4, "meshlets_per_grab": 1, "checked": 1},
                                    {"warps_per_cta": 16, "meshlets_per_grab": 3}])
@pytest.mark.parametrize("which", ["scene", "smooth_scene"])
def test_cull_views_vs_oracle(request, which, tuning):
    """One launch against n views gives, per view, the oracle's survivors for
    that matrix (as a multiset); positions of meshlets passing any view are
    the oracle's to 0 ulp."""
    blob, vps = request.getfixturevalue(which)
    f = blob.fields()
    ref_pos = O.decode(blob)[2]
    for use_cones in (False, True):
        db = device_batch_from_oracle(blob, cones=use_cones)
        for n in (1, 3, 8):
            views = _views_of(blob, vps, n)
            outs, pos, st = _run_views(db, views, tuning)
            assert st == 0
            any_pass = np.zeros(f["V"].size, bool)
            for v in range(n):
                ref, _, passed = O.decode_cull(blob, views[v], cones=blob.cones if use_cones else None)
                assert outs[v].shape == ref.shape, (v, outs[v].shape, ref.shape)
                assert np.array_equal(_sorted_rows(outs[v]), _sorted_rows(ref)), v
                any_pass |= passed.astype(bool)
            vm = np.repeat(any_pass, f["V"].astype(np.int64))
            assert np.array_equal(pos.reshape(-1, 3)[vm].view(np.uint32), ref_pos[vm].view(np.uint32))


def test_cull_views_graph_64_views(smooth_scene):
    """The multi-view graph over more views than one launch takes: every
    count equals the oracle's, the last launch's regions hold its views."""
    import torch
    blob, vps = smooth_scene
    db = device_batch_from_oracle(blob, cones=True)
    T, V = db.stats["total_tris"], db.stats["total_verts"]
    views = np.concatenate([_views_of(blob, vps, 8)] * 3)[:19]  # 3 launches: 8 + 8 + 3
    stride = 3 * T
    tri = torch.zeros(8 * stride, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(len(views), dtype=torch.int32, device="cuda")
    pos = torch.zeros(3 * V, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    scratch = mc.new_scratch()
    d_vps = torch.from_numpy(np.ascontiguousarray(views, np.float32)).cuda()
    g = mc.mc_graph_capture_cull_views(db, d_vps, len(views), tri, stride, cnt, pos, st, scratch)
    for _ in range(2):
        g.launch()
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and int(scratch.abs().sum()) == 0
    c = cnt.cpu().numpy()
    t = tri.cpu().numpy().view(np.uint32)
    for v in range(len(views)):
        ref, _, _ = O.decode_cull(blob, views[v], cones=blob.cones)
        assert c[v] == ref.shape[0], v
        if v >= 16:  # the last launch's views (regions 0..2)
            r = v - 16
            got = t[r * stride: r * stride + 3 * int(c[v])].reshape(-1, 3)
            assert np.array_equal(_sorted_rows(got), _sorted_rows(ref))


def test_cull_views_arguments():
    import torch
    blob = O.encode_mesh(G.grid_mesh(8), (64, 126), 16, 0)
    db = device_batch_from_oracle(blob)
    T, V = db.stats["total_tris"], db.stats["total_verts"]
    vps = torch.zeros((9, 16), dtype=torch.float32, device="cuda")
    tri = torch.zeros(9 * 3 * T, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(9, dtype=torch.int32, device="cuda")
    pos = torch.zeros(3 * V, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    scratch = mc.new_scratch()
    for n, stride in ((0, 3 * T), (9, 3 * T), (2, 3 * T - 1)):
        with pytest.raises(mc.CodecError) as e:
            mc.mc_decode_cull_views(db, vps, n, tri, stride, cnt, pos, st, scratch)
        assert e.value.status == 1


def test_corrupt_stream_flagged_by_checked_cull_kernels():
    """A meshlet whose increment flags claim one vertex more than V: every
    checked cull form (one view, ordered, several views) reports
    MC_ERR_CORRUPT, finishes and leaves the scratch reset."""
    import torch
    from tests import blobpack as bp
    good = ([0, 1, 0, 1, 0], [0, 1, 2, 3, 4, 5, 6])
    desc, payload, grids = bp.pack([good] * 3)
    bad = payload.copy().view(np.uint32)
    off1 = int(desc.view(np.uint32)[1, 0]) * 4
    bad[off1 + 1] &= ~np.uint32(1 << 3)
    T, V = 15, 21
    db = mc.DeviceBatch.from_arrays(desc, bad.view(np.uint8), grids, T, V, 8)
    vp = np.diag([1e-6, 1e-6, 1e-6, 1.0]).astype(np.float32).reshape(16)
    d_vps = torch.from_numpy(np.ascontiguousarray(np.stack([vp, vp]))).cuda()
    for form in ("one", "ordered", "views"):
        tri = torch.zeros(2 * (3 * T + 3), dtype=torch.int32, device="cuda")
        cnt = torch.zeros(2, dtype=torch.int32, device="cuda")
        pos = torch.zeros(3 * V, dtype=torch.float32, device="cuda")
        st = torch.zeros(1, dtype=torch.int32, device="cuda")
        scratch = mc.new_scratch()
        t = {"checked": 1}
        if form == "one":
            mc.mc_decode_cull(db, d_vps[0], tri, cnt, pos, st, scratch, t)
        elif form == "ordered":
            mc.mc_decode_cull_ordered(db, d_vps[0], tri, cnt, pos, st, scratch, None, t)
        else:
            mc.mc_decode_cull_views(db, d_vps, 2, tri, 3 * T + 3, cnt, pos, st, scratch, t)
        torch.cuda.synchronize()
        assert int(st.item()) & (1 << mc.MC_ERR_CORRUPT), form
        assert int(scratch.abs().sum()) == 0, form



@pytest.mark.parametrize("grab", [1, 2, 5])
def test_fixed_grab_rounds_on_a_small_grid(scene, grab):
    """One warp per CTA and one CTA per SM make the grid's warps few enough
    for this batch to run the grab loop's fixed rounds (warp w takes grabs w,
    w + W, ... for 3/4 of an even split's rounds), then the queue's tail and,
    for grabs of 5 (1992 meshlets), a partial last grab: the batch decode, the one-view cull
    and the multi-view cull still give the oracle's results."""
    blob, vps = scene
    n_grabs = -(-blob.fields()["V"].size // grab)
    assert n_grabs // (152 * 1) * 3 // 4 >= 1  # the fixed rounds run on a 152-SM part
    tuning = {"warps_per_cta": 1, "ctas_per_sm": 1, "meshlets_per_grab": grab}
    db = device_batch_from_oracle(blob)
    assert_same_decode(run_decode(db, "batch", tuning), O.decode(blob), f"batch grab {grab}")
    f = blob.fields()
    ref_pos = O.decode(blob)[2]
    for vp in vps[:2]:
        ref_tri, ref_cpos, passed = O.decode_cull(blob, vp)
        tri, pos, st = _run(db, vp, tuning)
        assert st == 0
        assert np.array_equal(_sorted_rows(tri), _sorted_rows(ref_tri))
        vm = np.repeat(passed, f["V"].astype(np.int64)).astype(bool)
        assert np.array_equal(pos.reshape(-1, 3)[vm].view(np.uint32), ref_cpos[vm].view(np.uint32))
    views = _views_of(blob, vps, 3)
    outs, pos, st = _run_views(db, views, tuning)
    assert st == 0
    any_pass = np.zeros(f["V"].size, bool)
    for v in range(3):
        ref, _, passed = O.decode_cull(blob, views[v])
        assert np.array_equal(_sorted_rows(outs[v]), _sorted_rows(ref)), v
        any_pass |= passed.astype(bool)
    vm = np.repeat(any_pass, f["V"].astype(np.int64))
    assert np.array_equal(pos.reshape(-1, 3)[vm].view(np.uint32), ref_pos[vm].view(np.uint32))
