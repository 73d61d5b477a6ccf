"""Pins of the oracle's normal-cone meshlet culling (the per-meshlet cull data
of Sec. 3 / Sec. 5: a cone holding the meshlet's triangle normals, used to
drop meshlets that face away from the camera as a whole).

What is pinned, without retyping the oracle's formulas:
  * containment: every decoded vertex lies in the record's sphere and every
    non-degenerate triangle normal lies in the record's cone;
  * a planar patch has the tightest cone (its plane normal, s = 2^-20);
  * the camera position recovered from a clip matrix is the eye the matrix
    was built from; an affine projection has none;
  * conservativeness: every triangle of a rejected meshlet faces away from
    the eye in FP64 (brute force over many eyes);
  * decode + cull with cones = decode + cull without cones minus the
    rejected meshlets, exactly.
"""
import numpy as np
import pytest

import oracle as O
from paper_2404_06359_gb300 import meshgen as G


def _records(blob):
    c = blob.cones.view(np.float32).reshape(-1, 8).astype(np.float64)
    return c[:, 0:3], c[:, 3], c[:, 4:7], c[:, 7]


def _meshlet_geometry(blob, m):
    loc, pos, _ = O.decode_meshlet(blob, m)
    p = pos.astype(np.float64)
    t = loc.astype(np.int64)
    t = t[(t[:, 0] != t[:, 1]) & (t[:, 1] != t[:, 2]) & (t[:, 0] != t[:, 2])]
    n = np.cross(p[t[:, 1]] - p[t[:, 0]], p[t[:, 2]] - p[t[:, 0]])
    ln = np.linalg.norm(n, axis=1)
    keep = ln > 0
    return p, t[keep], n[keep] / ln[keep, None]


@pytest.fixture(scope="module")
def meshes():
    rng = np.random.Generator(np.random.PCG64(2024))
    return [G.uv_sphere(20_000, rng), G.torus(30_000, rng), G.grid_mesh(40, 0.25, 77)]


@pytest.mark.parametrize("limits", [(64, 126), (128, 128)])
def test_cone_contains_vertices_and_normals(meshes, limits):
    for mesh in meshes:
        blob = O.encode_mesh(mesh, limits, 16, 0)
        ctr, rad, axis, s = _records(blob)
        assert np.all(np.abs(np.linalg.norm(axis, axis=1) - 1.0) < 1e-6)
        assert np.all((s > 0) & (s <= 1))
        for m in range(blob.n_meshlets):
            p, t, n = _meshlet_geometry(blob, m)
            assert np.linalg.norm(p - ctr[m], axis=1).max() <= rad[m]
            if s[m] < 1:
                cos_a = np.sqrt(1.0 - s[m] ** 2)
                assert (n @ axis[m]).min() >= cos_a - 1e-7, m


def test_planar_patch_has_the_tightest_cone():
    mesh = G.grid_mesh(16, 0.25, 5)
    mesh.pos[:, 2] = 0.0  # flatten: every normal is +z (counter-clockwise grid in xy)
    blob = O.encode_mesh(mesh, (64, 126), 16, 0)
    _, _, axis, s = _records(blob)
    tight = np.float32(np.nextafter(np.float32(2.0 ** -20), np.float32(1))) \
        if np.float64(np.float32(2.0 ** -20)) < 2.0 ** -20 else np.float32(2.0 ** -20)
    assert np.all(s == tight)
    assert np.all(np.abs(axis[:, 2]) == 1.0) and np.all(axis[:, :2] == 0.0)
    assert len(np.unique(np.sign(axis[:, 2]))) == 1


def _look_at(eye, target, up):
    f = target - eye
    f = f / np.linalg.norm(f)
    r = np.cross(f, up)
    r = r / np.linalg.norm(r)
    u = np.cross(r, f)
    v = np.eye(4)
    v[0, :3], v[1, :3], v[2, :3] = r, u, -f
    v[:3, 3] = -v[:3, :3] @ eye
    return v


def _frustum(fovy, near, far):
    t = 1.0 / np.tan(np.radians(fovy) / 2)
    p = np.zeros((4, 4))
    p[0, 0] = p[1, 1] = t
    p[2, 2] = (far + near) / (near - far)
    p[2, 3] = 2 * far * near / (near - far)
    p[3, 2] = -1.0
    return p


def test_view_eye_recovers_the_camera():
    rng = np.random.Generator(np.random.PCG64(3))
    for _ in range(200):
        eye = rng.normal(0, 5, 3)
        tgt = rng.normal(0, 1, 3)
        vp = (_frustum(rng.uniform(30, 90), 0.05, 50.0) @ _look_at(eye, tgt, np.array([0, 0, 1.0])))
        got = O.view_eye(vp.astype(np.float32))
        assert got is not None
        assert np.linalg.norm(got - eye) <= 1e-4 * (1 + np.linalg.norm(eye))
    ortho = np.eye(4)
    ortho[2, 2] = -0.1
    assert O.view_eye(ortho.astype(np.float32)) is None


def test_rejected_meshlets_face_away_brute_force(meshes):
    """Every triangle of every rejected meshlet faces away from the eye
    (FP64, from the decoded positions), over eyes near and far, inside and
    outside the bounding sphere."""
    rng = np.random.Generator(np.random.PCG64(11))
    total_rejected = 0
    for mesh in meshes[:2]:
        blob = O.encode_mesh(mesh, (64, 126), 16, 0)
        geo = [_meshlet_geometry(blob, m) for m in range(blob.n_meshlets)]
        for _ in range(40):
            d = rng.normal(size=3)
            eye = (d / np.linalg.norm(d) * rng.uniform(0.3, 6.0)).astype(np.float32)
            for m in range(blob.n_meshlets):
                if not O.cone_test(blob.cones[m], eye):
                    continue
                total_rejected += 1
                p, t, n = geo[m]
                facing = np.einsum("ij,ij->i", n, p[t[:, 0]] - eye.astype(np.float64))
                assert facing.min() >= 0.0, (m, facing.min())
    assert total_rejected > 1000


@pytest.mark.parametrize("noise", [0.0, 0.01])
def test_cull_with_cones_drops_exactly_the_rejected_meshlets(noise):
    mesh = G.uv_sphere(20_000, np.random.Generator(np.random.PCG64(5)), noise=noise)
    blob = O.encode_mesh(mesh, (64, 126), 16, 0)
    c = mesh.pos.astype(np.float64).mean(0)
    r = float(np.linalg.norm(mesh.pos - c, axis=1).max())
    f = blob.fields()
    fractions = []
    for vp in G.camera_poses(8, c, r, seed=9, distance=3.0):
        plain, pos0, pass0 = O.decode_cull(blob, vp)
        coned, pos1, pass1 = O.decode_cull(blob, vp, cones=blob.cones)
        eye = O.view_eye(vp)
        rej = np.array([O.cone_test(blob.cones[m], eye) for m in range(blob.n_meshlets)])
        assert np.array_equal(pass1, pass0 & ~rej)
        owner = np.searchsorted(f["vertex_base"].astype(np.int64), plain[:, 0].astype(np.int64),
                                side="right") - 1
        assert np.array_equal(coned, plain[~rej[owner]])
        vm = np.repeat(pass1.astype(bool), f["V"].astype(np.int64))
        assert np.array_equal(pos1[vm], pos0[vm])
        fractions.append(rej[pass0.astype(bool)].mean())
    # a smooth sphere seen from 3 radii: 2/3 of its surface faces away (the
    # tangent cone touches at acos(1/3)), so a large share of meshlets but
    # fewer than 2/3 are rejected; radial noise of 1 % of the radius,
    # comparable to the edge length here, widens the cones and leaves few
    if noise == 0.0:
        assert 0.3 < np.mean(fractions) < 2 / 3, fractions
    else:
        assert np.mean(fractions) < 0.25, fractions
