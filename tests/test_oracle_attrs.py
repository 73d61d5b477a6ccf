"""Pins of the oracle's attribute-vector quantisation (Sec. 4.4: every
attribute channel -- here normals and texture coordinates beside the
position -- on its own crack-free global grid at b bits; Tab. 3 reports the
resulting information content per channel).

Pinned against facts, not against the oracle's own formulas:
  * every decoded channel is within half a grid step of the input (plus the
    FP32 rounding of the result);
  * a vertex shared by several meshlets decodes to the same bits in each
    (no cracks);
  * the information content log2(W / Delta) of every channel is at least
    log2(2^b - 1) ~ b (the paper's claim, with W the channel's extent over
    the mesh), up to the FP32 rounding of Delta;
  * the connectivity and positions decode exactly as without attributes, and
    each payload block grows by exactly the attribute words.
"""
import numpy as np
import pytest

import oracle as O
from paper_2404_06359_gb300 import meshgen as G


@pytest.fixture(scope="module")
def cases():
    rng = np.random.Generator(np.random.PCG64(404))
    out = []
    for mesh, lim, bits in [(G.uv_sphere(20_000, rng), (64, 126), 16),
                            (G.torus(15_000, rng), (128, 128), 16),
                            (G.grid_mesh(32), (64, 126), 12),
                            (G.uv_sphere(6_000, rng), (256, 256), 20)]:
        at = G.vertex_attributes(mesh)
        out.append((mesh, at, bits, O.encode_mesh(mesh, lim, 16, 0, attrs=at, attr_bits=bits),
                    O.encode_mesh(mesh, lim, 16, 0)))
    return out


def _grid(blob):
    g = blob.attrs["agrids"].view(np.float32).reshape(-1, 12)
    return g[0, 0:5].astype(np.float64), g[0, 5:10].astype(np.float64)


def test_attributes_within_half_a_step(cases):
    for mesh, at, bits, blob, _ in cases:
        got = O.decode_attrs(blob).astype(np.float64)
        want = at[blob.stats["vmap"]].astype(np.float64)
        _, D = _grid(blob)
        ulp = np.spacing(np.abs(got).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(got - want) <= D / 2 + 1.5 * ulp), mesh.kind


def test_shared_vertices_decode_identically(cases):
    for mesh, at, bits, blob, _ in cases:
        got = O.decode_attrs(blob)
        vm = blob.stats["vmap"]
        order = np.argsort(vm, kind="stable")
        vs, gs = vm[order], got[order].view(np.uint32)
        same = vs[1:] == vs[:-1]
        assert same.any()
        assert np.array_equal(gs[1:][same], gs[:-1][same])


def test_information_content_at_least_b(cases):
    rows = []
    for mesh, at, bits, blob, _ in cases:
        _, D = _grid(blob)
        W = at.max(0).astype(np.float64) - at.min(0).astype(np.float64)
        info = np.log2(W / D)
        rows.append((mesh.kind, bits, np.round(info, 2)))
        # log2(2^b - 1) ~ b; Delta is rounded up to FP32 (and raised a step at a
        # time if needed), which may cost a few FP32 steps of 2^-23 relative
        assert np.all(info >= np.log2(2.0 ** bits - 1) - np.log2(1 + 2.0 ** -20)), (mesh.kind, info)
    print("information content (normal x y z, u, v):", rows)


def test_connectivity_and_positions_unchanged(cases):
    for mesh, at, bits, blob, plain in cases:
        assert np.array_equal(blob.desc[:, 12:], plain.desc[:, 12:])  # V, T', w, b, grid, L
        for x, y in zip(O.decode(blob)[:3], O.decode(plain)[:3]):
            assert np.array_equal(x, y)
        f = blob.fields()
        V = f["V"].astype(np.int64)
        nw = (f["Tp"].astype(np.int64) + 31) // 32
        base = 2 * nw + ((f["Tp"].astype(np.int64) + 2 - V) * f["w"].astype(np.int64) + 31) // 32 \
            + (3 * V * 16 + 31) // 32
        words = base + (5 * V * bits + 31) // 32
        assert blob.payload.size == int(16 * ((words + 3) // 4).sum())
