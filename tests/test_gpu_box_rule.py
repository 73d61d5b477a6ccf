"""The quantisation-box rule on the GPU, in every decode and cull form.

A meshlet's minimum L must leave room for its whole box: L + 2^b - 1 < 2^32
(Sec. 4.4 adds q to L as a 32-bit integer; the encoder never writes a
minimum closer to 2^32).  At L = 2^32 - 2^b every form decodes exactly like
the oracle (top vertex at g = 2^32 - 1, the split dequantisation path); one
more and every form reports MC_ERR_CORRUPT for that meshlet, decodes the
others, finishes and leaves its scratch reset.  Without the rule the box
corner L + 2^b - 1 would wrap below L and the frustum test could drop a
visible meshlet with no error.
"""
import numpy as np
import pytest

import oracle as O
from paper_2404_06359_gb300 import codec as mc
from tests import blobpack as bp
from tests.gpu_util import block_words_max

pytestmark = pytest.mark.gpu

CASES = [([0, 1, 0, 1, 0], [0, 1, 2, 3, 4, 5, 6]), ([0, 0, 0, 1], [0, 1, 2, 3, 4, 1]),
         ([0, 1, 1, 0, 1, 0], [0, 1, 2, 3, 0, 4, 5, 2])]
GRID = (-2.0, 1.0, 0.5, 2.0 ** -20, 3e-7, 1e-5)


def _blob(b, L_mid):
    """Three meshlets at bit width b; the middle one has minimum L_mid, the
    others 0 (one descriptor each, packed separately and concatenated)."""
    qmax = 2 ** b - 1
    parts = []
    for i, case in enumerate(CASES):
        L = L_mid if i == 1 else (0, 0, 0)
        parts.append(bp.pack([case], pos_bits=b, q_fn=lambda v, c: qmax if v == 0 else v % 7,
                             L=L, grid=GRID))
    descs, pays, off16, vb, tb = [], [], 0, 0, 0
    for desc, payload, grids in parts:
        d = desc.copy().view(np.uint32).reshape(-1, 8)
        d[:, 0] += off16
        d[:, 1] += vb
        d[:, 2] += tb
        vb += int(d[0, 3] & 0xFFFF)
        tb += int(d[0, 3] >> 16)
        off16 += payload.size // 16
        descs.append(d.view(np.uint8).reshape(-1, 32))
        pays.append(payload)
    return np.concatenate(descs), np.concatenate(pays), parts[0][2], tb, vb


def _vp():
    # everything at the origin's scale is inside: a tiny uniform scale
    return np.diag([1e-12, 1e-12, 1e-12, 1.0]).astype(np.float32).reshape(16)


def _run_forms(db, T, V):
    """status, decoded outputs of each form (None where the form has none)."""
    import torch
    res = {}
    d_vp = torch.from_numpy(_vp()).cuda()
    d_vps = torch.from_numpy(np.ascontiguousarray(np.stack([_vp(), _vp()]))).cuda()
    M = db.stats["n_meshlets"]
    for form in ("plain", "batch", "noalloc", "cull", "ordered", "views", "requests"):
        out = db.outputs()
        out["local"].fill_(0xAA)
        out["pos"].fill_(float("nan"))
        scratch = mc.new_scratch()
        tri = torch.zeros(2 * (3 * T + 3), dtype=torch.int32, device="cuda")
        cnt = torch.zeros(2, dtype=torch.int32, device="cuda")
        if form == "plain":
            mc.mc_decode_plain(db, 0, M, out["local"], out["global"], out["pos"], out["status"])
        elif form == "batch":
            mc.mc_decode_batch(db, out["local"], out["global"], out["pos"], out["status"], scratch)
        elif form == "noalloc":
            mc.mc_decode_batch_noalloc(db, out["local"], out["global"], out["pos"], out["status"])
        elif form == "cull":
            mc.mc_decode_cull(db, d_vp, tri, cnt, out["pos"], out["status"], scratch)
        elif form == "ordered":
            mc.mc_decode_cull_ordered(db, d_vp, tri, cnt, out["pos"], out["status"], scratch)
        elif form == "views":
            mc.mc_decode_cull_views(db, d_vps, 2, tri, 3 * T + 3, cnt, out["pos"], out["status"],
                                    scratch)
        else:
            r = np.zeros(1, mc.REQUEST_DTYPE)
            r["n_meshlets"] = M
            r["tri_count"], r["vert_count"] = T, V
            r["d_local"], r["d_global"] = out["local"].data_ptr(), out["global"].data_ptr()
            r["d_pos"] = out["pos"].data_ptr()
            d_r = torch.from_numpy(r.view(np.uint8).copy()).cuda()
            mc.mc_decode_requests(db, d_r, 1, M, out["status"], scratch)
        torch.cuda.synchronize()
        assert int(scratch.abs().sum()) == 0, form
        cull = form in ("cull", "ordered", "views")
        res[form] = (int(out["status"].item()),
                     None if cull else out["local"].cpu().numpy().reshape(-1, 3),
                     out["pos"].cpu().numpy().reshape(-1, 3),
                     tri[: 3 * int(cnt[0].item())].cpu().numpy().view(np.uint32).reshape(-1, 3)
                     if cull else None)
    return res


@pytest.mark.parametrize("b", [12, 16, 27, 32])
def test_top_of_grid_decodes_and_one_past_is_corrupt(b):
    lim = 2 ** 32 - 2 ** b
    # valid: the middle meshlet's box ends exactly at 2^32 - 1
    desc, payload, grids, T, V = _blob(b, (lim, lim, lim))
    ob = O.Blob(desc, payload, grids)
    loc, glob, pos, _ = O.decode(ob)
    ref_tri, ref_pos, _ = O.decode_cull(ob, _vp())
    db = mc.DeviceBatch.from_arrays(desc, payload, grids, T, V, block_words_max(desc))
    for form, (st, l, p, tri) in _run_forms(db, T, V).items():
        assert st == 0, (form, st)
        if l is not None:
            assert np.array_equal(l, loc), form
            assert np.array_equal(p.view(np.uint32), pos.view(np.uint32)), form
        else:
            assert np.array_equal(p.view(np.uint32), ref_pos.view(np.uint32)), form
            srt = lambda t: t[np.lexsort(t.T[::-1])]
            assert np.array_equal(srt(tri), srt(ref_tri)), form
    vtop = int(desc.view(np.uint32).reshape(-1, 8)[1, 1])  # the middle meshlet's vertex 0
    assert (pos[vtop] == [O.dequant32(2 ** 32 - 1, GRID[c], GRID[3 + c]) for c in range(3)]).all()
    # one past, in each channel: corrupt in every form; meshlets 0 and 2 still decode
    for c in range(3):
        L = [lim, lim, lim]
        L[c] += 1
        desc2, payload2, grids2, T2, V2 = _blob(b, tuple(L))
        db2 = mc.DeviceBatch.from_arrays(desc2, payload2, grids2, T2, V2, block_words_max(desc2))
        t0, t1 = len(CASES[0][0]), len(CASES[0][0]) + len(CASES[1][0])
        v0 = int(desc2.view(np.uint32).reshape(-1, 8)[1, 1])
        v1 = int(desc2.view(np.uint32).reshape(-1, 8)[2, 1])
        for form, (st, l, p, tri) in _run_forms(db2, T2, V2).items():
            assert st & (1 << mc.MC_ERR_CORRUPT), (form, c, st)
            if l is not None:
                assert np.array_equal(l[:t0], loc[:t0]) and np.array_equal(l[t1:], loc[t1:]), form
                assert np.array_equal(p[:v0].view(np.uint32), pos[:v0].view(np.uint32)), form
                assert np.array_equal(p[v1:].view(np.uint32), pos[v1:].view(np.uint32)), form


def test_max_verts_bounds_every_meshlet():
    """mc_device_batch.max_verts sizes the fused culls' per-warp vertex
    buffers, so a meshlet with more vertices than it claims is rejected as
    corrupt (by every form) instead of overrunning them; the true largest V
    (or 0, the T' + 2 bound) decodes like the oracle."""
    import torch
    from paper_2404_06359_gb300 import meshgen as G
    from tests.gpu_util import max_tris, max_verts
    blob = O.encode_mesh(G.grid_mesh(12), (64, 126), 16, 0)
    vmax = max_verts(blob.desc)
    loc, _, pos, _ = O.decode(blob)
    T, V = blob.total_tris, blob.total_verts
    args = (blob.desc, blob.payload, blob.grids, T, V, block_words_max(blob.desc), max_tris(blob.desc))
    for mv in (0, vmax):
        res = _run_forms(mc.DeviceBatch.from_arrays(*args, max_verts=mv), T, V)
        for form, (st, l, p, tri) in res.items():
            assert st == 0, (mv, form)
            if l is not None:
                assert np.array_equal(l, loc), (mv, form)
    Vs = blob.fields()["V"].astype(np.int64)
    res = _run_forms(mc.DeviceBatch.from_arrays(*args, max_verts=vmax - 1), T, V)
    for form, (st, l, p, tri) in res.items():
        assert st & (1 << mc.MC_ERR_CORRUPT), form
        if l is not None:  # meshlets within the bound still decode
            f = blob.fields()
            for m in np.nonzero(Vs < vmax)[0][:5]:
                tb, tp = int(f["tri_base"][m]), int(f["Tp"][m])
                assert np.array_equal(l[tb:tb + tp], loc[tb:tb + tp]), form
