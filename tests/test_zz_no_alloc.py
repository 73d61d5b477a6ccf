"""The allocation-free batched decode against the regular one.

mc_decode_batch_noalloc exists for callers that cannot give the library any
device memory of its own -- hosts that own every allocation, or render loops
where a cudaMalloc would synchronise the device mid-frame.  It keeps its
work-queue counters in a small static device array instead of a caller
buffer.  This test decodes the same batch through both entry points of the C
ABI, twice in a row, and requires outputs identical to each other and to the
CPU oracle's decode of the same blob (bit for bit: indices exact, positions
0 ulp, the tolerance of every decode test here).  It lives in its own file,
collected last, and builds everything it needs itself, so it also runs alone.
"""
import numpy as np
import pytest

import oracle as O
from paper_2404_06359_gb300 import codec as mc
from paper_2404_06359_gb300 import meshgen as G

pytestmark = pytest.mark.gpu


def _batch():
    rng = np.random.Generator(np.random.PCG64(2026))
    parts = [O.encode_mesh(G.uv_sphere(15_000, rng), (64, 126), 16, 0),
             O.encode_mesh(G.torus(9_000, rng), (128, 128), lambda n: G.meshlet_bits(n, 3), 1),
             O.encode_mesh(G.grid_mesh(20), (256, 256), 20, 0)]
    blob = O.concat(parts)
    w = blob.desc.view(np.uint32).reshape(-1, 8)
    V, T = (w[:, 3] & 0xFFFF).astype(np.int64), (w[:, 3] >> 16).astype(np.int64)
    rw, b = (w[:, 4] & 0xFF).astype(np.int64), ((w[:, 4] >> 8) & 0xFF).astype(np.int64)
    words = 2 * ((T + 31) // 32) + ((T + 2 - V) * rw + 31) // 32 + (3 * V * b + 31) // 32
    mbw = int(((words + 3) // 4 * 4).max())
    return blob, mc.DeviceBatch.from_arrays(blob.desc, blob.payload, blob.grids, blob.total_tris,
                                            blob.total_verts, mbw)


def test_noalloc_matches_regular_entry_point_twice():
    import torch
    blob, db = _batch()
    loc, glob, pos, _ = O.decode(blob, want_pos64=False)
    ref = db.outputs()
    scratch = mc.new_scratch()
    mc.mc_decode_batch(db, ref["local"], ref["global"], ref["pos"], ref["status"], scratch)
    torch.cuda.synchronize()
    assert int(ref["status"].item()) == 0
    want = {k: ref[k].cpu().numpy() for k in ("local", "global", "pos")}
    assert np.array_equal(want["local"].reshape(-1, 3), loc)
    assert np.array_equal(want["global"].view(np.uint32).reshape(-1, 3), glob)
    assert np.array_equal(want["pos"].view(np.uint32).reshape(-1, 3), pos.view(np.uint32))
    out = db.outputs()
    for call in range(2):
        out["local"].fill_(0xAA)
        out["global"].fill_(-1)
        out["pos"].fill_(float("nan"))
        mc.mc_decode_batch_noalloc(db, out["local"], out["global"], out["pos"], out["status"])
        torch.cuda.synchronize()
        assert int(out["status"].item()) == 0, f"call {call}: status"
        assert np.array_equal(out["local"].cpu().numpy(), want["local"]), f"call {call}: local"
        assert np.array_equal(out["global"].cpu().numpy(), want["global"]), f"call {call}: global"
        got = out["pos"].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, want["pos"].view(np.uint32)), f"call {call}: positions"
