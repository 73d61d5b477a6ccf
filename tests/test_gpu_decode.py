"""GPU parity: every decode kernel against the CPU oracle, bit for bit.

Indices (u8 local, u32 global) must be identical and FP32 positions identical
to 0 ulp (both sides evaluate the same fma sequence of Sec. 4.4).  Inputs
are oracle-encoded meshes (no input or expected value comes from the CUDA
path) and hand-packed streams (tests/blobpack.py).
"""
import numpy as np
import pytest

import oracle as O
from paper_2404_06359_gb300 import codec as mc
from paper_2404_06359_gb300 import meshgen as G
from tests import blobpack as bp
from tests.gpu_util import assert_same_decode, block_words_max, device_batch_from_oracle, run_decode

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def grid_blob():
    return O.encode_mesh(G.grid_mesh(), (64, 126), 16, 0)


@pytest.fixture(scope="module")
def mixed_batch():
    """Several meshes, all three meshlet limits, w = ceil(log2 V), random b in
    {12, 16, 20}, meshlets shuffled -- spans many tiles and ragged tails."""
    rng = np.random.Generator(np.random.PCG64(44))
    parts = [
        O.encode_mesh(G.uv_sphere(9_000, rng), (64, 126), 16, 0),
        O.encode_mesh(G.torus(7_000, rng), (128, 128), lambda n: G.meshlet_bits(n, 1), 1,
                      perm=lambda n: G.meshlet_permutation(n, 2)),
        O.encode_mesh(G.height_field_disc(30_000, seed=3), np.array(G.SECTOR_LIMITS).reshape(-1),
                      lambda n: G.meshlet_bits(n, 4), 1, perm=lambda n: G.meshlet_permutation(n, 5)),
        O.encode_mesh(G.uv_sphere(12_000, rng), (256, 256), 20, 0),
        O.encode_mesh(G.grid_mesh(5), (8, 5), 7, 1),
    ]
    return O.concat(parts)


def test_plain_grid_8192(grid_blob):
    """64x64-quad grid, 8,192 triangles, 64/126, b = 16: plain one-launch decode."""
    ref = O.decode(grid_blob)
    db = device_batch_from_oracle(grid_blob)
    for warps in (1, 4, 8, 32):
        assert_same_decode(run_decode(db, "plain", {"warps_per_cta": warps}), ref, f"plain w{warps}")


PAIR_TUNINGS = [{"lanes_per_meshlet": 16, "warps_per_cta": 4, "meshlets_per_grab": 4},
                {"lanes_per_meshlet": 16, "warps_per_cta": 8, "meshlets_per_grab": 3},
                {"lanes_per_meshlet": 16, "warps_per_cta": 16, "meshlets_per_grab": 16},
                {"lanes_per_meshlet": 16, "warps_per_cta": 4, "meshlets_per_grab": 2, "checked": 1}]


@pytest.mark.parametrize("tuning", [None, {"warps_per_cta": 4, "meshlets_per_grab": 1},
                                    {"warps_per_cta": 16, "meshlets_per_grab": 8},
                                    {"warps_per_cta": 8, "meshlets_per_grab": 3, "ctas_per_sm": 1},
                                    {"warps_per_cta": 8, "checked": 1}] + PAIR_TUNINGS)
def test_batch_mixed_vs_oracle(mixed_batch, tuning):
    ref = O.decode(mixed_batch)
    db = device_batch_from_oracle(mixed_batch)
    assert_same_decode(run_decode(db, "batch", tuning), ref, f"batch {tuning}")


def test_plain_mixed_vs_oracle(mixed_batch):
    ref = O.decode(mixed_batch)
    db = device_batch_from_oracle(mixed_batch)
    assert_same_decode(run_decode(db, "plain", {"checked": 1}), ref, "plain checked")
    res = run_decode(db, "plain", None, local=False, global_=True)
    assert_same_decode(res, ref, "plain no-local")


@pytest.mark.parametrize("tp", [1, 2, 3, 4, 5, 6, 7, 8])
def test_bruteforce_corpus(tp):
    """All flag words x all first-appearance streams of T' <= 8 (7.7 M meshlets
    at T' = 8): GPU == oracle walk, bit for bit."""
    cases = list(bp.enumerate_cases(tp)) if tp < 8 else None
    if cases is None:
        streams = np.array([(0, 1, 2) + s for s in bp.restricted_growth(7)], np.int64)
        nf = 1 << 7
        flags = np.zeros((nf * streams.shape[0], 8), np.int64)
        fl = ((np.arange(nf)[:, None] >> np.arange(7)[None, :]) & 1)
        flags[:, 1:] = np.repeat(fl, streams.shape[0], 0)
        stream = np.tile(streams, (nf, 1))
    else:
        flags = np.array([c[0] for c in cases], np.int64)
        stream = np.array([c[1] for c in cases], np.int64)
    desc, payload, grids, V = bp.pack_small(flags, stream)
    blob = O.Blob(desc, payload, grids)
    ref = O.decode(blob, want_pos64=False)
    db = mc.DeviceBatch.from_arrays(desc, payload, grids, blob.total_tris, blob.total_verts, 8)
    assert_same_decode(run_decode(db, "batch"), ref, f"bruteforce T'={tp}")
    assert_same_decode(run_decode(db, "batch", {"checked": 1}), ref, f"bruteforce checked T'={tp}")
    for t in (PAIR_TUNINGS[0], PAIR_TUNINGS[-1]):  # two meshlets per warp
        assert_same_decode(run_decode(db, "batch", t), ref, f"bruteforce T'={tp} {t}")


@pytest.mark.parametrize("tuning", [None, {"meshlets_per_grab": 4}] + PAIR_TUNINGS[:2])
def test_batch_descriptors_out_of_order(mixed_batch, tuning):
    """Descriptors in another order than their payload blocks (the format
    only needs each descriptor to point at its block): no grab's blocks form
    one range, so every block is staged on its own (meshlet by meshlet, or
    pair by pair with two meshlets per warp); the outputs follow the
    descriptors' bases and equal the oracle's decode of the same blob."""
    rng = np.random.Generator(np.random.PCG64(46))
    perm = rng.permutation(mixed_batch.n_meshlets)
    blob = O.Blob(mixed_batch.desc[perm].copy(), mixed_batch.payload, mixed_batch.grids)
    ref = O.decode(blob)
    db = device_batch_from_oracle(blob)
    assert_same_decode(run_decode(db, "batch", tuning), ref, f"out of order {tuning}")


def test_long_fans_reuse_widths_and_bits():
    rng = np.random.Generator(np.random.PCG64(77))
    cases = []
    for tp in (31, 32, 33, 63, 64, 65, 100, 200, 254, 255, 256):
        s = [0, 1, 2]
        seen = 3
        for _ in range(tp - 1):
            if (rng.random() < 0.4 and seen < 256) or seen < 5:
                s.append(seen)
                seen += 1
            else:
                s.append(int(rng.integers(0, seen)))
        run = int(rng.integers(1, tp + 1))
        flags = [0] + [1] * min(run, tp - 1) + list(rng.integers(0, 2, max(0, tp - 1 - run)))
        cases.append((flags[:tp], s))
    for b in (1, 5, 12, 16, 20, 27, 32):
        for wmode in (8, "log2"):
            desc, payload, grids = bp.pack(cases, reuse_w=wmode, pos_bits=b,
                                           q_fn=lambda v, c, b=b: int(rng.integers(0, min(2 ** b, 2 ** 31))),
                                           L=tuple(min(x, 2 ** 32 - 2 ** b) for x in (7, 2 ** 20, 3)),
                                           grid=(-1.5, 2.0, 0.25, 1e-3, 3e-5, 0.5))
            blob = O.Blob(desc, payload, grids)
            ref = O.decode(blob)
            db = mc.DeviceBatch.from_arrays(desc, payload, grids, blob.total_tris, blob.total_verts,
                                            block_words_max(desc))
            assert_same_decode(run_decode(db, "batch"), ref, f"b={b} w={wmode}")
            assert_same_decode(run_decode(db, "plain", {"checked": 1}), ref, f"b={b} w={wmode}")
            for t in (PAIR_TUNINGS[0], PAIR_TUNINGS[-1]):
                assert_same_decode(run_decode(db, "batch", t), ref, f"b={b} w={wmode} {t}")


def test_corrupt_streams_flagged_by_checked_kernel():
    torch = _torch()
    good = ([0, 1, 0, 1, 0], [0, 1, 2, 3, 4, 5, 6])
    desc, payload, grids = bp.pack([good] * 3)
    bad_payload = payload.copy().view(np.uint32)
    # meshlet 1: increment flags claim one vertex more than V
    off1 = int(desc.view(np.uint32)[1, 0]) * 4
    bad_payload[off1 + 1] &= ~np.uint32(1 << 3)
    db = mc.DeviceBatch.from_arrays(desc, bad_payload.view(np.uint8), grids, 15, 21, 8)
    for mode in ("plain", "batch"):
        out = run_decode(db, mode, {"checked": 1})
        assert int(out["status"][0]) & (1 << mc.MC_ERR_CORRUPT)
    out = run_decode(db, "batch", PAIR_TUNINGS[-1])
    assert int(out["status"][0]) & (1 << mc.MC_ERR_CORRUPT)
    # the pair's other meshlets are decoded regardless
    ref = O.decode(O.Blob(desc, payload, grids))
    assert np.array_equal(out["local"].reshape(-1, 3)[:5], ref[0][:5])
    assert np.array_equal(out["local"].reshape(-1, 3)[10:], ref[0][10:])
    # a descriptor pointing outside the payload is rejected by every kernel
    d2 = desc.copy().view(np.uint32)
    d2[2, 0] = 10_000
    db2 = mc.DeviceBatch.from_arrays(d2.view(np.uint8), payload, grids, 15, 21, 8)
    out = run_decode(db2, "batch", None)
    assert int(out["status"][0]) & (1 << mc.MC_ERR_CORRUPT)
    torch.cuda.synchronize()


def test_empty_and_single_meshlet():
    torch = _torch()
    one = O.encode_mesh(G.Mesh(np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0.5]], np.float32),
                               np.array([[0, 1, 2]], np.uint32)), (64, 126), 16, 0)
    ref = O.decode(one)
    db = device_batch_from_oracle(one)
    assert_same_decode(run_decode(db, "batch"), ref, "single")
    assert_same_decode(run_decode(db, "plain"), ref, "single plain")
    # zero meshlets: a no-op that leaves the scratch zero
    empty = mc.DeviceBatch.from_arrays(np.zeros((0, 32), np.uint8), np.zeros(16, np.uint8),
                                       one.grids, 0, 0, 4)
    out = empty.outputs()
    s = mc.new_scratch()
    mc.mc_decode_batch(empty, out["local"], out["global"], out["pos"], out["status"], s)
    torch.cuda.synchronize()
    assert int(s.abs().sum()) == 0


def test_graph_replay_and_autotune(mixed_batch):
    torch = _torch()
    ref = O.decode(mixed_batch)
    db = device_batch_from_oracle(mixed_batch)
    out = db.outputs()
    scratch = mc.new_scratch()
    best, ms = mc.mc_autotune(db, out["local"], out["global"], out["pos"], out["status"], scratch)
    assert best.warps_per_cta in (4, 8, 16) and ms > 0
    g = mc.mc_graph_capture_batch(db, out["local"], out["global"], out["pos"], out["status"], scratch)
    for _ in range(3):
        out["pos"].zero_()
        out["local"].fill_(255)
        n0 = mc.mc_launch_count()
        g.launch()
        torch.cuda.synchronize()
        assert mc.mc_launch_count() == n0 + 1
        res = {k: v.cpu().numpy() for k, v in out.items()}
        assert_same_decode(res, ref, "graph replay")
    assert int(scratch.abs().sum()) == 0


@pytest.mark.parametrize("n_meshes,pinned", [(1, False), (1, True), (60, True)])
def test_host_buffer_decode_matches(n_meshes, pinned):
    """mc_decode_batch_host (copies in, decode, copies out) on a library blob;
    60 tori give more than 8192 meshlets, so the call runs as several
    overlapped chunks on the library's internal streams."""
    torch = _torch()
    rng = np.random.Generator(np.random.PCG64(12))
    blobs = []
    for i in range(n_meshes):
        mesh = G.torus(20_000, rng)
        m = mc.mc_meshletize(mesh.tris, mesh.n_verts, [(64, 126)])
        blobs.append(mc.mc_encode(m, mesh.pos, 16, 0, mesh_id=i))
    blob = blobs[0] if n_meshes == 1 else mc.mc_blob_concat(blobs)
    a = blob.arrays()
    ref = O.decode(O.Blob(a["desc"], a["payload"], a["grids"]))
    s = blob.stats()
    assert (s["n_meshlets"] > 8192) == (n_meshes > 1)
    d_desc = torch.empty(32 * s["n_meshlets"], dtype=torch.uint8, device="cuda")
    d_pay = torch.empty(s["payload_bytes"], dtype=torch.uint8, device="cuda")
    d_grids = torch.empty(32 * s["n_grids"], dtype=torch.uint8, device="cuda")
    T, V = s["total_tris"], s["total_verts"]
    d_loc = torch.empty(3 * T, dtype=torch.uint8, device="cuda")
    d_glob = torch.empty(3 * T, dtype=torch.int32, device="cuda")
    d_pos = torch.empty(3 * V, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    scratch = mc.new_scratch()
    h_loc = torch.full((3 * T,), 0xEE, dtype=torch.uint8).pin_memory()
    h_glob = torch.full((3 * T,), -1, dtype=torch.int32).pin_memory()
    h_pos = torch.full((3 * V,), float("nan"), dtype=torch.float32).pin_memory()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        mc.mc_decode_batch_host(blob, d_desc, d_pay, d_grids, d_loc, d_glob, d_pos, st, scratch,
                                h_loc, h_glob, h_pos, None, side,
                                host_inputs=mc.pinned_inputs(blob) if pinned else None)
    side.synchronize()  # the call is complete once its stream is
    res = {"local": h_loc.numpy(), "global": h_glob.numpy(), "pos": h_pos.numpy(),
           "status": st.cpu().numpy()}
    assert_same_decode(res, ref, "host-buffer decode")
    assert int(scratch.abs().sum()) == 0


@pytest.fixture(scope="module")
def gts_batches():
    """Plain GTS blocks (w = 0): a batch of them alone and one mixing them with
    GTS-Reuse blocks of both reuse widths, all three limits, several b."""
    rng = np.random.Generator(np.random.PCG64(45))
    hf = G.height_field_disc(20_000, seed=8)
    gts = [
        O.encode_mesh(G.uv_sphere(9_000, rng), (64, 126), 16, 2),
        O.encode_mesh(G.torus(7_000, rng), (128, 128), lambda n: G.meshlet_bits(n, 1), 2,
                      perm=lambda n: G.meshlet_permutation(n, 2)),
        O.encode_mesh(hf, np.array(G.SECTOR_LIMITS).reshape(-1), 20, 2),
        O.encode_mesh(G.grid_mesh(5), (8, 5), 7, 2),
    ]
    reuse = [O.encode_mesh(G.torus(5_000, rng), (64, 126), 16, 0),
             O.encode_mesh(G.uv_sphere(6_000, rng), (256, 256), 12, 1)]
    return O.concat(gts), O.concat([gts[0], reuse[0], gts[1], reuse[1], gts[3]])


@pytest.mark.parametrize("which", [0, 1])
@pytest.mark.parametrize("tuning", [None, {"warps_per_cta": 4, "meshlets_per_grab": 1},
                                    {"warps_per_cta": 16, "meshlets_per_grab": 8},
                                    {"warps_per_cta": 8, "checked": 1}] + PAIR_TUNINGS)
def test_plain_gts_batch_vs_oracle(gts_batches, which, tuning):
    blob = gts_batches[which]
    ref = O.decode(blob)
    db = device_batch_from_oracle(blob)
    assert_same_decode(run_decode(db, "batch", tuning), ref, f"gts batch {which} {tuning}")
    if tuning is None:
        assert_same_decode(run_decode(db, "plain", {"checked": 1}), ref, f"gts plain {which}")


def test_plain_gts_corrupt_entry_flagged(gts_batches):
    """An entry naming a vertex that was never introduced: the checked kernels
    report MC_ERR_CORRUPT, the unchecked ones still finish."""
    blob = gts_batches[0]
    f = blob.fields()
    m = int(np.argmax(f["Tp"]))
    tp = int(f["Tp"][m])
    start = 16 * int(f["off16"][m]) + 4 * ((tp + 31) // 32)
    bad = blob.payload.copy()
    ent = bad[start:start + tp - 1]
    bad[start + int(np.argmax(ent == ent.max()))] = min(255, int(ent.max()) + 1)
    broken = O.Blob(blob.desc, bad, blob.grids)
    db = device_batch_from_oracle(broken)
    for mode in ("batch", "plain"):
        res = run_decode(db, mode, {"checked": 1})
        assert int(res["status"][0]) & (1 << 3), mode
    res = run_decode(db, "batch", PAIR_TUNINGS[-1])
    assert int(res["status"][0]) & (1 << 3), "pairs"

    res = run_decode(db, "batch")
    assert int(res["status"][0]) == 0
