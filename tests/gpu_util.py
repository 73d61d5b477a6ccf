"""Shared helpers of the GPU parity tests (no computation of the method here:
blob bookkeeping and comparisons only)."""
from __future__ import annotations

import numpy as np

import oracle as O
from paper_2404_06359_gb300 import codec as mc


def block_words_max(desc: np.ndarray, n_attr: int = 0, attr_bits: int = 0) -> int:
    w = desc.view(np.uint32).reshape(-1, 8)
    V = (w[:, 3] & 0xFFFF).astype(np.int64)
    T = (w[:, 3] >> 16).astype(np.int64)
    rw = (w[:, 4] & 0xFF).astype(np.int64)
    b = ((w[:, 4] >> 8) & 0xFF).astype(np.int64)
    R = T + 2 - V
    nw = (T + 31) // 32
    conn = np.where(rw == 0, nw + (T + 2) // 4, 2 * nw + (R * rw + 31) // 32)  # w = 0: plain GTS
    words = conn + (3 * V * b + 31) // 32 + (n_attr * V * attr_bits + 31) // 32
    return int(((words + 3) // 4 * 4).max()) if words.size else 4


def max_tris(desc: np.ndarray) -> int:
    w = desc.view(np.uint32).reshape(-1, 8)
    return int((w[:, 3] >> 16).max()) if w.shape[0] else 1


def max_verts(desc: np.ndarray) -> int:
    w = desc.view(np.uint32).reshape(-1, 8)
    return int((w[:, 3] & 0xFFFF).max()) if w.shape[0] else 3


def device_batch_from_oracle(blob: O.Blob, cones: bool = False) -> mc.DeviceBatch:
    at = blob.attrs
    return mc.DeviceBatch.from_arrays(blob.desc, blob.payload, blob.grids, blob.total_tris,
                                      blob.total_verts,
                                      block_words_max(blob.desc, at["n_attr"] if at else 0,
                                                      at["attr_bits"] if at else 0),
                                      max_tris(blob.desc), cones=blob.cones if cones else None,
                                      attrs=at, max_verts=max_verts(blob.desc))


def run_decode(db: mc.DeviceBatch, mode="batch", tuning=None, local=True, global_=True):
    import torch
    out = db.outputs(local, global_)
    for k in ("local", "global", "pos"):
        if out[k] is not None:
            out[k].fill_(0xFF if k != "pos" else 0)
    if mode == "plain":
        mc.mc_decode_plain(db, 0, db.stats["n_meshlets"], out["local"], out["global"], out["pos"],
                           out["status"], tuning)
    else:
        scratch = mc.new_scratch()
        mc.mc_decode_batch(db, out["local"], out["global"], out["pos"], out["status"], scratch, tuning)
        torch.cuda.synchronize()
        assert int(scratch.abs().sum()) == 0, "work-queue scratch not left zeroed"
    torch.cuda.synchronize()
    res = {k: (None if v is None else v.cpu().numpy()) for k, v in out.items()}
    return res


def assert_same_decode(res: dict, ref, what=""):
    loc, glob, pos, _ = ref
    assert int(res["status"][0]) == 0, f"{what}: device status {int(res['status'][0]):#x}"
    if res["local"] is not None:
        got = res["local"].reshape(-1, 3)
        bad = np.nonzero((got != loc).any(1))[0]
        assert bad.size == 0, f"{what}: {bad.size} local triangles differ, first {bad[:5]}"
    if res["global"] is not None:
        got = res["global"].view(np.uint32).reshape(-1, 3)
        assert np.array_equal(got, glob), f"{what}: global indices differ"
    gp = res["pos"].reshape(-1, 3)
    same = gp.view(np.uint32) == pos.view(np.uint32)
    assert same.all(), f"{what}: {(~same).sum()} position components differ (0 ulp required)"
