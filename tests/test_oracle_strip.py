"""Pins of the oracle's strip decoding against definitions outside the oracle.

* Textbook primitives (tests/golden/gl_strip_fan.json, OpenGL triangle strips
  and fans): alternating flags must decode as a triangle strip (the paper's
  ATS, Sec. 2), constant flags as fans -- at lengths past one 32-bit word
  (Sec. 4.2: fans longer than 31 triangles need the earlier flag words).
* Brute force: every flag word and every first-appearance stream with
  T' <= 7 decodes identically under the oracle's sequential walk and under
  the parallel closed form of Sec. 4.2/4.3 restated in tests/blobpack.py.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
from tests import blobpack as bp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "gl_strip_fan.json")


def _blob(cases, **kw):
    desc, payload, grids = bp.pack(cases, **kw)
    return O.Blob(desc, payload, grids)


def _decode_all(blob):
    loc, _, _, _ = O.decode(blob, want_pos64=False)
    return loc.astype(np.int64)


def _gl_strip(n_verts):
    return [(i, i + 1, i + 2) if i % 2 == 0 else (i + 1, i, i + 2) for i in range(n_verts - 2)]


def _gl_fan(center, rim):
    return [(center, rim[i], rim[i + 1]) for i in range(len(rim) - 1)]


def _canon(t):
    t = tuple(int(x) for x in t)
    i = t.index(min(t))
    return t[i:] + t[:i]


def test_golden_fixture_matches_gl_rules():
    g = json.load(open(GOLDEN))
    assert [tuple(t) for t in g["strip_8"]] == _gl_strip(8)
    assert [tuple(t) for t in g["fan_8"]] == _gl_fan(0, list(range(1, 8)))
    fan1 = _gl_fan(1, [7, 6, 5, 4, 3, 2, 0])[::-1]
    assert [_canon(t) for t in g["fan_about_1_8"]] == [_canon(t) for t in fan1]


def test_alternating_flags_decode_as_strip_golden():
    g = json.load(open(GOLDEN))
    flags = [0, 1, 0, 1, 0, 1]
    blob = _blob([(flags, list(range(8)))])
    assert _decode_all(blob).tolist() == g["strip_8"]


def test_left_flags_decode_as_fan_golden():
    g = json.load(open(GOLDEN))
    blob = _blob([([0] * 6, list(range(8)))])
    assert _decode_all(blob).tolist() == g["fan_8"]


def test_right_flags_decode_as_fan_about_1_golden():
    g = json.load(open(GOLDEN))
    blob = _blob([([0] + [1] * 5, list(range(8)))])
    assert _decode_all(blob).tolist() == g["fan_about_1_8"]


@pytest.mark.parametrize("tp", [3, 31, 32, 33, 64, 65, 200, 254])  # V = T' + 2 <= 256
def test_long_strips_and_fans(tp):
    stream = list(range(tp + 2))
    strip = [0] + [(k % 2) for k in range(1, tp)]          # R at odd k
    fan_l = [0] * tp
    fan_r = [0] + [1] * (tp - 1)
    loc = _decode_all(_blob([(strip, stream), (fan_l, stream), (fan_r, stream)], reuse_w=8,
                            pos_bits=1))
    assert loc[:tp].tolist() == [list(t) for t in _gl_strip(tp + 2)]
    assert loc[tp:2 * tp].tolist() == [list(t) for t in _gl_fan(0, list(range(1, tp + 2)))]
    rim = list(range(tp + 1, 1, -1)) + [0]
    fan1 = [_canon(t) for t in _gl_fan(1, rim)[::-1]]
    assert [_canon(t) for t in loc[2 * tp:]] == fan1


def test_fan_after_strip_across_word_boundary():
    """A strip part followed by a 40-triangle fan: the fan pivot lies in the
    previous flag word for the late triangles (Sec. 4.2)."""
    head = [0, 1, 0, 1, 0, 1]            # triangles 0..5 alternate
    tp = len(head) + 40
    flags = head + [1] * 40              # then a run of right turns
    stream = list(range(tp + 2))
    loc = _decode_all(_blob([(flags, stream)]))
    # triangle 5 is (I6?..): after the alternating head the last triangle is
    # (6, 5, 7) (GL strip rule, odd index); a run of right turns pivots on its
    # middle vertex 5: (7, 5, 8), (8, 5, 9), ...
    assert tuple(loc[5]) == (6, 5, 7)
    for i, k in enumerate(range(6, tp)):
        assert tuple(loc[k]) == (7 + i, 5, 8 + i)


@pytest.mark.parametrize("tp", [1, 2, 3, 4, 5, 6, 7])
def test_bruteforce_walk_equals_closed_form(tp):
    cases = list(bp.enumerate_cases(tp))
    flags = np.array([c[0] for c in cases], np.int64)
    stream = np.array([c[1] for c in cases], np.int64)
    desc, payload, grids, V = bp.pack_small(flags, stream)
    blob = O.Blob(desc, payload, grids)
    loc, glob, pos, _ = O.decode(blob, want_pos64=False)
    got = loc.astype(np.int64).reshape(len(cases), tp, 3)
    want = bp.closed_form(flags, stream)
    assert np.array_equal(got, want)
    # global = vertex_base + local; positions all at the grid origin (q = 0)
    vb = blob.fields()["vertex_base"].astype(np.int64)
    assert np.array_equal(glob.reshape(len(cases), tp, 3).astype(np.int64), want + vb[:, None, None])
    assert np.all(pos == 0)


def test_bruteforce_count_t8_sample():
    """T' = 8 (the largest size named in the brute-force pin): a seeded sample
    of 200k of the ~7.7 M cases (the full corpus runs in the GPU suite)."""
    rng = np.random.Generator(np.random.PCG64(8))
    streams = np.array([(0, 1, 2) + s for s in bp.restricted_growth(7)], np.int64)
    n = 200_000
    flags = np.concatenate([np.zeros((n, 1), np.int64), rng.integers(0, 2, (n, 7))], 1)
    stream = streams[rng.integers(0, streams.shape[0], n)]
    desc, payload, grids, V = bp.pack_small(flags, stream)
    loc, _, _, _ = O.decode(O.Blob(desc, payload, grids), want_pos64=False)
    assert np.array_equal(loc.astype(np.int64).reshape(n, 8, 3), bp.closed_form(flags, stream))


def test_reuse_widths_and_position_bits():
    """Reuse entries at w = ceil(log2 V) and positions at odd bit widths
    straddling word boundaries decode to the packed values."""
    rng = np.random.Generator(np.random.PCG64(5))
    cases = []
    for tp in (5, 17, 33, 70, 130, 256):
        s = [0, 1, 2]
        seen = 3
        for _ in range(tp - 1):
            if rng.random() < 0.5 and seen < 256:
                s.append(seen)
                seen += 1
            else:
                s.append(int(rng.integers(0, seen)))
        cases.append(([0] + list(rng.integers(0, 2, tp - 1)), s))
    for b in (1, 7, 12, 16, 20, 31, 32):
        qs = {}

        def q_fn(v, c, b=b):
            qs[(v, c)] = int(rng.integers(0, 2 ** b))
            return qs[(v, c)]
        for bi, (flags, s) in enumerate(cases):
            qs.clear()
            desc, payload, grids = bp.pack([(flags, s)], reuse_w="log2", pos_bits=b, q_fn=q_fn,
                                           grid=(0.0, 0.0, 0.0, 1.0, 1.0, 1.0))
            blob = O.Blob(desc, payload, grids)
            loc, pos, pos64 = O.decode_meshlet(blob, 0)
            st = np.array(s, np.int64)[None]
            want = bp.closed_form(np.array(flags, np.int64)[None], st)[0]
            assert np.array_equal(loc.astype(np.int64), want)
            for (v, c), q in qs.items():
                assert pos64[v, c] == float(q)      # G = 0, Delta = 1: x = g = q


def test_corrupt_streams_rejected():
    good = ([0, 1, 0, 1], [0, 1, 2, 3, 4, 5])
    desc, payload, grids = bp.pack([good])
    O.decode(O.Blob(desc, payload, grids))
    # bit 0 of the L/R word must be 0
    p2 = payload.copy().view(np.uint32)
    p2[0] |= 1
    with pytest.raises(O.OracleError):
        O.decode(O.Blob(desc, p2.view(np.uint8), grids))
    # V that disagrees with the increment flags
    d2 = desc.copy().view(np.uint32)
    d2[0, 3] = (d2[0, 3] & 0xFFFF0000) | 5
    with pytest.raises(O.OracleError):
        O.decode(O.Blob(d2.view(np.uint8), payload, grids))
    # payload offset beyond the payload
    d3 = desc.copy().view(np.uint32)
    d3[0, 0] = 1000
    with pytest.raises(O.OracleError):
        O.decode(O.Blob(d3.view(np.uint8), payload, grids))

