"""Test-side packer: hand-made strip streams -> blobs in the documented format.

Used to feed decoders (oracle and GPU) with streams that no encoder produced:
textbook strips/fans, exhaustive enumerations, corrupt inputs.  Written from
the format description only (32-byte descriptor; payload of L/R words,
increment words, reuse bits, position bits; 32-byte grid entries).
"""
from __future__ import annotations

import itertools

import numpy as np


def ceil_log2(v: int) -> int:
    w = 0
    while (1 << w) < v:
        w += 1
    return w


def _put(words: np.ndarray, bit: int, nbits: int, value: int):
    for i in range(nbits):
        if (value >> i) & 1:
            words[(bit + i) >> 5] |= np.uint32(1 << ((bit + i) & 31))


def pack(cases, reuse_w=8, pos_bits=1, q_fn=None, L=(0, 0, 0), grid=(0.0, 0.0, 0.0, 1.0, 1.0, 1.0)):
    """cases: iterable of (flags[T'], stream[T'+2]) with stream a restricted
    growth sequence starting 0,1,2 (local ids).  reuse_w: int or 'log2'.
    Returns (desc uint8[M,32], payload uint8[...], grids uint8[1,32])."""
    descs, pay = [], []
    off_words = 0
    vbase = tbase = 0
    for flags, stream in cases:
        flags = [int(x) for x in flags]
        stream = [int(x) for x in stream]
        tp = len(flags)
        assert len(stream) == tp + 2 and stream[:3] == [0, 1, 2]
        inc, reuse, seen = [0] * tp, [], 3
        for k in range(1, tp):
            n = stream[k + 2]
            if n == seen:
                inc[k] = 1
                seen += 1
            else:
                assert n < seen
                reuse.append(n)
        V, R = seen, len(reuse)
        w = ceil_log2(V) if reuse_w == "log2" else int(reuse_w)
        nw = (tp + 31) // 32
        rw = (R * w + 31) // 32
        pw = (3 * V * pos_bits + 31) // 32
        n = (2 * nw + rw + pw + 3) // 4 * 4
        words = np.zeros(n, np.uint32)
        for k in range(tp):
            _put(words, k, 1, flags[k])
            _put(words, 32 * nw + k, 1, inc[k])
        for r, val in enumerate(reuse):
            _put(words, 32 * 2 * nw + r * w, w, val)
        for v in range(V):
            for c in range(3):
                q = 0 if q_fn is None else int(q_fn(v, c))
                _put(words, 32 * (2 * nw + rw) + (3 * v + c) * pos_bits, pos_bits, q)
        d = np.zeros(8, np.uint32)
        d[0], d[1], d[2] = off_words // 4, vbase, tbase
        d[3] = V | (tp << 16)
        d[4] = w | (pos_bits << 8) | (0 << 16)
        d[5:8] = L
        descs.append(d)
        pay.append(words)
        off_words += n
        vbase += V
        tbase += tp
    g = np.zeros(8, np.uint32)
    gf = g.view(np.float32)
    gf[0:3] = grid[0:3]
    g[3] = pos_bits
    gf[4:7] = grid[3:6]
    desc = np.stack(descs).astype(np.uint32).view(np.uint8).reshape(-1, 32)
    payload = np.concatenate(pay).view(np.uint8)
    return desc, payload, g.view(np.uint8).reshape(1, 32)


def restricted_growth(length: int, seen: int = 3):
    """All index streams n_1..n_length where each entry is either the next new
    vertex (== number seen so far) or any earlier one."""
    if length == 0:
        yield ()
        return
    for first in range(seen + 1):
        for rest in restricted_growth(length - 1, seen + (first == seen)):
            yield (first,) + rest


def enumerate_cases(tp: int):
    """Every (flags, stream) pair with T' = tp: flag 0 fixed to 0."""
    streams = [(0, 1, 2) + s for s in restricted_growth(tp - 1)]
    for fl in itertools.product((0, 1), repeat=tp - 1):
        flags = (0,) + fl
        for s in streams:
            yield flags, s


def closed_form(flags: np.ndarray, stream: np.ndarray) -> np.ndarray:
    """Parallel-style decode written from Sec. 4.2: for triangle k the third
    vertex is the stream entry just before the last earlier triangle whose
    L/R flag differs from flag k (stream entry 0 when none differs); right
    triangles are (I[k+1], old, I[k+2]), left ones (old, I[k+1], I[k+2]).
    flags [N, T'], stream [N, T'+2] -> triangles [N, T', 3]."""
    N, tp = flags.shape
    out = np.zeros((N, tp, 3), np.int64)
    for k in range(tp):
        j = np.full(N, -1, np.int64)
        for jj in range(k):
            diff = flags[:, jj] != flags[:, k]
            j = np.where(diff, jj, j)
        old = stream[np.arange(N), j + 1]
        prev, cur = stream[:, k + 1], stream[:, k + 2]
        right = flags[:, k] == 1
        out[:, k, 0] = np.where(right, prev, old)
        out[:, k, 1] = np.where(right, old, prev)
        out[:, k, 2] = cur
    return out


def pack_small(flags: np.ndarray, stream: np.ndarray):
    """Vectorised ``pack`` for many cases with the same T' <= 8, w = 8, b = 1,
    all q = 0, each meshlet in its own 8-word (32-byte) payload slot."""
    N, tp = flags.shape
    assert tp <= 8 and stream.shape == (N, tp + 2)
    F = np.zeros(N, np.uint64)
    INC = np.zeros(N, np.uint64)
    seen = np.full(N, 3, np.int64)
    R = np.zeros(N, np.int64)
    reuse_bits = np.zeros(N, np.uint64)
    for k in range(tp):
        F |= flags[:, k].astype(np.uint64) << np.uint64(k)
        if k == 0:
            continue
        n = stream[:, k + 2].astype(np.int64)
        new = n == seen
        INC |= new.astype(np.uint64) << np.uint64(k)
        reuse_bits |= np.where(new, 0, n).astype(np.uint64) << (np.uint64(8) * R.astype(np.uint64))
        R += (~new).astype(np.int64)
        seen += new.astype(np.int64)
    V = seen
    rw = (R * 8 + 31) // 32
    words = np.zeros((N, 8), np.uint32)
    words[:, 0] = F.astype(np.uint32)
    words[:, 1] = INC.astype(np.uint32)
    words[:, 2] = (reuse_bits & np.uint64(0xFFFFFFFF)).astype(np.uint32)
    words[:, 3] = (reuse_bits >> np.uint64(32)).astype(np.uint32)
    # position words sit right after the reuse words and are all zero (q = 0)
    words[rw == 0, 2] = 0
    words[rw <= 1, 3] = 0
    d = np.zeros((N, 8), np.uint32)
    d[:, 0] = 2 * np.arange(N)
    d[:, 1] = np.concatenate([[0], np.cumsum(V)[:-1]])
    d[:, 2] = tp * np.arange(N)
    d[:, 3] = V.astype(np.uint32) | (tp << 16)
    d[:, 4] = 8 | (1 << 8)
    g = np.zeros(8, np.uint32)
    g.view(np.float32)[4:7] = 1.0
    g[3] = 1
    return (d.view(np.uint8).reshape(-1, 32), words.reshape(-1).view(np.uint8),
            g.view(np.uint8).reshape(1, 32), V)
