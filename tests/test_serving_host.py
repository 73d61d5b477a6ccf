"""Host-side logic of the serving loop (no GPU): the first-fit HBM budget
allocator never overlaps, never exceeds its capacity and coalesces freed
space."""
import numpy as np

from paper_2404_06359_gb300.serving import ALIGN, FirstFit, out_bytes


def test_first_fit_random_workload():
    rng = np.random.Generator(np.random.PCG64(1))
    cap = 1 << 20
    a = FirstFit(cap)
    live = {}
    for step in range(5000):
        if live and (rng.random() < 0.45 or len(live) > 200):
            k = list(live)[int(rng.integers(0, len(live)))]
            a.release(*live.pop(k))
        else:
            got = a.alloc(int(rng.integers(1, 40_000)))
            if got is not None:
                live[step] = got
        spans = sorted(live.values())
        for (o1, s1), (o2, _) in zip(spans, spans[1:]):
            assert o1 + s1 <= o2
        assert all(o % ALIGN == 0 and o + s <= cap for o, s in spans)
        assert a.used == sum(s for _, s in spans) <= cap
        free = sorted(a.free)
        assert all(f1[0] + f1[1] < f2[0] for f1, f2 in zip(free, free[1:]))  # coalesced
    for o, s in list(live.values()):
        a.release(o, s)
    assert a.free == [(0, cap)] and a.used == 0


def test_out_bytes_aligned():
    l, g, p = out_bytes(1001, 600)
    assert l >= 3003 and g >= 12012 and p >= 7200
    assert l % ALIGN == g % ALIGN == p % ALIGN == 0
