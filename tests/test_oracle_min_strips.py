"""Optimality of the strips: the oracle's exact fewest-strips search, pinned,
and the greedy path covers of both encoders measured against it.

The strips of a meshlet are a path cover of its triangles' adjacency graph
(two triangles are adjacent when they share an edge); Sec. 4.1 finds a
minimum one with a MILP (maximise the adjacency edges used, no fork, no
cycle).  orc_min_strips computes the same minimum by branch and bound for
small meshlets, plus a lower bound valid at any size.

Pins of the search, from outside it:
* hand-made graphs whose minimum is known: a row of triangles (one strip),
  a closed fan of six triangles around a vertex (a cycle: one strip), a
  triangle with a neighbour on every edge (a star K_1,3: two strips), two
  triangles far apart (two strips);
* brute force: every subset of the adjacency edges of small meshlets, the
  largest that keeps every triangle on at most two chosen edges and closes no
  cycle (the graph built here from the triangles' directed edges).
"""
import itertools

import numpy as np
import pytest

import oracle as O
from paper_2404_06359_gb300 import meshgen as G


def _adjacency(tris: np.ndarray):
    """Undirected adjacency edges (i < j) of a consistently wound triangle
    set: triangle j holds the directed edge opposite to one of triangle i."""
    owner = {}
    for i, t in enumerate(tris):
        for e in range(3):
            owner[(int(t[e]), int(t[(e + 1) % 3]))] = i
    edges = set()
    for i, t in enumerate(tris):
        for e in range(3):
            j = owner.get((int(t[(e + 1) % 3]), int(t[e])))
            if j is not None and j != i:
                edges.add((min(i, j), max(i, j)))
    return sorted(edges)


def _brute_min_paths(n: int, edges) -> int:
    """n minus the largest edge subset with all degrees <= 2 and no cycle."""
    best = 0
    for r in range(len(edges), 0, -1):
        if r <= best:
            break
        for sub in itertools.combinations(edges, r):
            deg = [0] * n
            parent = list(range(n))

            def find(x):
                while parent[x] != x:
                    parent[x] = parent[parent[x]]
                    x = parent[x]
                return x
            ok = True
            for u, v in sub:
                deg[u] += 1
                deg[v] += 1
                ru, rv = find(u), find(v)
                if deg[u] > 2 or deg[v] > 2 or ru == rv:
                    ok = False
                    break
                parent[ru] = rv
            if ok:
                best = r
                break
    return n - best


def _min(tris, greedy=None):
    ids = np.arange(len(tris), dtype=np.uint32)
    return O.min_strips(np.asarray(tris, np.uint32), ids, greedy or len(tris))


def test_hand_made_graphs():
    row = []  # a row of 5 quads, each split in two: a path of 10 triangles
    for i in range(5):
        a, b, c, d = i, i + 1, 6 + i, 6 + i + 1
        row += [(a, b, d), (a, d, c)]
    assert _min(row) == (1, 1)
    fan = [(0, 1 + i, 1 + (i + 1) % 6) for i in range(6)]  # closed fan: a 6-cycle
    assert _min(fan) == (1, 1)
    star = [(0, 1, 2), (1, 0, 3), (2, 1, 4), (0, 2, 5)]  # K_1,3
    assert _min(star) == (2, 2)
    apart = [(0, 1, 2), (3, 4, 5)]
    assert _min(apart) == (2, 2)


@pytest.mark.parametrize("seed", range(6))
def test_search_equals_brute_force(seed):
    rng = np.random.Generator(np.random.PCG64(100 + seed))
    mesh = [G.uv_sphere(600, rng), G.torus(500, rng), G.height_field_disc(800, seed=seed)][seed % 3]
    mtri, mstart, _ = O.meshletize(mesh.tris, mesh.n_verts, (12, 9))
    checked = 0
    for m in range(len(mstart) - 1):
        ids = mtri[mstart[m]:mstart[m + 1]]
        t = mesh.tris[ids]
        edges = _adjacency(t)
        if len(edges) > 14:
            continue
        mn, lo = O.min_strips(mesh.tris, ids, len(ids))
        assert mn == _brute_min_paths(len(ids), edges), m
        assert lo <= mn
        checked += 1
    assert checked >= 20


def _covers(mesh, limits):
    """Per meshlet: (T, greedy strips, fewest strips or 0, lower bound)."""
    n_classes = 1 if mesh.tri_class is None else int(mesh.tri_class.max()) + 1
    mtri, mstart, _ = O.meshletize(mesh.tris, mesh.n_verts, tuple(limits) * n_classes, mesh.tri_class)
    out = []
    for m in range(len(mstart) - 1):
        ids = mtri[mstart[m]:mstart[m + 1]]
        greedy = O.stripify(mesh.tris, ids)[4]
        mn, lo = O.min_strips(mesh.tris, ids, greedy, max_nodes=2_000_000 if len(ids) <= 24 else 0)
        out.append((len(ids), greedy, mn, lo))
    return np.array(out, np.int64)


def test_greedy_covers_against_the_optimum_on_small_meshlets():
    """Meshlets of at most 24 triangles, searched to the end: the greedy cover
    (best of 16 randomised covers, as both encoders emit it) never uses fewer
    strips than the minimum, and the report gives how often it is optimal."""
    rng = np.random.Generator(np.random.PCG64(7))
    rows = []
    for mesh in (G.uv_sphere(4000, rng), G.torus(4000, rng), G.height_field_disc(5000, seed=3)):
        for lim in ((16, 20), (20, 24), (12, 16)):
            rows.append(_covers(mesh, lim))
    r = np.concatenate(rows)
    done = r[:, 2] > 0
    assert done.mean() > 0.99
    T, greedy, mn, lo = r[done].T
    assert (mn <= greedy).all() and (lo <= mn).all()
    gap = greedy - mn
    print(f"\n{done.sum()} meshlets of <= 24 triangles: greedy optimal in {np.mean(gap == 0):.1%}, "
          f"mean extra strips {gap.mean():.3f}, max {gap.max()}; restarts per meshlet "
          f"greedy {np.mean(greedy - 1):.3f} vs minimum {np.mean(mn - 1):.3f}")
    assert np.mean(gap == 0) > 0.8


def test_lower_bound_at_the_papers_limits():
    """At 128/256 (Tab. 1's setting) no search finishes; every greedy cover is
    at least the endpoint lower bound, and the report puts the restarts per
    meshlet beside Tab. 1 (1.64 with optimal strips, 2.46 with its ETA
    heuristic, on its scanned mesh)."""
    rng = np.random.Generator(np.random.PCG64(8))
    rows = [_covers(m, (128, 256)) for m in (G.uv_sphere(40000, rng), G.torus(40000, rng),
                                             G.height_field_disc(40000, seed=4))]
    r = np.concatenate(rows)
    T, greedy, _, lo = r.T
    assert (lo <= greedy).all()
    print(f"\n{len(r)} meshlets at 128/256: restarts per meshlet {np.mean(greedy - 1):.3f} "
          f"(lower bound {np.mean(lo - 1):.3f}); Tab. 1: 1.64 optimal, 2.46 ETA")
