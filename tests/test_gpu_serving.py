"""GPU checks of the serving path: the multi-request kernel decodes every
request exactly as the oracle decodes its meshlets (renumbered to the
request), and in the continuous-batching loop each request's result is the
same in the mix as when decoded alone."""
import numpy as np
import pytest

import oracle as O
from paper_2404_06359_gb300 import codec as mc
from paper_2404_06359_gb300 import meshgen as G
from paper_2404_06359_gb300 import serving as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    blob, tris = S.build_pool(n_meshes=24, t_lo=1_000, t_hi=60_000, seed=99)
    return blob, tris


def _oracle_request(ob, f, mi):
    """Oracle decode of one mesh's meshlets, renumbered to the mesh."""
    loc, glob, pos, _ = O.decode(ob, mi["first_meshlet"], mi["n_meshlets"], want_pos64=False)
    t0, v0 = mi["tri_base"], mi["vertex_base"]
    T, V = mi["n_tris"], mi["n_verts"]
    return (loc[t0:t0 + T].reshape(-1), (glob[t0:t0 + T] - v0).reshape(-1),
            pos[v0:v0 + V].reshape(-1))


def _one_launch(srv, meshes_idx):
    import torch
    reqs = [S.Request(i, int(m), 0.0) for i, m in enumerate(meshes_idx)]
    for rq in reqs:
        rq.alloc = srv.budget.alloc(srv.need(rq.mesh))
    srv._launch(0, reqs, None, True)
    torch.cuda.synchronize()
    outs = [srv.read_outputs(rq) for rq in reqs]
    for rq in reqs:
        srv.budget.release(*rq.alloc)
    srv.busy[0] = None
    return outs


def test_requests_kernel_vs_oracle(pool):
    blob, _ = pool
    srv = S.Server(blob, budget_bytes=1 << 30, n_streams=2)
    a = blob.arrays()
    ob = O.Blob(a["desc"], a["payload"], a["grids"])
    f = ob.fields()
    order = np.random.Generator(np.random.PCG64(5)).permutation(len(srv.meshes))
    outs = _one_launch(srv, order)
    assert int(srv.status.item()) == 0
    for m, out in zip(order, outs):
        rl, rg, rp = _oracle_request(ob, f, srv.meshes[m])
        assert np.array_equal(out["local"], rl)
        assert np.array_equal(out["global"], rg.astype(np.uint32))
        assert np.array_equal(out["pos"].view(np.uint32), rp.view(np.uint32))


def test_serving_mix_equals_alone(pool):
    blob, _ = pool
    srv = S.Server(blob, budget_bytes=256 << 20, n_streams=3, max_batch=16)
    rng = np.random.Generator(np.random.PCG64(7))
    n = 200
    arrivals = np.sort(rng.uniform(0, 0.05, n))     # a burst: requests overlap on the GPU
    mesh_ids = rng.integers(0, len(srv.meshes), n)
    done, stats = srv.run(arrivals, mesh_ids, keep_outputs=True)
    assert stats["requests"] == n and stats["status"] == 0
    assert stats["launches"] < n                      # requests were batched together
    assert stats["peak_budget_bytes"] <= 256 << 20
    alone = {}
    for m in sorted(set(int(x) for x in mesh_ids)):
        alone[m] = _one_launch(srv, [m])[0]
    for rq in done:
        ref = alone[rq.mesh]
        for k in ("local", "global"):
            assert np.array_equal(rq.outputs[k], ref[k]), (rq.rid, k)
        assert np.array_equal(rq.outputs["pos"].view(np.uint32), ref["pos"].view(np.uint32))
    assert stats["p99_ms"] >= stats["p50_ms"] > 0


def test_admission_waits_for_memory(pool):
    blob, _ = pool
    srv = S.Server(blob, budget_bytes=0, n_streams=2, max_batch=4)
    biggest = max(range(len(srv.meshes)), key=srv.need)
    cap = srv.need(biggest) * 2                       # at most two requests resident
    srv.budget = S.FirstFit(cap)
    srv.slab = __import__("torch").empty(cap, dtype=__import__("torch").uint8, device="cuda")
    srv.base = srv.slab.data_ptr()
    arrivals = np.zeros(12)
    mesh_ids = np.full(12, biggest)
    done, stats = srv.run(arrivals, mesh_ids, keep_outputs=False)
    assert stats["requests"] == 12 and stats["status"] == 0
    assert stats["peak_budget_bytes"] <= cap
    assert stats["launches"] >= 6
