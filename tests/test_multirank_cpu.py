"""The benchmark's multi-rank host logic on 2 gloo processes (CPU): barrier,
max-over-ranks timing and whole-job aggregation, and per-rank seeding of the
workloads (each rank decodes its own batch; there is no data-path
collective)."""
import os
import socket

import numpy as np
import torch.multiprocessing as tmp



def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    import numpy as np
    import torch.distributed as dist
    import bench
    from paper_2404_06359_gb300 import meshgen as G
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    bench._barrier(ws)
    t = bench._allreduce_max(10.0 + 5.0 * rank, ws)
    meshes = G.surface_batch(2, 1000, 2000, G.SEED_BASE + 2 + 1000 * rank)
    q.put((rank, t, float(meshes[0].pos.astype(np.float64).sum()) + meshes[0].n_tris, dist.get_world_size()))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = tmp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [15.0, 15.0]          # both see the slowest rank
    assert res[0][2] != res[1][2]                       # ranks decode different batches
    assert all(r[3] == 2 for r in res)


def test_aggregate_is_whole_job():
    import bench
    # two ranks, 1e6 triangles each per step, 10 steps in 2 ms (slowest rank)
    assert np.isclose(bench.aggregate_gtps(2, 1_000_000, 10, 2.0), 10.0)
