"""A bounded device wait that runs out, on the GPU, without a hang or a trap.

The ordered fused cull resolves each grab's output position by a look-back
over its predecessors' published survivor counts (a wait on global memory
only).  Here the work queue is started past grab 0, so grab 0 is never
decoded and its state word is never published: every later grab's
look-back must give up after the short limit set in mc_tuning.wait_cycles,
report MC_ERR_TIMEOUT in the status word, and the kernel must still finish
and leave its scratch reset.  The same context then decodes correctly.
"""
import numpy as np
import pytest

import oracle as O
from paper_2404_06359_gb300 import codec as mc
from paper_2404_06359_gb300 import meshgen as G
from tests.gpu_util import device_batch_from_oracle

pytestmark = pytest.mark.gpu


def test_ordered_lookback_gives_up_on_an_unpublished_grab():
    import torch
    blob = O.encode_mesh(G.grid_mesh(48), (64, 126), 16, 0)
    assert blob.n_meshlets > 12
    db = device_batch_from_oracle(blob)
    T, V = db.stats["total_tris"], db.stats["total_verts"]
    c = np.array([24.0, 24.0, 0.0])
    vp = G.camera_poses(1, c, 40.0, seed=3)[0]
    d_vp = torch.from_numpy(np.ascontiguousarray(vp, np.float32)).cuda()
    tri = torch.zeros(3 * T + 3, dtype=torch.int32, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    pos = torch.zeros(3 * V, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    tune = {"warps_per_cta": 4, "meshlets_per_grab": 3, "wait_cycles": 100_000}
    scratch = mc.new_scratch()
    scratch[0] = 3  # the queue starts at meshlet 3: grab 0 is never taken
    mc.mc_decode_cull_ordered(db, d_vp, tri, cnt, pos, st, scratch, None, tune)
    torch.cuda.synchronize()
    assert int(st.item()) & (1 << mc.MC_ERR_TIMEOUT)
    assert int(scratch.abs().sum()) == 0
    # the context is intact: the same call from an empty queue is the oracle's result
    st.zero_()
    mc.mc_decode_cull_ordered(db, d_vp, tri, cnt, pos, st, scratch, None,
                              {"warps_per_cta": 4, "meshlets_per_grab": 3})
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    ref, _, _ = O.decode_cull(blob, vp)
    assert int(cnt.item()) == ref.shape[0]
    got = tri[: 3 * int(cnt.item())].cpu().numpy().view(np.uint32).reshape(-1, 3)
    assert np.array_equal(got, ref)
