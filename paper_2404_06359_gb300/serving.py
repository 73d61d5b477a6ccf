"""Serving loop: continuous batching of decode requests over a resident pool.

Meshes of different sizes arrive as a Poisson stream.  Their compressed
meshlets live in one device-resident pool batch; each request names a mesh
and needs decoded output buffers (u8 local + u32 global indices, FP32
positions), carved out of a fixed HBM budget by a first-fit allocator.  A
request is admitted when its buffers fit the budget and an in-flight slot is
free; admitted requests are packed into the next `mc_decode_requests`
launch (one persistent kernel over all their meshlets) on one of several
streams, so requests that arrive while others are on the GPU join the next
launch and their work overlaps on the device.  Completion is observed through
CUDA events; latency = arrival -> completion of the launch holding the
request, on the device clock referenced to the host clock at start-up.
"""
from __future__ import annotations

import time
from collections import deque
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np

from . import codec as mc
from . import meshgen as G

ALIGN = 256


class FirstFit:
    """First-fit allocator over [0, capacity) bytes (offsets ALIGN-aligned)."""

    def __init__(self, capacity: int):
        self.capacity = capacity
        self.free = [(0, capacity)]  # sorted, disjoint (offset, size)
        self.used = 0
        self.peak = 0

    def alloc(self, size: int):
        size = (size + ALIGN - 1) // ALIGN * ALIGN
        for i, (off, sz) in enumerate(self.free):
            if sz >= size:
                if sz == size:
                    self.free.pop(i)
                else:
                    self.free[i] = (off + size, sz - size)
                self.used += size
                self.peak = max(self.peak, self.used)
                return off, size
        return None

    def release(self, off: int, size: int):
        self.used -= size
        i = 0
        while i < len(self.free) and self.free[i][0] < off:
            i += 1
        self.free.insert(i, (off, size))
        # merge with neighbours
        if i + 1 < len(self.free) and off + size == self.free[i + 1][0]:
            self.free[i] = (off, size + self.free[i + 1][1])
            self.free.pop(i + 1)
        if i > 0 and self.free[i - 1][0] + self.free[i - 1][1] == self.free[i][0]:
            self.free[i - 1] = (self.free[i - 1][0], self.free[i - 1][1] + self.free[i][1])
            self.free.pop(i)


def out_bytes(n_tris: int, n_verts: int) -> tuple[int, int, int]:
    """Aligned sizes of a request's local, global and position buffers."""
    a = lambda n: (n + ALIGN - 1) // ALIGN * ALIGN  # noqa: E731
    return a(3 * n_tris), a(12 * n_tris), a(12 * n_verts)


def build_pool(n_meshes: int = 128, t_lo: int = 1_000, t_hi: int = 2_000_000, seed: int = G.SEED_BASE + 5,
               threads: int = 0):
    """Seeded pool: spheres, tori and height fields with log-uniform triangle
    counts, each meshletized at one of the three meshlet limits (random),
    w = ceil(log2 V), 16-bit positions; concatenated into one batch."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = []
    for i in range(n_meshes):
        t = int(round(np.exp(rng.uniform(np.log(t_lo), np.log(t_hi)))))
        kind = int(rng.integers(0, 3))
        lim = G.SECTOR_LIMITS[int(rng.integers(0, 3))]
        specs.append((i, t, kind, lim, int(rng.integers(0, 2 ** 31))))

    def make(spec):
        i, t, kind, lim, s = spec
        r = np.random.Generator(np.random.PCG64(s))
        if kind == 0:
            m = G.uv_sphere(t, r)
        elif kind == 1:
            m = G.torus(t, r)
        else:
            m = G.height_field_disc(t, seed=s)
            m.tri_class = None
        ml = mc.mc_meshletize(m.tris, m.n_verts, [lim], None, n_threads=1)
        blob = mc.mc_encode(ml, m.pos, 16, 1, mesh_id=i, n_threads=1)
        return blob, m.n_tris
    with ThreadPoolExecutor(threads or None) as ex:
        out = list(ex.map(make, specs))
    pool = mc.mc_blob_concat([b for b, _ in out])
    return pool, [t for _, t in out]


@dataclass
class Request:
    rid: int
    mesh: int
    arrival: float          # seconds since start
    admitted: float = -1.0
    done: float = -1.0
    launch: int = -1
    alloc: tuple = ()
    outputs: dict = field(default_factory=dict)


class Server:
    """Continuous-batching decode server over a resident pool (see module doc)."""

    def __init__(self, pool_blob, budget_bytes: int = 8 << 30, n_streams: int = 4,
                 max_inflight: int = 256, max_batch: int = 64, device="cuda", tuning=None):
        import torch
        self.torch = torch
        self.db = mc.DeviceBatch(pool_blob, device)
        self.meshes = self.db.meshes
        self.budget = FirstFit(budget_bytes)
        self.slab = torch.empty(budget_bytes, dtype=torch.uint8, device=device)
        self.base = self.slab.data_ptr()
        self.streams = [torch.cuda.Stream() for _ in range(n_streams)]
        self.scratch = [mc.new_scratch(device) for _ in range(n_streams)]
        self.status = torch.zeros(1, dtype=torch.int32, device=device)
        self.max_inflight = max_inflight
        self.max_batch = max_batch
        self.tuning = tuning
        # request tables: one pinned host + device pair per stream
        self.h_tab = [torch.empty(max_batch * 64, dtype=torch.uint8).pin_memory() for _ in range(n_streams)]
        self.d_tab = [torch.empty(max_batch * 64, dtype=torch.uint8, device=device) for _ in range(n_streams)]
        self.busy = [None] * n_streams   # (event, [requests]) in flight per stream
        self.launches = 0

    def need(self, mesh: int) -> int:
        mi = self.meshes[mesh]
        return sum(out_bytes(mi["n_tris"], mi["n_verts"]))

    def _launch(self, si: int, batch: list, t0_event, keep_outputs: bool):
        torch = self.torch
        tab = np.zeros(len(batch), mc.REQUEST_DTYPE)
        work = 0
        for i, rq in enumerate(batch):
            mi = self.meshes[rq.mesh]
            off = rq.alloc[0]
            bl, bg, _ = out_bytes(mi["n_tris"], mi["n_verts"])
            tab[i] = (mi["first_meshlet"], mi["n_meshlets"], work, 0, mi["tri_base"], mi["vertex_base"],
                      mi["n_tris"], mi["n_verts"], self.base + off, self.base + off + bl,
                      self.base + off + bl + bg, 0)
            work += mi["n_meshlets"]
        raw = tab.view(np.uint8)
        s = self.streams[si]
        self.h_tab[si][: raw.size].copy_(torch.from_numpy(raw))
        with torch.cuda.stream(s):
            self.d_tab[si][: raw.size].copy_(self.h_tab[si][: raw.size], non_blocking=True)
            mc.mc_decode_requests(self.db, self.d_tab[si], len(batch), work, self.status,
                                  self.scratch[si], self.tuning, s)
            ev = torch.cuda.Event(enable_timing=True)
            ev.record(s)
        self.busy[si] = (ev, batch)
        self.launches += 1
        for rq in batch:
            rq.launch = self.launches

    def _retire(self, si: int, t0_event, t_ref: float, keep_outputs: bool, done: list):
        ev, batch = self.busy[si]
        t_done = t_ref + t0_event.elapsed_time(ev) * 1e-3
        for rq in batch:
            rq.done = t_done
            if keep_outputs:
                rq.outputs = self.read_outputs(rq)
            self.budget.release(*rq.alloc)
            done.append(rq)
        self.busy[si] = None

    def read_outputs(self, rq: Request) -> dict:
        mi = self.meshes[rq.mesh]
        off = rq.alloc[0]
        bl, bg, bp = out_bytes(mi["n_tris"], mi["n_verts"])
        T, V = mi["n_tris"], mi["n_verts"]
        s = self.slab
        return {"local": s[off: off + 3 * T].cpu().numpy().copy(),
                "global": s[off + bl: off + bl + 12 * T].cpu().numpy().view(np.uint32).copy(),
                "pos": s[off + bl + bg: off + bl + bg + 12 * V].cpu().numpy().view(np.float32).copy()}

    def run(self, arrivals: np.ndarray, mesh_ids: np.ndarray, keep_outputs: bool = False,
            realtime: bool = True, poll_sleep: float = 0.0):
        """Serves the requests; returns (completed requests, stats)."""
        torch = self.torch
        reqs = [Request(i, int(m), float(t)) for i, (t, m) in enumerate(zip(arrivals, mesh_ids))]
        for rq in reqs:
            if self.need(rq.mesh) > self.budget.capacity:
                raise ValueError(f"mesh {rq.mesh} needs more than the whole budget")
        pending = deque()
        admitted = deque()
        done: list = []
        nxt = 0
        inflight = 0
        t0_event = torch.cuda.Event(enable_timing=True)
        t0_event.record(self.streams[0])
        t0_event.synchronize()
        t_ref = 0.0
        start = time.perf_counter()
        rr = 0
        while len(done) < len(reqs):
            now = time.perf_counter() - start if realtime else float("inf")
            while nxt < len(reqs) and reqs[nxt].arrival <= now:
                pending.append(reqs[nxt])
                nxt += 1
            # retire finished launches
            for si in range(len(self.streams)):
                if self.busy[si] is not None and self.busy[si][0].query():
                    inflight -= len(self.busy[si][1])
                    self._retire(si, t0_event, t_ref, keep_outputs, done)
            # admit in arrival order while memory and slots allow
            while pending and inflight + len(admitted) < self.max_inflight:
                rq = pending[0]
                a = self.budget.alloc(self.need(rq.mesh))
                if a is None:
                    break
                rq.alloc = a
                rq.admitted = time.perf_counter() - start
                admitted.append(pending.popleft())
            # launch the admitted requests on a free stream
            if admitted:
                for k in range(len(self.streams)):
                    si = (rr + k) % len(self.streams)
                    if self.busy[si] is None:
                        batch = [admitted.popleft() for _ in range(min(self.max_batch, len(admitted)))]
                        inflight += len(batch)
                        self._launch(si, batch, t0_event, keep_outputs)
                        rr = si + 1
                        break
            if poll_sleep:
                time.sleep(poll_sleep)
        torch.cuda.synchronize()
        wall = time.perf_counter() - start
        status = int(self.status.item())
        lat = np.array([rq.done - rq.arrival for rq in done])
        tris = sum(self.meshes[rq.mesh]["input_tris"] for rq in done)
        stats = {"requests": len(done), "launches": self.launches, "wall_s": wall,
                 "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                 "mean_batch": len(done) / max(1, self.launches),
                 "input_triangles": int(tris), "gtps": tris / wall / 1e9,
                 "peak_budget_bytes": self.budget.peak, "status": status}
        return done, stats
