"""Benchmark: batched GTS-Reuse meshlet decode on GB300.

Default workload (cfg2): 256 seeded UV-spheres/tori, ~16.2 M triangles,
meshlets 64/126, 16-bit positions, 8-bit reuse indices, decoded to u8 local +
u32 global indices + FP32 positions by one persistent launch replayed from a
CUDA graph.  One step = one decode of the whole batch (inputs resident in
HBM); L2 is flushed (a write of at least twice its size) between timed steps.
The default run adds a `cfg3` record: the 50 M-triangle height field (mixed
meshlet limits, per-meshlet bit widths, shuffled) measured the same way.

After the timed steps the outputs of the last step are kept and compared,
element for element, with the CPU oracle's decode of the same meshlets (the
oracle run that the `cpu_baseline` leg times); the line's `parity` key says
how many meshlets were compared and how many differed, and any difference
ends the run with a non-zero exit code after the line is printed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config 1|2|3|4|5]
  python bench.py --impl reference ...   # the CPU oracle, same metric

Prints one JSON line (rank 0).  Under torchrun each rank decodes its own
seeded batch (weak scaling, no data-path collective).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "decoded Gtps (bit-exact) & % of HBM roofline vs plain decode; p50/p99 latency"
WORKLOADS = {
    1: "cfg1: 64x64-quad jittered grid, 8,192 triangles, meshlets 64/126, b=16, w=8, "
       "u8 local + f32 positions, plain one-launch decode",
    2: "cfg2: 256 seeded UV-spheres/tori, T log-uniform 10k-200k (16.2M triangles), meshlets "
       "64/126, b=16, w=8, u8 local + u32 global + f32 positions, one persistent launch (CUDA graph)",
    3: "cfg3: 50M-triangle disc height field, 3 sectors at 64/126, 128/128, 256/256, w=ceil(log2 V), "
       "b in {12,16,20} per meshlet, shuffled, u8 + u32 + f32, one persistent launch (CUDA graph)",
    4: "cfg4: cfg2 generator grown to >=50M triangles, fused decode + frustum/normal-cone/back-face cull + "
       "compaction, 64 camera poses, one CUDA graph",
    5: "cfg5: serving loop, Poisson arrivals (2000 meshes/s) over a resident pool of seeded "
       "spheres/tori/height fields (1k-2M triangles, mixed meshlet limits), 8 GB output budget, "
       "continuous batching over 4 streams",
}
L2_NOTE = "flushed between steps (a write of max(256 MB, 2 x L2 + 16 MB) on the timing stream)"


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e nominal, for the second fraction beside the measured peak

# DRAM bytes (read + write) of one launch of the dominant kernel, from an ncu
# capture of the same kernel on the same inputs (cfg2: one decode_batch launch
# on the cfg2 batch; cfg4: one 8-view decode_cull_views launch on the batch
# reduced to 20 M triangles, scaled by decoded triangle slots), per decoded
# triangle slot and keyed by the hash of the kernel source it was taken on;
# reported only while the sources match.
NCU_TRAFFIC = {  # config -> (device-code hash, DRAM bytes per decoded triangle slot)
    2: ("e25682d000018455", (86884608 + 327910912) / 16932154),
    4: ("b09b78db4776337e", (113451008 + 1033029120) / 20923636),
}


def _kernel_hash(config: int):
    """Hash of the device code the config's dominant kernel is built from: the
    shared device headers and its kernel file (kernels.cu for the decoders,
    cull_views.cu with the cull helpers for the multi-view cull), each up to
    its host launchers, with comments and whitespace left out (an edit of a
    comment leaves the captured counters valid)."""
    import hashlib
    import re
    h = hashlib.sha256()
    files = ["cull_views.cu", "cull_common.cuh"] if config == 4 else ["kernels.cu"]
    for p in ["paper_2404_06359_gb300/csrc/device/" + f
              for f in files + ["decode_warp.cuh", "grab_loop.cuh"]]:
        with open(os.path.join(ROOT, p), "rb") as f:
            b = f.read()
        b = b.split(b"// ------------------------------------------------------------- launchers")[0]
        b = re.sub(rb"/\*.*?\*/", b" ", b, flags=re.S)
        b = re.sub(rb"//[^\n]*", b" ", b)
        h.update(re.sub(rb"\s+", b" ", b).strip())
    return h.hexdigest()[:16]


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        vis = os.environ.get("CUDA_VISIBLE_DEVICES")
        phys = device_index
        if vis:
            try:
                phys = int(vis.split(",")[device_index])
            except ValueError:
                phys = device_index
        self.cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                    "-i", str(phys), "-lms", "50"]
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # the timed region starts once sampling runs (nvidia-smi takes a
            # moment to attach), so the samples cover it
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0 and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except Exception:
                self.proc.kill()
            self.t.join(1)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _allreduce_max(x: float, ws: int) -> float:
    """Max over ranks (timing is reported as the slowest rank's)."""
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_gtps(ws: int, tris_per_rank: int, steps: int, max_total_ms: float) -> float:
    """Whole-job throughput: every rank decodes its own batch each step
    (weak scaling), divided by the slowest rank's time."""
    return ws * tris_per_rank * steps / (max_total_ms * 1e-3) / 1e9


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def build_workload(cfg: int, rank: int, codec: str = "reuse", attrs: bool = False,
                   cfg4_tris: int = 50_000_000, strip_search: int = 0):
    from paper_2404_06359_gb300 import workloads as W
    if strip_search and cfg != 2:
        raise SystemExit("--strip-search applies to config 2")
    if cfg == 1:
        blob, meshes = W.cfg1()
        return blob, meshes, None
    if cfg == 2:
        blob, meshes = W.cfg2(rank, plain_gts=codec == "gts", attrs=attrs,
                              strip_search_nodes=strip_search)
        return blob, meshes, None
    if cfg == 3:
        blob, meshes = W.cfg3(rank, plain_gts=codec == "gts")
        return blob, meshes, None
    if cfg == 4:
        return W.cfg4(rank, min_tris=cfg4_tris)
    raise SystemExit(f"unknown config {cfg}")


# ------------------------------------------------------------- the oracle leg
class OracleSample:
    """The oracle's sequential C decode (or, given a view-projection matrix,
    its fused decode + normal-cone/frustum/back-face cull for that view) over
    the first `count` meshlets of the batch, into output arrays allocated
    once (so a timed call pays for no allocation); `count` is sized from a
    probe so that one call takes about budget_s.  arrays: the blob's desc,
    payload, grids (and cones) as numpy arrays."""

    def __init__(self, arrays: dict, budget_s: float, vp=None):
        import oracle as O
        self.O, self.vp = O, vp
        self.a = a = arrays
        self.ob = ob = O.Blob(a["desc"], a["payload"], a["grids"])
        self.n = n = ob.n_meshlets
        T, V = ob.total_tris, ob.total_verts
        self.loc, self.glob = np.zeros(3 * T, np.uint8), np.zeros(3 * T, np.uint32)
        self.pos = np.zeros(3 * V, np.float32)
        self.out = np.zeros(3 * T + 3, np.uint32) if vp is not None else None
        self.passed = np.zeros(n, np.uint8) if vp is not None else None
        self.n_out = 0
        self.run(min(n, 2000))
        t0 = time.perf_counter()
        self.run(min(n, 2000))
        probe = time.perf_counter() - t0
        self.count = int(min(n, max(2000, 2000 * budget_s / max(probe, 1e-6))))
        # input (non-degenerate) triangles of the sample, counted outside any timing
        O.decode_into(ob, 0, self.count, self.loc, self.glob, self.pos)
        f = ob.fields()
        self.t_end = int(f["tri_base"][self.count - 1]) + int(f["Tp"][self.count - 1])
        self.v_end = int(f["vertex_base"][self.count - 1]) + int(f["V"][self.count - 1])
        t = self.loc[:3 * self.t_end].reshape(-1, 3).astype(np.int16)
        self.tris = int(((t[:, 0] != t[:, 1]) & (t[:, 1] != t[:, 2]) & (t[:, 0] != t[:, 2])).sum())
        self.run(self.count)  # first touch of the sample's output pages

    def run(self, count=None):
        count = self.count if count is None else count
        if self.vp is None:
            self.O.decode_into(self.ob, 0, count, self.loc, self.glob, self.pos)
        else:
            self.n_out = self.O.decode_cull_into(self.ob, self.vp, 0, count, self.a.get("cones"),
                                                 self.out, self.pos, self.passed)

    def timed(self) -> float:
        """One call over the sample; seconds."""
        t0 = time.perf_counter()
        self.run()
        return time.perf_counter() - t0

    def describe(self, dt: float) -> str:
        what = "decode + FP32 dequant" if self.vp is None else \
            "decode + frustum/normal-cone/back-face cull + compaction, one view"
        return (f"first {self.count} of {self.n} meshlets ({self.tris} input triangles) of the same "
                f"batch, sequential C {what} in one call, {dt:.2f} s, 1 thread")


def cpu_oracle_baseline(smp: OracleSample, all_cores: bool = True, budget_s: float = 5.0):
    """The oracle on one host core over its sample (and, with all_cores, the
    same calls on every host core)."""
    dt = smp.timed()
    res = {"value": smp.tris / dt / 1e9, "unit": "Gtps", "cores": 1, "kind": "oracle",
           "sample": smp.describe(dt)}
    if all_cores:
        res["all_cores"] = _oracle_all_cores(smp, budget_s)
    return res


def _oracle_all_cores(smp: OracleSample, budget_s):
    """The same oracle calls run concurrently on disjoint meshlet ranges of
    the sample, one range and one thread per host core (the C calls release
    the GIL); passes repeat until about budget_s.  Writes into its own
    arrays, so the sample's outputs stay as the timed call left them."""
    from concurrent.futures import ThreadPoolExecutor
    O, ob, a, vp, count, tris = smp.O, smp.ob, smp.a, smp.vp, smp.count, smp.tris
    threads = os.cpu_count() or 1
    bounds = np.linspace(0, count, threads + 1).astype(np.int64)
    T, V = ob.total_tris, ob.total_verts
    tp = ob.fields()["Tp"].astype(np.int64)
    pos = np.zeros(3 * V, np.float32)
    if vp is None:
        loc, glob = np.zeros(3 * T, np.uint8), np.zeros(3 * T, np.uint32)

        def part(i):
            if bounds[i + 1] > bounds[i]:
                O.decode_into(ob, int(bounds[i]), int(bounds[i + 1] - bounds[i]), loc, glob, pos)
    else:
        outs = [np.zeros(3 * int(tp[bounds[i]:bounds[i + 1]].sum()) + 3, np.uint32)
                for i in range(threads)]

        def part(i):
            if bounds[i + 1] > bounds[i]:
                O.decode_cull_into(ob, vp, int(bounds[i]), int(bounds[i + 1] - bounds[i]),
                                   a.get("cones"), outs[i], pos)
    with ThreadPoolExecutor(threads) as ex:
        list(ex.map(part, range(threads)))  # pages in the outputs
        reps, t0 = 0, time.perf_counter()
        while True:
            list(ex.map(part, range(threads)))
            reps += 1
            el = time.perf_counter() - t0
            if el >= budget_s or reps >= 200:
                break
    return {"value": tris * reps / el / 1e9, "unit": "Gtps", "cores": threads,
            "sample": f"the same {count} meshlets in {threads} equal ranges, one oracle call per "
                      f"range on {threads} threads, {reps} passes in {el:.2f} s"}


def _sorted_rows(t: np.ndarray) -> np.ndarray:
    t = t.reshape(-1, 3)
    key = (t[:, 0].astype(np.uint64) << np.uint64(32)) | t[:, 1].astype(np.uint64)
    return t[np.lexsort((t[:, 2], key))]


def parity_decode(smp: OracleSample, host: dict) -> dict:
    """The last timed step's decoded arrays against the oracle's decode of the
    sample's meshlets (indices exact, positions 0 ulp); counts the meshlets
    with any differing triangle or vertex."""
    f = smp.ob.fields()
    c, te, ve = smp.count, smp.t_end, smp.v_end
    tb = f["tri_base"][:c].astype(np.int64)
    vb = f["vertex_base"][:c].astype(np.int64)
    assert (np.diff(tb) >= 0).all() and (np.diff(vb) >= 0).all(), "bases not in blob order"
    bad_t = (host["local"][:3 * te].reshape(-1, 3) != smp.loc[:3 * te].reshape(-1, 3)).any(1)
    if host.get("global") is not None:
        g = host["global"][:3 * te].view(np.uint32).reshape(-1, 3)
        bad_t |= (g != smp.glob[:3 * te].reshape(-1, 3)).any(1)
    p = host["pos"][:3 * ve].view(np.uint32).reshape(-1, 3)
    bad_v = (p != smp.pos[:3 * ve].view(np.uint32).reshape(-1, 3)).any(1)
    bad = np.zeros(c, bool)
    bad[np.searchsorted(tb, np.nonzero(bad_t)[0], side="right") - 1] = True
    bad[np.searchsorted(vb, np.nonzero(bad_v)[0], side="right") - 1] = True
    return {"checked_meshlets": c, "of_meshlets": smp.n, "mismatches": int(bad.sum()),
            "compared": "u8 local + " + ("u32 global + " if host.get("global") is not None else "")
                        + "FP32 position bits of the last timed step vs the oracle's decode"}


def parity_cull(smp: OracleSample, host: dict, view: int) -> dict:
    """One view's survivors of the last timed step against the oracle's
    decode + cull of that view over the sample's meshlets (as multisets: the
    kernel's order across warps is unspecified), plus the positions of the
    sample's meshlets that pass the meshlet tests (0 ulp)."""
    f = smp.ob.fields()
    vb = f["vertex_base"].astype(np.int64)
    assert (np.diff(vb) >= 0).all(), "vertex bases not in blob order"
    got = host["tri"].reshape(-1, 3)
    got = got[got[:, 0] < smp.v_end]  # survivors of the sample's meshlets
    ref = smp.out[:3 * smp.n_out].reshape(-1, 3)
    tri_bad = 0 if got.shape == ref.shape and np.array_equal(_sorted_rows(got), _sorted_rows(ref)) \
        else max(1, abs(got.shape[0] - ref.shape[0]))
    vm = np.repeat(smp.passed[:smp.count].astype(bool), f["V"][:smp.count].astype(np.int64))
    p = host["pos"][:3 * smp.v_end].view(np.uint32).reshape(-1, 3)[vm]
    pos_bad = int((p != smp.pos[:3 * smp.v_end].view(np.uint32).reshape(-1, 3)[vm]).any(1).sum())
    return {"checked_meshlets": smp.count, "of_meshlets": smp.n, "mismatches": tri_bad + pos_bad,
            "survivors_compared": int(ref.shape[0]), "view": view,
            "compared": "surviving global index triples (multiset) and FP32 position bits of the "
                        "meshlets that pass, last timed step vs the oracle's decode + cull"}


# ------------------------------------------------------------- the GPU arm
def _timed_steps(step, stream, flush, warmup, steps, ws, local, clocks=True):
    """W untimed steps, then K steps each bracketed by CUDA events on
    `stream`, with an L2 flush (on the same stream) after every step;
    barrier + synchronize on both sides.  Returns (ms per step array,
    library launches in the timed region, clock summary)."""
    import torch
    from paper_2404_06359_gb300 import codec as mc
    for _ in range(warmup):
        step()
        flush.zero_()
    torch.cuda.synchronize()
    _barrier(ws)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    n0 = mc.mc_launch_count()
    clk = ClockSampler(local) if clocks else None
    if clk:
        clk.__enter__()
    try:
        for e0, e1 in evs:
            e0.record(stream)
            step()
            e1.record(stream)
            flush.zero_()
        torch.cuda.synchronize()
    finally:
        if clk:
            clk.__exit__(None, None, None)
    launches = mc.mc_launch_count() - n0
    _barrier(ws)
    torch.cuda.synchronize()
    times = np.array([e0.elapsed_time(e1) for e0, e1 in evs])  # ms
    return times, launches, clk.summary() if clk else None


def _parse_tuning(mc, text: str):
    """--tuning warps,ctas_per_sm,meshlets_per_grab[,lanes_per_meshlet]."""
    v = [int(x) for x in text.split(",")]
    return mc.mc_tuning(v[0], v[1], v[2], 0, 0, v[3] if len(v) > 3 else 32)


def _roofline(bytes_per_launch, per_launch_s, traffic, extra=None):
    peak, peak_kind = _peaks()
    ach = bytes_per_launch / per_launch_s / 1e9
    r = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
         "frac": round(ach / peak, 4), "traffic": traffic,
         "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS hbm_gbs)",
         "algorithmic_bytes_per_launch": int(bytes_per_launch),
         "frac_of_nominal": round(ach / NOMINAL_HBM_GBS, 4)}
    if extra:
        r.update(extra)
    return r


def measure_decode(args, cfg, blob, ws, local, stream, flush, main=True):
    """Times the decode of `blob` (cfg 1: plain one-launch decoder; else the
    persistent batched kernel from a CUDA graph, autotuned); returns
    (record, host copies of the last timed step's outputs)."""
    import torch
    from paper_2404_06359_gb300 import codec as mc
    from paper_2404_06359_gb300 import workloads as W
    attrs = args.attrs and main
    stats = blob.stats()
    arrays = blob.arrays()
    input_tris = stats["input_tris"]
    db = mc.DeviceBatch(blob, "cuda", attrs=attrs)
    want_global = cfg != 1
    out = db.outputs(True, want_global)
    if attrs:  # full 8-float vertices instead of positions
        out["vertex"] = torch.empty(8 * stats["total_verts"], dtype=torch.float32, device="cuda")
    scratch = mc.new_scratch()
    nbytes = W.algorithmic_bytes(stats, arrays["desc"], True, want_global, vertices=attrs)
    rec = {}
    with torch.cuda.stream(stream):
        if cfg == 1:
            graph, tune = None, {"warps_per_cta": 4}
        else:
            if args.tuning:
                tune = _parse_tuning(mc, args.tuning)
            else:
                tune, _ = mc.mc_autotune(db, out["local"], out["global"], out["pos"], out["status"],
                                         scratch, stream)
            graph = None if attrs else mc.mc_graph_capture_batch(
                db, out["local"], out["global"], out["pos"], out["status"], scratch, tune, stream)
            rec["tuning"] = {"warps_per_cta": tune.warps_per_cta, "ctas_per_sm": tune.ctas_per_sm,
                             "meshlets_per_grab": tune.meshlets_per_grab,
                             "lanes_per_meshlet": tune.lanes_per_meshlet or 32}

        def step():
            if graph is not None:
                graph.launch(stream)
            elif attrs:
                mc.mc_decode_batch_vertices(db, out["local"], out["global"], out["vertex"],
                                            out["status"], scratch, tune, stream)
            else:
                mc.mc_decode_plain(db, 0, stats["n_meshlets"], out["local"],
                                   out["global"] if want_global else None, out["pos"], out["status"],
                                   tune, stream)

        times, launches, clocks = _timed_steps(step, stream, flush, args.warmup, args.steps, ws, local,
                                               clocks=main or not args.no_clocks)
        # the last timed step's outputs, for the parity check against the oracle
        host = {"local": out["local"].cpu().numpy(),
                "global": out["global"].cpu().numpy() if want_global else None,
                "pos": (out["vertex"].view(-1, 8)[:, :3].reshape(-1) if attrs else out["pos"]).cpu().numpy()}
        status = int(out["status"].item())
        assert status == 0, f"device status {status:#x}"

        # plain one-launch-per-mesh decoder on the same batch (the baseline)
        plain = None
        if cfg != 1 and args.plain_steps > 0 and not attrs:
            pt = []
            for i in range(args.plain_steps + 2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for msh in db.meshes:
                    mc.mc_decode_plain(db, msh["first_meshlet"], msh["n_meshlets"], out["local"],
                                       out["global"], out["pos"], out["status"], None, stream)
                e1.record(stream)
                flush.zero_()
                torch.cuda.synchronize()
                if i >= 2:
                    pt.append(e0.elapsed_time(e1))
            pms = float(np.mean(pt))
            plain = {"value": input_tris / (pms * 1e-3) / 1e9, "unit": "Gtps", "ms_per_step": pms,
                     "launches_per_step": len(db.meshes),
                     "meshlets_per_launch": round(stats["n_meshlets"] / max(1, len(db.meshes)), 1),
                     "note": "one launch per mesh over the same resident batch, warp per meshlet; "
                             "the batched kernel's advantage over it grows with the number of "
                             "meshes (launch count): with one mesh it is one launch as well"}

        # end to end through the C ABI with host buffers (pinned), copies timed
        e2e = None
        if main and args.e2e_steps > 0 and not attrs:
            T, V = stats["total_tris"], stats["total_verts"]
            d_desc = torch.empty(32 * stats["n_meshlets"], dtype=torch.uint8, device="cuda")
            d_pay = torch.empty(stats["payload_bytes"], dtype=torch.uint8, device="cuda")
            d_grid = torch.empty(32 * stats["n_grids"], dtype=torch.uint8, device="cuda")
            h_loc = torch.empty(3 * T, dtype=torch.uint8).pin_memory()
            h_glob = torch.empty(3 * T, dtype=torch.int32).pin_memory() if want_global else None
            h_pos = torch.empty(3 * V, dtype=torch.float32).pin_memory()
            h_in = mc.pinned_inputs(blob)  # the step's inputs, in pinned host memory
            et = []
            for i in range(args.e2e_steps + 2):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                mc.mc_decode_batch_host(blob, d_desc, d_pay, d_grid, out["local"],
                                        out["global"] if want_global else None, out["pos"],
                                        out["status"], scratch, h_loc, h_glob, h_pos, tune, stream,
                                        host_inputs=h_in)
                e1.record(stream)
                torch.cuda.synchronize()
                if i >= 2:
                    et.append(e0.elapsed_time(e1))
            ems = _allreduce_max(float(np.mean(et)), ws)
            e2e = {"value": ws * input_tris / (ems * 1e-3) / 1e9, "unit": "Gtps", "ms_per_step": ems,
                   "h2d_bytes_per_step": int(32 * stats["n_meshlets"] + stats["payload_bytes"]
                                             + 32 * stats["n_grids"]),
                   "d2h_bytes_per_step": int(3 * T + (12 * T if want_global else 0) + 12 * V)}

    total_ms = _allreduce_max(float(times.sum()), ws)
    per_launch_s = times.mean() * 1e-3
    tr = NCU_TRAFFIC.get(cfg)
    traffic = None
    if (main and tr and tr[0] == _kernel_hash(cfg) and args.codec == "reuse" and not attrs):
        traffic = int(tr[1] * stats["total_tris"])
    rec.update({
        "value": round(aggregate_gtps(ws, input_tris, args.steps, total_ms), 3),
        "ms_per_step": round(total_ms / args.steps, 5),
        "decoded_slot_gtps": round(aggregate_gtps(ws, stats["total_tris"], args.steps, total_ms), 3),
        "latency_ms": {"min": round(float(times.min()), 5),
                       "p50": round(float(np.percentile(times, 50)), 5),
                       "p99": round(float(np.percentile(times, 99)), 5)},
        "roofline": _roofline(nbytes["total"], per_launch_s, traffic,
                              {"bytes_per_input_triangle": round(nbytes["total"] / input_tris, 2),
                               "block_padding_bytes": nbytes["padding"]}),
        "gpu_launches": int(launches), "clocks": clocks, "plain": plain, "e2e": e2e,
    })
    return rec, host


def _config_dict(cfg, stats, codec="reuse", attrs=False, cfg4_tris=50_000_000, ws=1, strip_search=0):
    return {"workload": WORKLOADS[cfg] + (" [plain GTS connectivity]" if codec == "gts" else "")
            + (f" [fewest-strips search, {strip_search} nodes per meshlet]" if strip_search else "")
            + (" [8-channel vertices: position, normal, texture coordinate; 32 B out]" if attrs else "")
            + (f" [reduced to >= {cfg4_tris} triangles]" if cfg == 4 and cfg4_tris != 50_000_000 else ""),
            "connectivity_bits_per_triangle": round(stats["conn_bits"] / stats["input_tris"], 3),
            "input_triangles": int(stats["input_tris"]),
            "decoded_triangle_slots": int(stats["total_tris"]), "vertices": int(stats["total_verts"]),
            "meshlets": int(stats["n_meshlets"]), "l2": L2_NOTE,
            "parallelism": f"{ws} independent replica(s), no collective"}


def measure_cull(args, blob, vps, ws, local, stream, flush):
    """cfg4: one step = the fused decode + cull of the batch under all views
    (one CUDA graph of ceil(64 / v) multi-view launches, v = --cull-views);
    returns (record, host copies of the last timed step's outputs)."""
    import torch
    from paper_2404_06359_gb300 import codec as mc
    from paper_2404_06359_gb300 import workloads as W
    stats = blob.stats()
    arrays = blob.arrays()
    input_tris = stats["input_tris"]
    db = mc.DeviceBatch(blob, "cuda", cones=True)  # normal-cone meshlet test on
    out = db.outputs(False, False)
    scratch = mc.new_scratch()
    T = stats["total_tris"]
    cv = args.cull_views
    stride = 3 * T + 3
    rec = {}
    with torch.cuda.stream(stream):
        tri = torch.empty(cv * stride, dtype=torch.int32, device="cuda")
        d_vps = torch.from_numpy(np.ascontiguousarray(vps, np.float32)).cuda()
        counts = torch.zeros(len(vps), dtype=torch.int32, device="cuda")
        tune = None
        if args.tuning:
            tune = _parse_tuning(mc, args.tuning)

        def capture_cull(batch):
            if cv == 1:
                return mc.mc_graph_capture_cull(batch, d_vps, len(vps), tri, counts, out["pos"],
                                                out["status"], scratch, tune, stream)
            return mc.mc_graph_capture_cull_views(batch, d_vps, len(vps), tri, stride, counts,
                                                  out["pos"], out["status"], scratch, tune, stream)
        graph = capture_cull(db)
        launches_per_step = (len(vps) + cv - 1) // cv
        times, launches, clocks = _timed_steps(lambda: graph.launch(stream), stream, flush,
                                               args.warmup, args.steps, ws, local)
        # the last timed step's outputs: region 0 holds the first view of its last launch
        view0 = len(vps) - cv
        counts_np = counts.cpu().numpy().astype(np.int64)
        host = {"tri": tri[: 3 * int(counts_np[view0])].cpu().numpy().view(np.uint32),
                "pos": out["pos"].cpu().numpy(), "view": view0}
        assert int(out["status"].item()) == 0, f"device status {int(out['status'].item()):#x}"
        bytes_per_launch = W.cull_bytes(stats, arrays, vps, counts_np, cones=True, views_per_launch=cv)

        def time_graph(g, n):
            ts = []
            for i in range(3 + n):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g()
                e1.record(stream)
                flush.zero_()
                if i >= 3:
                    ts.append((e0, e1))
            torch.cuda.synchronize()
            return float(np.mean([a_.elapsed_time(b_) for a_, b_ in ts]))

        n_other = max(3, args.steps // 10)
        if args.no_cull_extras:
            return _cull_record(rec, args, vps, stats, arrays, times, launches, clocks, counts_np,
                                bytes_per_launch, launches_per_step, ws), host
        if cv > 1:
            # the same step with one single-view launch per view
            g_1 = mc.mc_graph_capture_cull(db, d_vps, len(vps), tri, counts, out["pos"],
                                           out["status"], scratch, tune, stream)
            ms1 = time_graph(lambda: g_1.launch(stream), n_other)
            assert int(out["status"].item()) == 0
            assert np.array_equal(counts.cpu().numpy().astype(np.int64), counts_np)
            b1 = W.cull_bytes(stats, arrays, vps, counts_np, cones=True)
            a1 = b1 / (ms1 * 1e-3 / len(vps)) / 1e9
            rec["cull_one_view_per_launch"] = {
                "value": round(input_tris * len(vps) / (ms1 * 1e-3) / 1e9, 3), "unit": "Gtps",
                "ms_per_step": round(ms1, 5), "launches_per_step": len(vps),
                "algorithmic_bytes_per_launch": b1, "achieved_GBps": round(a1, 1),
                "frac": round(a1 / _peaks()[0], 4)}
        # the same step without the normal-cone test (frustum + per-triangle only)
        db_nc = mc.DeviceBatch(blob, "cuda")
        g_nc = capture_cull(db_nc)
        nc_ms = time_graph(lambda: g_nc.launch(stream), n_other)
        assert int(out["status"].item()) == 0
        counts_nc = counts.cpu().numpy().astype(np.int64)
        # the same step with survivors in meshlet order (decoupled look-back)
        d_order = torch.empty(int(mc.lib().mc_cull_order_bytes(mc.C.byref(db.c))), dtype=torch.uint8,
                              device="cuda")

        def ordered():
            for v in range(len(vps)):
                mc.mc_decode_cull_ordered(db, d_vps[v], tri, counts[v:v + 1], out["pos"],
                                          out["status"], scratch, d_order, tune, stream)
        or_ms = time_graph(ordered, n_other)
        assert int(out["status"].item()) == 0
        assert np.array_equal(counts.cpu().numpy().astype(np.int64), counts_np)
    rec["cull_ordered"] = {
        "value": round(input_tris * len(vps) / (or_ms * 1e-3) / 1e9, 3), "unit": "Gtps",
        "ms_per_step": round(or_ms, 5), "launches_per_step": len(vps),
        "note": "survivors in meshlet order; launched one view at a time (no graph)"}
    rec["cull_without_cones"] = {
        "value": round(input_tris * len(vps) / (nc_ms * 1e-3) / 1e9, 3), "unit": "Gtps",
        "ms_per_step": round(nc_ms, 5),
        "kept_fraction_mean": float(counts_nc.mean() / input_tris),
        "algorithmic_bytes_per_launch": W.cull_bytes(stats, arrays, vps, counts_nc, views_per_launch=cv)}
    return _cull_record(rec, args, vps, stats, arrays, times, launches, clocks, counts_np,
                        bytes_per_launch, launches_per_step, ws), host


def _cull_record(rec, args, vps, stats, arrays, times, launches, clocks, counts_np,
                 bytes_per_launch, launches_per_step, ws):
    input_tris, T, cv = stats["input_tris"], stats["total_tris"], args.cull_views
    rec["cull"] = {"kept_fraction_mean": float(counts_np.mean() / input_tris), "views": len(vps),
                   "views_per_launch": cv, "triangles_per_step": input_tris * len(vps)}
    total_ms = _allreduce_max(float(times.sum()), ws)
    per_launch_s = (times.mean() * 1e-3) / launches_per_step
    tr = NCU_TRAFFIC.get(4)
    traffic = int(tr[1] * T) if tr and tr[0] == _kernel_hash(4) and cv == 8 else None
    rec.update({
        "value": round(aggregate_gtps(ws, input_tris * len(vps), args.steps, total_ms), 3),
        "ms_per_step": round(total_ms / args.steps, 5),
        "decoded_slot_gtps": round(aggregate_gtps(ws, T * len(vps), args.steps, total_ms), 3),
        "latency_ms": {"min": round(float(times.min()), 5),
                       "p50": round(float(np.percentile(times, 50)), 5),
                       "p99": round(float(np.percentile(times, 99)), 5)},
        "roofline": _roofline(bytes_per_launch, per_launch_s, traffic,
                              {"bytes_per_input_triangle": round(bytes_per_launch / input_tris, 2)}),
        "gpu_launches": int(launches), "clocks": clocks, "plain": None, "e2e": None,
    })
    return rec


def run_cfg3_record(args, ws, rank, local, stream, flush):
    """The cfg3 sub-record of the default run: the largest decode workload,
    timed as the main line is, with its own oracle leg (one core, the whole
    batch) and parity check."""
    import torch
    t_build = time.time()
    blob, _, _ = build_workload(3, rank)
    t_build = time.time() - t_build
    stats = blob.stats()
    rec, host = measure_decode(args, 3, blob, ws, local, stream, flush, main=False)
    rec["config"] = _config_dict(3, stats, ws=ws)
    rec["build_s"] = round(t_build, 1)
    if rank == 0 and not args.no_cpu_baseline:
        smp = OracleSample(blob.arrays(), args.cfg3_cpu_seconds)
        rec["cpu_baseline"] = cpu_oracle_baseline(smp, all_cores=False)
        rec["parity"] = parity_decode(smp, host)
    del host
    torch.cuda.empty_cache()
    return rec


# ------------------------------------------------------------- reference arm
def oracle_workload(cfg: int, rank: int, cfg4_tris: int = 50_000_000):
    """The benchmark workloads encoded by the oracle (test infrastructure,
    byte-identical to the library's encoder): (blob arrays, stats, views)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle as O
    from paper_2404_06359_gb300 import meshgen as G
    seed = G.SEED_BASE + cfg
    vps = None
    if cfg == 1:
        mesh = G.grid_mesh(64, 0.25, seed)
        ob = O.encode_mesh(mesh, (64, 126), 16, 0)
        input_tris = mesh.n_tris
    elif cfg in (2, 4):
        meshes = G.surface_batch(256, 10_000, 200_000, G.SEED_BASE + 2 + 1000 * rank,
                                 min_total_tris=cfg4_tris if cfg == 4 else 0)
        with ThreadPoolExecutor(os.cpu_count() or 4) as ex:
            parts = list(ex.map(lambda im: O.encode_mesh(im[1], (64, 126), 16, 0, mesh_id=im[0]),
                                enumerate(meshes)))
        ob = O.concat(parts)
        input_tris = sum(m.n_tris for m in meshes)
        if cfg == 4:
            vps = G.scene_views(meshes, 64, G.SEED_BASE + 4 + rank)
    elif cfg == 3:
        s3 = seed + 1000 * rank
        mesh = G.height_field_disc(50_000_000, s3)
        ob = O.encode_mesh(mesh, np.array(G.SECTOR_LIMITS).reshape(-1),
                           lambda n: G.meshlet_bits(n, s3 + 1), 1,
                           perm=lambda n: G.meshlet_permutation(n, s3 + 2))
        input_tris = mesh.n_tris
    else:
        raise SystemExit(f"the reference arm covers configs 1-4, not {cfg}")
    stats = {"conn_bits": ob.stats["conn_bits"], "input_tris": input_tris,
             "total_tris": ob.total_tris, "total_verts": ob.total_verts, "n_meshlets": ob.n_meshlets}
    arrays = {"desc": ob.desc, "payload": ob.payload, "grids": ob.grids, "cones": ob.cones}
    return arrays, stats, vps


def run_reference(args, ws, rank):
    """The CPU oracle as the reference arm: the same workload, encoded by the
    oracle itself, decoded by the oracle's sequential C decoder (cfg4: decode +
    cull of one view), a bounded sample per step."""
    if rank != 0:
        return
    arrays, stats, vps = oracle_workload(args.config, 0, args.cfg4_tris)
    vp = vps[len(vps) - args.cull_views] if args.config == 4 else None
    # one oracle call per step over a fixed sample, sized so that the whole run
    # takes about ref_seconds of oracle time (at least 2000 meshlets a call)
    smp = OracleSample(arrays, max(0.01, args.ref_seconds / (args.warmup + args.steps)), vp)
    per, dts = [], []
    for i in range(args.warmup + args.steps):
        dt = smp.timed()
        if i >= args.warmup:
            per.append(smp.tris / dt / 1e9)
            dts.append(dt)
    v = float(np.mean(per))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gtps", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u32/f32", "data": "synthetic",
           "config": _config_dict(args.config, stats, cfg4_tris=args.cfg4_tris, ws=max(1, args.gpus)),
           "cpu_baseline": {"value": v, "unit": "Gtps", "cores": 1, "kind": "oracle",
                            "sample": smp.describe(float(np.mean(dts))) + " (mean per step)"},
           "e2e": {"value": v, "unit": "Gtps", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_serving(args, ws, rank):
    """cfg5: the continuous-batching loop for --serve-seconds of arrivals."""
    from paper_2404_06359_gb300 import meshgen as G
    from paper_2404_06359_gb300 import serving as S
    t_build = time.time()
    pool, _ = S.build_pool(args.pool_meshes, seed=G.SEED_BASE + 5 + 1000 * rank)
    t_build = time.time() - t_build
    srv = S.Server(pool, budget_bytes=8 << 30, n_streams=4)
    # warm-up: a short burst (not reported)
    wa, wm = G.poisson_arrivals(args.rate, 0.2, len(srv.meshes), G.SEED_BASE + 7)
    srv.run(wa, wm)
    srv.launches = 0
    arr, mid = G.poisson_arrivals(args.rate, args.serve_seconds, len(srv.meshes), G.SEED_BASE + 6)
    n0 = mc_launches()
    with ClockSampler(int(os.environ.get("LOCAL_RANK", "0"))) as clk:
        done, st = srv.run(arr, mid)
    launches = mc_launches() - n0
    g = _allreduce_max(st["wall_s"], ws)
    value = aggregate_gtps(ws, st["input_triangles"], 1, g * 1e3)
    res = {"metric": METRIC, "value": round(value, 4), "unit": "Gtps", "n_gpus": ws, "steps": 1,
           "warmup": args.warmup, "ms_per_step": round(g * 1e3, 2), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "u32/f32", "data": "synthetic",
           "config": {"workload": WORKLOADS[5], "pool_meshes": args.pool_meshes,
                      "rate_per_s": args.rate, "seconds": args.serve_seconds},
           "latency_ms": {"p50": round(st["p50_ms"], 3), "p99": round(st["p99_ms"], 3)},
           "serving": st, "gpu_launches": int(launches), "clocks": clk.summary(),
           "roofline": None, "build_s": round(t_build, 1)}
    if rank == 0:
        print(json.dumps(res), flush=True)


def mc_launches():
    from paper_2404_06359_gb300 import codec as mc
    return mc.mc_launch_count()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--config", type=int, default=2)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-seconds", type=float, default=20.0)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--cfg3-cpu-seconds", type=float, default=3.0,
                    help="oracle budget of the cfg3 record's one-core leg (covers the whole batch)")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip the oracle legs (and with them the parity check)")
    ap.add_argument("--no-cfg3", action="store_true", help="config 2 without the cfg3 record")
    ap.add_argument("--no-clocks", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--no-cull-extras", action="store_true",
                    help="config 4 without the one-view, no-cone and ordered variants")
    ap.add_argument("--plain-steps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--tuning", default="",
                    help="warps,ctas_per_sm,meshlets_per_grab[,lanes_per_meshlet] (skips the autotuner)")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--pool-meshes", type=int, default=512)
    ap.add_argument("--attrs", action="store_true",
                    help="config 2 with 8-channel vertices (position, normal, texture coordinate; "
                         "16-bit attributes) decoded by mc_decode_batch_vertices")
    ap.add_argument("--cull-views", type=int, default=8, choices=range(1, 9), metavar="1..8",
                    help="config 4: views per fused-cull launch (1 = one launch per view)")
    ap.add_argument("--cfg4-tris", type=int, default=50_000_000,
                    help="config 4 batch size (smaller only for profiler captures)")
    ap.add_argument("--codec", choices=("reuse", "gts"), default="reuse",
                    help="connectivity encoding of configs 2/3: GTS-Reuse (default) or plain GTS "
                         "(one stored 8-bit entry per triangle)")
    ap.add_argument("--strip-search", type=int, default=0, metavar="NODES",
                    help="config 2 encoded with the fewest-strips search (node budget per meshlet)")
    args = ap.parse_args()
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch

    assert args.warmup >= 3, "at least 3 warm-up steps"
    torch.cuda.set_device(local)
    if args.config == 5:
        run_serving(args, ws, rank)
        return
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if args.codec == "gts" and args.config not in (2, 3):
        raise SystemExit("--codec gts applies to configs 2 and 3")
    if args.attrs and args.config != 2:
        raise SystemExit("--attrs applies to config 2")
    t_build = time.time()
    blob, meshes, vps = build_workload(args.config, rank, args.codec, args.attrs, args.cfg4_tris,
                                       args.strip_search)
    t_build = time.time() - t_build
    stats = blob.stats()
    stream = torch.cuda.Stream()
    l2 = int(getattr(torch.cuda.get_device_properties(local), "L2_cache_size", 0) or 129 << 20)
    flush_mb = max(256, (2 * l2 >> 20) + 16)  # a write of at least twice the L2 between steps
    flush = torch.empty(flush_mb * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    cull = args.config == 4
    if cull:
        rec, host = measure_cull(args, blob, vps, ws, local, stream, flush)
    else:
        rec, host = measure_decode(args, args.config, blob, ws, local, stream, flush, main=True)
    res = {"metric": METRIC, "value": rec.pop("value"), "unit": "Gtps", "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec.pop("ms_per_step"),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/f32",
           "data": "synthetic",
           "config": _config_dict(args.config, stats, args.codec, args.attrs, args.cfg4_tris, ws,
                                  args.strip_search),
           "l2_flush": {"bytes_written": flush_mb << 20, "l2_bytes": l2}}
    res.update(rec)
    res["build_s"] = round(t_build, 1)
    parity_ok = True
    if rank == 0 and not args.no_cpu_baseline:
        vp = vps[host["view"]] if cull else None
        smp = OracleSample(blob.arrays(), args.cpu_seconds, vp)
        res["cpu_baseline"] = cpu_oracle_baseline(smp)
        res["parity"] = parity_cull(smp, host, host["view"]) if cull else parity_decode(smp, host)
        parity_ok = res["parity"]["mismatches"] == 0
        del smp
    del host
    if (args.config == 2 and not args.no_cfg3 and args.codec == "reuse" and not args.attrs
            and not args.strip_search):
        res["cfg3"] = run_cfg3_record(args, ws, rank, local, stream, flush)
        if "parity" in res["cfg3"]:
            parity_ok = parity_ok and res["cfg3"]["parity"]["mismatches"] == 0
    if rank == 0:
        print(json.dumps(res), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    if not parity_ok:
        sys.exit(3)


if __name__ == "__main__":
    main()
