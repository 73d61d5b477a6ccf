"""Benchmark: batched GTS-Reuse meshlet decode on GB300.

Default workload (cfg2): 256 seeded UV-spheres/tori, ~16.2 M triangles,
meshlets 64/126, 16-bit positions, 8-bit reuse indices, decoded to u8 local +
u32 global indices + FP32 positions by one persistent launch replayed from a
CUDA graph.  One step = one decode of the whole batch (inputs resident in
HBM); L2 is flushed (a write of at least twice its size) between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config 1|2|3|4]
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


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# DRAM bytes (read + write) of one launch of the dominant kernel from an ncu
# capture (profiles/decode_batch_cfg2.md for cfg2: one decode_batch launch;
# profiles/decode_cull_views_cfg4.md for cfg4: one 8-view decode_cull_views
# launch, captured on the 20 M-triangle reduction of the batch), per decoded
# triangle slot and keyed by the kernel-source hash it was taken on; reported
# only while the sources match.  Both captures predate the meshletizer's
# shared-edge pick (same meshes, 7 % more meshlets), so the figure is scaled
# by decoded triangle slots from that partition of the same meshes.
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e nominal, for the second fraction beside the measured peak

NCU_TRAFFIC = {  # config -> (device-code hash, DRAM bytes per decoded triangle slot)
    2: ("846363d9384b0863", (86.488064e6 + 328.722688e6) / 17124622),
    4: ("61f54bf40e08143c", (114.16832e6 + 1030.18e6) / 21162408),
}


def _kernel_hash(config: int):
    """Hash of the device code the config's dominant kernel is built from: the
    shared device headers and its kernel file (kernels.cu for the decoders,
    cull_views.cu with the cull helpers for the multi-view cull), each up to
    its host launchers."""
    import hashlib
    h = hashlib.sha256()
    files = ["cull_views.cu", "cull_common.cuh"] if config == 4 else ["kernels.cu"]
    for p in ["paper_2404_06359_gb300/csrc/device/" + f
              for f in files + ["decode_warp.cuh", "grab_loop.cuh"]]:
        with open(os.path.join(ROOT, p), "rb") as f:
            b = f.read()
        h.update(b.split(b"// ------------------------------------------------------------- launchers")[0])
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
                   cfg4_tris: int = 50_000_000):
    from paper_2404_06359_gb300 import workloads as W
    if cfg == 1:
        blob, meshes = W.cfg1()
        return blob, meshes, None
    if cfg == 2:
        blob, meshes = W.cfg2(rank, plain_gts=codec == "gts", attrs=attrs)
        return blob, meshes, None
    if cfg == 3:
        blob, meshes = W.cfg3(rank, plain_gts=codec == "gts")
        return blob, meshes, None
    if cfg == 4:
        return W.cfg4(rank, min_tris=cfg4_tris)
    raise SystemExit(f"unknown config {cfg}")


class OracleSample:
    """The oracle's sequential C decode (or, given a view-projection matrix,
    its fused decode + normal-cone/frustum/back-face cull for that view) over
    the first `count` meshlets of the batch, into output arrays allocated
    once (so a timed call pays for no allocation); `count` is sized from a
    probe so that one call takes about budget_s."""

    def __init__(self, blob, budget_s: float, vp=None):
        import oracle as O
        self.O, self.vp = O, vp
        self.a = a = blob.arrays()
        self.ob = ob = O.Blob(a["desc"], a["payload"], a["grids"])
        self.n = n = ob.n_meshlets
        T, V = ob.total_tris, ob.total_verts
        self.loc, self.glob = np.zeros(3 * T, np.uint8), np.zeros(3 * T, np.uint32)
        self.pos = np.zeros(3 * V, np.float32)
        self.out = np.zeros(3 * T + 3, np.uint32) if vp is not None else None
        self.run(min(n, 2000))
        t0 = time.perf_counter()
        self.run(min(n, 2000))
        probe = time.perf_counter() - t0
        self.count = int(min(n, max(2000, 2000 * budget_s / max(probe, 1e-6))))
        # input (non-degenerate) triangles of the sample, counted outside any timing
        O.decode_into(ob, 0, self.count, self.loc, self.glob, self.pos)
        f = ob.fields()
        end = int(f["tri_base"][self.count - 1]) + int(f["Tp"][self.count - 1])
        t = self.loc[:3 * end].reshape(-1, 3).astype(np.int16)
        self.tris = int(((t[:, 0] != t[:, 1]) & (t[:, 1] != t[:, 2]) & (t[:, 0] != t[:, 2])).sum())
        self.run(self.count)  # first touch of the sample's output pages

    def run(self, count=None):
        count = self.count if count is None else count
        if self.vp is None:
            self.O.decode_into(self.ob, 0, count, self.loc, self.glob, self.pos)
        else:
            self.O.decode_cull_into(self.ob, self.vp, 0, count, self.a["cones"], self.out, self.pos)

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


def cpu_oracle_baseline(blob, budget_s: float = 10.0, vp=None, all_cores: bool = True):
    """The oracle on one host core over a sample of about budget_s (and, with
    all_cores, the same calls on every host core)."""
    smp = OracleSample(blob, budget_s, vp)
    dt = smp.timed()
    res = {"value": smp.tris / dt / 1e9, "unit": "Gtps", "cores": 1, "kind": "oracle",
           "sample": smp.describe(dt)}
    if all_cores:
        res["all_cores"] = _oracle_all_cores(smp.O, smp.ob, smp.a, vp, smp.count, smp.tris,
                                             min(budget_s, 5.0))
    return res


def _oracle_all_cores(O, ob, a, vp, count, tris, budget_s):
    """The same oracle calls run concurrently on disjoint meshlet ranges of
    the sample, one range and one thread per host core (the C calls release
    the GIL); passes repeat until about budget_s."""
    from concurrent.futures import ThreadPoolExecutor
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
                                   a["cones"], outs[i], pos)
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


def run_reference(args, ws, rank):
    if rank != 0:
        return
    blob, meshes, vps = build_workload(args.config, 0)
    vp = vps[0] if args.config == 4 else None
    per = []
    # one oracle call per step over a fixed sample, sized so that the whole run
    # takes about ref_seconds of oracle time (at least 2000 meshlets a call)
    smp = OracleSample(blob, max(0.01, args.ref_seconds / (args.warmup + args.steps)), vp)
    dts = []
    for i in range(args.warmup + args.steps):
        dt = smp.timed()
        if i >= args.warmup:
            per.append(smp.tris / dt / 1e9)
            dts.append(dt)
    v = float(np.mean(per))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Gtps", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "u32/f32", "data": "synthetic",
           "config": {"workload": WORKLOADS[args.config]},
           "cpu_baseline": {"value": v, "unit": "Gtps", "cores": 1, "kind": "oracle",
                            "sample": smp.describe(float(np.mean(dts))) + " (mean per step)"},
           "e2e": {"value": v, "unit": "Gtps", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_serving(args, ws, rank):
    """cfg5: the continuous-batching loop for --serve-seconds of arrivals."""
    import torch
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
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--plain-steps", type=int, default=20)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--tuning", default="", help="warps,ctas_per_sm,meshlets_per_grab (skips the autotuner)")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--rate", type=float, default=2000.0)
    ap.add_argument("--pool-meshes", type=int, default=128)
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
    args = ap.parse_args()
    ws, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch
    from paper_2404_06359_gb300 import codec as mc
    from paper_2404_06359_gb300 import workloads as W

    assert args.warmup >= 3, "at least 3 warm-up steps"
    torch.cuda.set_device(local)
    if args.config == 5:
        run_serving(args, ws, rank)
        return
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    t_build = time.time()
    if args.codec == "gts" and args.config not in (2, 3):
        raise SystemExit("--codec gts applies to configs 2 and 3")
    if args.attrs and args.config != 2:
        raise SystemExit("--attrs applies to config 2")
    blob, meshes, vps = build_workload(args.config, rank, args.codec, args.attrs, args.cfg4_tris)
    t_build = time.time() - t_build
    stats = blob.stats()
    db = mc.DeviceBatch(blob, "cuda", cones=args.config == 4,  # cfg4: normal-cone meshlet test on
                        attrs=args.attrs)
    arrays = blob.arrays()
    input_tris = stats["input_tris"]
    stream = torch.cuda.Stream()
    l2 = int(getattr(torch.cuda.get_device_properties(local), "L2_cache_size", 0) or 129 << 20)
    flush_mb = max(256, (2 * l2 >> 20) + 16)  # a write of at least twice the L2 between steps
    flush = torch.empty(flush_mb * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    scratch = mc.new_scratch()
    cull = args.config == 4
    want_local = True
    want_global = args.config != 1
    out = db.outputs(want_local, want_global)
    if args.attrs:  # full 8-float vertices instead of positions
        out["vertex"] = torch.empty(8 * stats["total_verts"], dtype=torch.float32, device="cuda")
    nbytes = W.algorithmic_bytes(stats, arrays["desc"], want_local, want_global,
                                 vertices=args.attrs)
    extra = {}
    with torch.cuda.stream(stream):
        if cull:
            T, V = stats["total_tris"], stats["total_verts"]
            tri = torch.empty(3 * T + 3, dtype=torch.int32, device="cuda")
            d_vps = torch.from_numpy(np.ascontiguousarray(vps, np.float32)).cuda()
            counts = torch.zeros(len(vps), dtype=torch.int32, device="cuda")
            tune = None
            if args.tuning:
                w_, c_, g_ = (int(x) for x in args.tuning.split(","))
                tune = mc.mc_tuning(w_, c_, g_, 0)
            cv = args.cull_views
            stride = 3 * T + 3
            tri = torch.empty(cv * stride, dtype=torch.int32, device="cuda")

            def capture_cull(batch):
                if cv == 1:
                    return mc.mc_graph_capture_cull(batch, d_vps, len(vps), tri, counts, out["pos"],
                                                    out["status"], scratch, tune, stream)
                return mc.mc_graph_capture_cull_views(batch, d_vps, len(vps), tri, stride, counts,
                                                      out["pos"], out["status"], scratch, tune,
                                                      stream)
            graph = capture_cull(db)
            launches_per_step = (len(vps) + cv - 1) // cv
        elif args.config == 1:
            graph = None
            launches_per_step = 1
            tune = {"warps_per_cta": 4}
        else:
            if args.tuning:
                w_, c_, g_ = (int(x) for x in args.tuning.split(","))
                tune = mc.mc_tuning(w_, c_, g_, 0)
            else:
                tune, tune_ms = mc.mc_autotune(db, out["local"], out["global"], out["pos"],
                                               out["status"], scratch, stream)
            graph = None if args.attrs else mc.mc_graph_capture_batch(
                db, out["local"], out["global"], out["pos"], out["status"], scratch, tune, stream)
            launches_per_step = 1
            extra["tuning"] = {"warps_per_cta": tune.warps_per_cta, "ctas_per_sm": tune.ctas_per_sm,
                               "meshlets_per_grab": tune.meshlets_per_grab}

        def step():
            if graph is not None:
                graph.launch(stream)
            elif args.attrs:
                mc.mc_decode_batch_vertices(db, out["local"], out["global"], out["vertex"],
                                            out["status"], scratch, tune, stream)
            else:
                mc.mc_decode_plain(db, 0, stats["n_meshlets"], out["local"],
                                   out["global"] if want_global else None, out["pos"], out["status"],
                                   tune, stream)

        for _ in range(args.warmup):
            step()
            flush.zero_()
        torch.cuda.synchronize()
        _barrier(ws)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        n0 = mc.mc_launch_count()
        with ClockSampler(local) as clk:
            for e0, e1 in evs:
                e0.record(stream)
                step()
                e1.record(stream)
                flush.zero_()
            torch.cuda.synchronize()
        launches = mc.mc_launch_count() - n0
        _barrier(ws)
        torch.cuda.synchronize()
        times = np.array([e0.elapsed_time(e1) for e0, e1 in evs])  # ms
        total_ms = _allreduce_max(float(times.sum()), ws)
        status = int(out["status"].item())
        assert status == 0, f"device status {status:#x}"

        # plain one-launch-per-mesh decoder on the same batch (the baseline)
        plain = None
        if not cull and args.config != 1 and args.plain_steps > 0 and not args.attrs:
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
                     "launches_per_step": len(db.meshes)}

        # end to end through the C ABI with host buffers (pinned), copies timed
        e2e = None
        if not cull and args.e2e_steps > 0 and not args.attrs:
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

    ms_step = total_ms / args.steps
    views = len(vps) if cull else 1  # the cull step decodes the batch once per view
    value = aggregate_gtps(ws, input_tris * views, args.steps, total_ms)
    peak, peak_kind = _peaks()
    per_launch_s = (times.mean() * 1e-3) / launches_per_step
    bytes_per_launch = nbytes["total"] if not cull else None
    if cull:
        counts_np = counts.cpu().numpy().astype(np.int64)
        bytes_per_launch = W.cull_bytes(stats, arrays, vps, counts_np, cones=True,
                                        views_per_launch=cv)
        if cv > 1:
            # the same step with one single-view launch per view
            g_1 = mc.mc_graph_capture_cull(db, d_vps, len(vps), tri, counts, out["pos"],
                                           out["status"], scratch, tune, stream)
            with torch.cuda.stream(stream):
                t1 = []
                for i in range(3 + max(3, args.steps // 10)):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    g_1.launch(stream)
                    e1.record(stream)
                    flush.zero_()
                    if i >= 3:
                        t1.append((e0, e1))
                torch.cuda.synchronize()
            ms1 = float(np.mean([a_.elapsed_time(b_) for a_, b_ in t1]))
            assert int(out["status"].item()) == 0
            assert np.array_equal(counts.cpu().numpy().astype(np.int64), counts_np)
            b1 = W.cull_bytes(stats, arrays, vps, counts_np, cones=True)
            a1 = b1 / (ms1 * 1e-3 / len(vps)) / 1e9
            extra["cull_one_view_per_launch"] = {
                "value": round(input_tris * len(vps) / (ms1 * 1e-3) / 1e9, 3), "unit": "Gtps",
                "ms_per_step": round(ms1, 5), "launches_per_step": len(vps),
                "algorithmic_bytes_per_launch": b1, "achieved_GBps": round(a1, 1),
                "frac": round(a1 / _peaks()[0], 4)}
        # the same step without the normal-cone test (frustum + per-triangle only)
        db_nc = mc.DeviceBatch(blob, "cuda")
        with torch.cuda.stream(stream):
            g_nc = capture_cull(db_nc)
            nc_t = []
            for i in range(3 + max(3, args.steps // 10)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g_nc.launch(stream)
                e1.record(stream)
                flush.zero_()
                if i >= 3:
                    nc_t.append((e0, e1))
            torch.cuda.synchronize()
        nc_ms = float(np.mean([a_.elapsed_time(b_) for a_, b_ in nc_t]))
        assert int(out["status"].item()) == 0
        counts_nc = counts.cpu().numpy().astype(np.int64)
        # the same step with survivors in meshlet order (decoupled look-back)
        d_order = torch.empty(int(mc.lib().mc_cull_order_bytes(mc.C.byref(db.c))), dtype=torch.uint8,
                              device="cuda")
        with torch.cuda.stream(stream):
            or_t = []
            for i in range(3 + max(3, args.steps // 10)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for v in range(len(vps)):
                    mc.mc_decode_cull_ordered(db, d_vps[v], tri, counts[v:v + 1], out["pos"],
                                              out["status"], scratch, d_order, tune, stream)
                e1.record(stream)
                flush.zero_()
                if i >= 3:
                    or_t.append((e0, e1))
            torch.cuda.synchronize()
        or_ms = float(np.mean([a_.elapsed_time(b_) for a_, b_ in or_t]))
        assert int(out["status"].item()) == 0
        assert np.array_equal(counts.cpu().numpy().astype(np.int64), counts_np)
        extra["cull_ordered"] = {
            "value": round(input_tris * len(vps) / (or_ms * 1e-3) / 1e9, 3), "unit": "Gtps",
            "ms_per_step": round(or_ms, 5), "launches_per_step": len(vps),
            "note": "survivors in meshlet order; launched one view at a time (no graph)"}
        extra["cull_without_cones"] = {
            "value": round(input_tris * len(vps) / (nc_ms * 1e-3) / 1e9, 3), "unit": "Gtps",
            "ms_per_step": round(nc_ms, 5),
            "kept_fraction_mean": float(counts_nc.mean() / input_tris),
            "algorithmic_bytes_per_launch": W.cull_bytes(stats, arrays, vps, counts_nc,
                                                         views_per_launch=cv)}
    roof = None
    if bytes_per_launch:
        ach = bytes_per_launch / per_launch_s / 1e9
        tr = NCU_TRAFFIC.get(args.config)
        traffic = None
        if (tr and tr[0] == _kernel_hash(args.config) and args.codec == "reuse" and not args.attrs
                and (args.config != 4 or args.cull_views == 8)):
            traffic = int(tr[1] * stats["total_tris"])  # per launch (8 views for cfg4)
        roof = {"bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "traffic": traffic,
                "peak_kind": f"{peak_kind} copy bandwidth (MEASURED_PEAKS hbm_gbs)",
                "algorithmic_bytes_per_launch": bytes_per_launch,
                "bytes_per_input_triangle": round(bytes_per_launch / input_tris, 2),
                "frac_of_nominal": round(ach / NOMINAL_HBM_GBS, 4),
                "block_padding_bytes": None if cull else nbytes["padding"]}
    if cull:
        extra["cull"] = {"kept_fraction_mean": float(counts_np.mean() / input_tris),
                         "views": len(vps), "views_per_launch": cv,
                         "triangles_per_step": input_tris * len(vps)}
    res = {
        "metric": METRIC, "value": round(value, 3), "unit": "Gtps", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32/f32", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.config] + (" [plain GTS connectivity]"
                                                          if args.codec == "gts" else "")
                   + (" [8-channel vertices: position, normal, texture coordinate; 32 B out]"
                      if args.attrs else "")
                   + (f" [reduced to >= {args.cfg4_tris} triangles]"
                      if args.config == 4 and args.cfg4_tris != 50_000_000 else ""),
                   "connectivity_bits_per_triangle": round(stats["conn_bits"] / input_tris, 3),
                   "input_triangles": input_tris,
                   "decoded_triangle_slots": stats["total_tris"], "vertices": stats["total_verts"],
                   "meshlets": stats["n_meshlets"], "l2": f"flushed between steps ({flush_mb} MB write, L2 {l2 >> 20} MB)",
                   "parallelism": f"{ws} independent replica(s), no collective"},
        "decoded_slot_gtps": round(aggregate_gtps(ws, stats["total_tris"] * views, args.steps,
                                                  total_ms), 3),
        "latency_ms": {"min": round(float(times.min()), 5),
                       "p50": round(float(np.percentile(times, 50)), 5),
                       "p99": round(float(np.percentile(times, 99)), 5)},
        "roofline": roof, "gpu_launches": int(launches), "clocks": clk.summary(),
        "plain": plain, "e2e": e2e, "build_s": round(t_build, 1),
    }
    res.update(extra)
    if rank == 0 and not args.no_cpu_baseline:
        res["cpu_baseline"] = cpu_oracle_baseline(blob, args.cpu_seconds, vps[0] if cull else None)
    if rank == 0:
        print(json.dumps(res), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
