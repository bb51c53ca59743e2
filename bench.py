"""Benchmark of the SurfelWarp per-frame hot path on one GB300.

A step is one frame of the full-size plain workload: upload a 640x480 depth
frame, 10 Gauss-Newton x 20 PCG iterations of the non-rigid solve over a
300k-surfel / 2048-node model of a bending sphere, then fusion and the inverse
warp.  Frames come from a seeded synthetic sequence rendered on the host
before timing.  Device timing: CUDA events on the library's stream around
each step, L2 flushed (a 512 MiB write) between steps, outside the events.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle (the only reference there is)
on a bounded sample of the same workload.
"""
import argparse
import json
import multiprocessing as mp
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "frames/s & p50/p99 frame latency: served batch vs plain GN solve, same GB300"
WORKLOAD = "plain_full: 640x480 bending sphere, 300k surfels, 2048 nodes, 10 GN x 20 PCG + fusion per frame"


def _render(args):
    seed, t = args
    import synth
    return t, synth.plain_full(seed=seed).frame(t)


def render_frames(seed, ts, procs):
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=max(1, min(procs, len(ts)))) as pool:
        out = dict(pool.map(_render, [(seed, t) for t in ts]))
    return [out[t] for t in ts]


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        try:
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9 and parts[1].isdigit():
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = sorted(int(r[1]) for r in rows)
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": int(rows[0][2]), "samples": len(rows),
                "reasons": sorted(reasons)}


def cpu_baseline_sample(scene, frame, gn, pcg):
    """Time the FP64 oracle on a bounded sample: one frame, 2 GN x pcg, fusion;
    scaled to frames/s of the full 10-GN frame by the GN fraction."""
    import oracle
    c = scene.cam
    st = oracle.OracleStream(oracle.Params(c.width, c.height, c.fx, c.fy, c.cx, c.cy))
    st.set_model(scene.surfel_v, scene.surfel_n, scene.surfel_r, scene.surfel_c, scene.surfel_t,
                 scene.node_p, scene.node_sigma)
    t0 = time.perf_counter()
    st.upload_depth(frame, 1)
    t1 = time.perf_counter()
    gs = 2
    st.solve_frame(gs, pcg)
    t2 = time.perf_counter()
    st.fuse_frame()
    t3 = time.perf_counter()
    per_frame = (t1 - t0) + (t2 - t1) * gn / gs + (t3 - t2)
    return {"value": 1.0 / per_frame, "unit": "frames/s", "cores": 1, "kind": "oracle",
            "sample": f"1 frame, {gs} of {gn} GN iterations x {pcg} PCG timed, solve scaled by {gn}/{gs}, "
                      "depth processing and fusion timed whole; numpy FP64, single-threaded BLAS"}


def run_reference(args):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import synth
    scene = synth.plain_full(seed=0)
    frames = render_frames(0, [1, 2], 2)
    import oracle  # noqa: F401
    times = []
    for k in range(args.warmup + args.steps):
        b = cpu_baseline_sample(scene, frames[k % 2], scene.gn_iters, scene.pcg_iters)
        if k >= args.warmup:
            times.append(1.0 / b["value"])
    ms = 1000.0 * float(np.mean(times))
    line = {"impl": "reference", "metric": METRIC, "value": 1000.0 / ms, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": b["sample"]},
            "cpu_baseline": {"value": 1000.0 / ms, "unit": "frames/s", "cores": 1, "kind": "oracle",
                             "sample": b["sample"]},
            "e2e": {"value": 1000.0 / ms, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    import synth
    scene = synth.plain_full(seed=0)
    n_frames = args.warmup + args.steps
    ts = [1 + (k % (scene.n_frames - 1)) for k in range(n_frames)]
    frames = render_frames(0, sorted(set(ts)), os.cpu_count() or 4)
    frame_of = dict(zip(sorted(set(ts)), frames))

    import torch
    import paper_1904_13073_gb300 as sw
    from paper_1904_13073_gb300 import build as B
    B.build()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    stream = torch.cuda.Stream()
    c = scene.cam
    v4, n4, t2, node4 = sw.model_arrays(scene)
    h = sw.sw_create_stream(sw.params_for(c, len(v4), len(node4)), stream)
    sw.sw_set_model(h, v4, n4, t2, node4)
    dev_frames = {t: torch.from_numpy(f).cuda() for t, f in frame_of.items()}
    host_frames = {t: torch.from_numpy(f).pin_memory() for t, f in frame_of.items()}
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    gn, pcg = scene.gn_iters, scene.pcg_iters
    torch.cuda.synchronize()

    def step(t, host):
        sw.sw_upload_depth(h, host_frames[t] if host else dev_frames[t], t)
        sw.sw_solve_frame(h, gn, pcg, want_stats=False)
        sw.sw_fuse_frame(h)

    # warm-up (also captures the solve graph)
    for k in range(args.warmup):
        step(ts[k], False)
    torch.cuda.synchronize()

    # device-resident timed region
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(os.path.join(ROOT, "gpurun_out", f"clocks_rank{rank}.csv") if os.path.isdir(
            os.path.join(ROOT, "gpurun_out")) else "/tmp/sw_clocks.csv") as clk:
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xff)
                starts[k].record(stream)
            step(ts[args.warmup + k], False)
            ends[k].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    lat = np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])
    ms = float(lat.sum()) / args.steps
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    clocks = clk.summary()

    # end to end through the C ABI: host depth in, node state out, every step
    pos = np.empty((len(node4), 4), np.float32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e_lat = []
    for k in range(args.steps):
        s0 = time.perf_counter()
        step(ts[args.warmup + k], True)
        pos, dq = sw.sw_read_nodes(h)
        e_lat.append(time.perf_counter() - s0)
    torch.cuda.synchronize()
    e2e_ms = 1000.0 * (time.perf_counter() - t0) / args.steps
    sw.sw_destroy_stream(h)

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": world * 1000.0 / ms, "unit": "frames/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "width": c.width, "height": c.height, "surfels": len(v4),
                   "nodes": len(node4), "gn_iters": gn, "pcg_iters": pcg, "streams": 1,
                   "l2": "flushed between steps (512 MiB write outside the events)",
                   "parallelism": "replicas" if world > 1 else "single"},
        "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
        "e2e": {"value": world * 1000.0 / e2e_ms, "unit": "frames/s",
                "h2d_bytes_per_step": c.width * c.height * 4, "d2h_bytes_per_step": len(node4) * 48,
                "p50_ms": 1000.0 * float(np.percentile(e_lat, 50)), "p99_ms": 1000.0 * float(np.percentile(e_lat, 99))},
        "clocks": clocks,
        "gpu_launches": None,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample(scene, frame_of[ts[0]], gn, pcg)
    print(json.dumps(line))


if __name__ == "__main__":
    main()
