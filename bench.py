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
import tempfile
import subprocess
import sys
import time

os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "frames/s & p50/p99 frame latency: served batch vs plain GN solve, same GB300"
WORKLOAD = "plain_full: 640x480 bending sphere, 300k surfels, 2048 nodes, 10 GN x 20 PCG + fusion per frame"


def _render(args):
    seed, t = args
    import synth
    return t, synth.plain_full(seed=seed).frame(t)


def max_over_ranks(value, dist, torch, device):
    """The largest of every rank's value (the job's time is its slowest
    replica's); the same on every rank."""
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_frames_per_s(ms_per_step_max, world):
    """Whole-job throughput of `world` replicas that each advance one frame
    per step: every replica's frames over the slowest replica's time."""
    return world * 1000.0 / ms_per_step_max


def render_frames(seed, ts, procs):
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=max(1, min(procs, len(ts)))) as pool:
        out = dict(pool.map(_render, [(seed, t) for t in ts]))
    return [out[t] for t in ts]


class Clocks:
    """nvidia-smi sampling during the timed region.  Each sample carries
    nvidia-smi's own timestamp; `__enter__` returns once the first sample
    is written (so that the sampler is running before the region starts),
    `region()` marks the timed region's start and end on the host clock, and
    `summary()` keeps the samples taken inside it (the nearest one on each
    side when the region is shorter than the sampling interval)."""

    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    INTERVAL_MS = 10

    def __init__(self, path):
        self.path = path
        self.proc = None
        self.t0 = self.t1 = None

    def _launch(self, interval_ms):
        self.f = open(self.path, "w")
        self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}", "--format=csv,noheader,nounits",
                                      "-lms", str(interval_ms)], stdout=self.f, stderr=subprocess.DEVNULL)
        deadline = time.time() + 5.0
        while time.time() < deadline and self.proc.poll() is None:
            if os.path.getsize(self.path) > 0:
                return True
            time.sleep(0.01)
        return os.path.getsize(self.path) > 0 and self.proc.poll() is None

    def __enter__(self):
        try:
            if not self._launch(self.INTERVAL_MS):   # a sampler that refuses the short interval: 100 ms
                if self.proc.poll() is None:
                    self.proc.terminate()
                self.proc.wait()
                self.f.close()
                self.INTERVAL_MS = 100
                self._launch(self.INTERVAL_MS)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(2.5 * self.INTERVAL_MS / 1000.0)   # the sample after the region
            self.proc.terminate()
            self.proc.wait()
            self.f.close()

    def start(self):
        self.t0 = time.time()

    def stop(self):
        self.t1 = time.time()

    @staticmethod
    def parse(lines):
        """(epoch seconds, fields after the timestamp) per well-formed line."""
        import datetime
        out = []
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10 or not parts[2].isdigit():
                continue
            try:
                t = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                continue
            out.append((t, parts[1:]))
        return out

    @staticmethod
    def summarise(samples, t0, t1):
        if not samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "samples": 0, "reasons": ["no samples"]}
        inside = [r for t, r in samples if t0 is not None and t1 is not None and t0 <= t <= t1]
        n_inside = len(inside)
        if not inside:   # a region shorter than the interval: the samples just before and after it
            before = [r for t, r in samples if t0 is not None and t < t0]
            after = [r for t, r in samples if t1 is not None and t > t1]
            inside = before[-1:] + after[:1] or [samples[-1][1]]
        sm = sorted(int(r[1]) for r in inside)
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in inside:
            for k, nm in enumerate(names):
                if r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": int(inside[0][2]), "samples": n_inside,
                "samples_used": len(inside), "interval_ms": Clocks.INTERVAL_MS, "reasons": sorted(reasons)}

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        with open(self.path) as f:
            return self.summarise(self.parse(f), self.t0, self.t1)


def measured_hbm_peak():
    """Measured copy bandwidth of this machine's GB300 (GB/s), else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def stage_bytes(n_s, n_n, nnzb, n_corr, n_pix, pcg_iters, merged=True):
    """Algorithmic bytes per launch of each stage (what the stage must move at
    least, per unit of work):
      depth      4 B depth read + 32 B of V/N maps written per pixel
      reg        144 B per 6x6 block written + 80 B of node data per node
      data       64 B per surfel (v_ref, n_ref, 4-NN ids, weights)
                 + 32 B per association (V, N gathered) + 32 B per node (DQ)
                 + 144 B per block and 24 B per node of JᵀJ / Jᵀe written;
                 with `merged` (the FP32 modes assemble both terms in one
                 launch, timed as the data stage) + the regulariser's 80 B
                 of node data per node, the system still written once
      pcg        per iteration 144 B per block (A read) + 192 B per node
                 (8 FP32 6-vectors), plus 252 B per node for the set-up
      fusion     96 B per surfel (warp: 64 read + 32 written) + 24 B per
                 surfel (index map) + 160 B per pixel (16 map entries + maps)
    """
    return {
        "depth": 36.0 * n_pix,
        "reg_assembly": 144.0 * nnzb + 80.0 * n_n,
        "data_assembly": 64.0 * n_s + 32.0 * n_corr + 32.0 * n_n + 144.0 * nnzb + 24.0 * n_n
        + (80.0 * n_n if merged else 0.0),
        "pcg": pcg_iters * (144.0 * nnzb + 192.0 * n_n) + 252.0 * n_n,
        "fusion": 120.0 * n_s + 160.0 * n_pix,
    }


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, mean of
# the two launches of one ncu capture) of this workload's kernels as they are
# now (the "pcg" stage is the preconditioner launch plus the cluster PCG
# launch; "data_assembly" is k_assemble, both terms);
# profiles/k_pcg_cluster_plain_full_300k_2048.md and
# profiles/k_assemble_plain_full_300k_2048.md give the commands.
PROFILED_TRAFFIC = {"pcg": 563968.0 + 3055872.0, "data_assembly": 26728960.0 + 26496.0}


def roofline(stage_ms, stage_n, n_s, n_n, nnzb, n_corr, n_pix, pcg_iters):
    peak, src = measured_hbm_peak()
    nbytes = stage_bytes(n_s, n_n, nnzb, n_corr, n_pix, pcg_iters)
    stages = {}
    for k, b in nbytes.items():
        if stage_n[k] == 0:
            continue
        per_launch_s = stage_ms[k] / stage_n[k] / 1000.0
        gbs = b / per_launch_s / 1e9
        stages[k] = {"achieved": gbs, "frac": gbs / peak, "us_per_launch": per_launch_s * 1e6,
                     "bytes_per_launch": b, "traffic": PROFILED_TRAFFIC.get(k)}
    dom = max(stages, key=lambda k: stage_ms[k])
    d = stages[dom]
    return {"stages": stages,
            "dominant": {"kernel": dom, "bound": "hbm", "achieved": d["achieved"], "peak": peak,
                         "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else src,
                         "unit": "GB/s", "frac": d["frac"], "traffic": PROFILED_TRAFFIC.get(dom),
                         "bytes_per_launch": d["bytes_per_launch"], "us_per_launch": d["us_per_launch"]}}


def oracle_stream(scene):
    import oracle
    c = scene.cam
    st = oracle.OracleStream(oracle.Params(c.width, c.height, c.fx, c.fy, c.cx, c.cy))
    st.set_model(scene.surfel_v, scene.surfel_n, scene.surfel_r, scene.surfel_c, scene.surfel_t,
                 scene.node_p, scene.node_sigma)
    return st


def host_cpu():
    """(CPU model, logical cores) of this host, for the baseline's record."""
    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Vendor ID") and not model:
                model = line.split(":", 1)[1].strip()
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return model or "unknown", os.cpu_count() or 1


def _oracle_replica(args):
    """One replica stream of the oracle on the full-size workload: set-up
    and `n_warm` whole frames untimed, then, once every replica is ready
    (the barrier), `n_frames` whole frames (depth processing, 10
    Gauss-Newton x 20 PCG iterations, fusion); returns their (start, end)
    wall-clock times."""
    seed, first_t, n_warm, n_frames, barrier = args
    import synth
    scene = synth.plain_full(seed=seed)
    ts = [1 + (first_t + k) % (scene.n_frames - 1) for k in range(n_warm + n_frames)]
    frames = [scene.frame(t) for t in ts]
    st = oracle_stream(scene)

    def run(k):
        st.upload_depth(frames[k], k + 1)
        st.solve_frame(scene.gn_iters, scene.pcg_iters)
        st.fuse_frame()
    for k in range(n_warm):
        run(k)
    barrier.wait()
    out = []
    for k in range(n_warm, n_warm + n_frames):
        t0 = time.time()
        run(k)
        out.append((t0, time.time()))
    return out


def oracle_whole_frames(n_frames, procs, n_warm=0):
    """The FP64 oracle as it stands on the host cores: `procs` independent
    replica streams (one single-threaded process each) share `n_frames`
    whole frames of the full-size workload after `n_warm` untimed frames
    each; the timed region runs from their common start to the last frame's
    end.  Returns (frames/s over the region, seconds per frame of one
    replica, region seconds, procs)."""
    procs = max(1, min(procs, n_frames))
    share = [n_frames // procs + (1 if k < n_frames % procs else 0) for k in range(procs)]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        barrier = m.Barrier(procs)
        with ctx.Pool(processes=procs) as pool:
            res = pool.map(_oracle_replica, [(0, 7 * k, n_warm, share[k], barrier) for k in range(procs)])
    starts = [a for r in res for a, _ in r]
    ends = [b for r in res for _, b in r]
    region = max(ends) - min(starts)
    per_frame = float(np.mean([b - a for r in res for a, b in r]))
    return n_frames / region, per_frame, region, procs


def oracle_sample_text(n_frames, procs, per_frame):
    model, ncpu = host_cpu()
    return (f"{n_frames} whole frames of the full-size workload (depth processing, 10 Gauss-Newton x 20 PCG, "
            f"fusion; nothing extrapolated) on {procs} independent single-threaded replica streams of the "
            f"numpy FP64 oracle; {per_frame:.2f} s per frame per replica; host {model}, {ncpu} logical cores")


def cpu_baseline_sample(n_frames=None):
    """The FP64 oracle on a bounded sample of the same workload: one whole
    timed frame per host core (at most 16), all in parallel, after set-up."""
    _, ncpu = host_cpu()
    procs = max(1, min(16, ncpu))
    n = n_frames or procs
    fps, per_frame, region, procs = oracle_whole_frames(n, procs)
    model, ncpu = host_cpu()
    return {"value": fps, "unit": "frames/s", "cores": procs, "kind": "oracle",
            "sample": oracle_sample_text(n, procs, per_frame), "cpu": model, "nproc": ncpu,
            "seconds_per_frame_one_core": per_frame, "timed_region_s": region}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    _, ncpu = host_cpu()
    procs = max(1, min(16, ncpu, args.steps))
    # warm-up: whole frames on every replica, untimed (W in all, at least
    # one per replica), then the timed region over the K steps
    n_warm = max(1, -(-args.warmup // procs))
    fps, per_frame, region, procs = oracle_whole_frames(args.steps, procs, n_warm)
    model, ncpu = host_cpu()
    ms = 1000.0 * region / args.steps
    sample = oracle_sample_text(args.steps, procs, per_frame)
    line = {"impl": "reference", "metric": METRIC, "value": fps, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": fps, "unit": "frames/s", "cores": procs, "kind": "oracle",
                             "sample": sample, "cpu": model, "nproc": ncpu,
                             "seconds_per_frame_one_core": per_frame},
            "e2e": {"value": fps, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def _batch_member_data(args):
    """Build member k of the uneven multi-stream workload in a worker process."""
    k, frame_ids, scale = args
    import synth
    from paper_1904_13073_gb300 import model_arrays
    s = synth.batch_member(k, scale=scale)
    c = s.cam
    return k, {"name": s.name, "cam": (c.width, c.height, c.fx, c.fy, c.cx, c.cy),
               "arrays": model_arrays(s), "frames": [s.frame(t) for t in frame_ids],
               "gn": s.gn_iters, "pcg": s.pcg_iters}


def _large_member_data(args):
    """A large stream of the serving workload: 640x480 sphere, 4096 nodes."""
    seed, frame_ids = args
    import synth
    from paper_1904_13073_gb300 import model_arrays
    s = synth.plain_full(seed=100 + seed, n_nodes=4096)
    c = s.cam
    return seed, {"name": f"sphere_640x480_{len(s.surfel_v)}s_{len(s.node_p)}n_large",
                  "cam": (c.width, c.height, c.fx, c.fy, c.cx, c.cy),
                  "arrays": model_arrays(s), "frames": [s.frame(t) for t in frame_ids],
                  "gn": s.gn_iters, "pcg": s.pcg_iters}


def large_workload(n_models, frame_ids):
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=max(1, min(os.cpu_count() or 4, n_models))) as pool:
        out = dict(pool.map(_large_member_data, [(k, frame_ids) for k in range(n_models)]))
    return [out[k] for k in range(n_models)]


def run_served(sw, members, large, n_regular, n_large, seconds, rate_hz, budget_gb, gn, pcg, seed=0,
               plain=False, wait_admission=True, adaptive=True):
    """The serving workload: n_regular streams of the uneven sizes (models
    reused from the uneven batch) plus n_large large ones, each submitting
    depth frames as a Poisson process of rate_hz (the same arrival trace for
    a given seed and rate); an eighth of the regular streams joins a third
    into the run and another eighth leaves at two thirds.  Frames go through
    the library's server: admission against the budget, then continuous
    batching (plain=False; with adaptive, the server's default, a step runs
    its frames one by one through their streams' own calls when its measured
    times say that is cheaper) or the plain one-frame-at-a-time path
    (plain=True, sw_server_set_plain).  Latency is completion minus
    submission on the server's clock.  A frame refused because its stream's
    queue is full or the stream is not admitted yet is counted as dropped.
    With wait_admission the arrivals start once every initial stream is
    admitted; without it (a budget that binds) they start at once and the
    admitted / waiting counts are sampled through the run."""
    import heapq
    from types import SimpleNamespace
    rng = np.random.default_rng(seed)
    specs = [members[k % len(members)] for k in range(n_regular)] + [large[k % len(large)] for k in range(n_large)]
    n = len(specs)
    late = set(range(n_regular - n_regular // 8, n_regular))
    leaving = set(range(n_regular // 8))
    srv = sw.sw_server_create(int(budget_gb * (1 << 30)), gn, pcg, queue_depth=4)
    if plain:
        sw.sw_server_set_plain(srv, True)
    sw.sw_server_set_adaptive(srv, adaptive)
    ids = {}

    def open_stream(k):
        m = specs[k]
        w, h_, fx, fy, cx, cy = m["cam"]
        cam = SimpleNamespace(width=w, height=h_, fx=fx, fy=fy, cx=cx, cy=cy)
        v4, n4, t2, node4 = m["arrays"]
        ids[k] = sw.sw_server_open(srv, sw.params_for(cam, len(v4), len(node4)), v4, n4, t2, node4)

    samples = []
    try:
        for k in range(n):
            if k not in late:
                open_stream(k)
        t_adm = time.perf_counter()
        while wait_admission and not all(sw.sw_server_is_admitted(srv, ids[k]) for k in ids):
            if time.perf_counter() - t_adm > 300:
                raise RuntimeError("streams were not admitted")
            time.sleep(0.01)
        # frames: the member's depth frames back and forth
        seqs = {k: [f for f in specs[k]["frames"]] + [f for f in specs[k]["frames"][-2:0:-1]] for k in range(n)}
        pos = {k: 0 for k in range(n)}
        t0 = time.perf_counter()
        events = [(float(rng.exponential(1.0 / rate_hz)), k) for k in range(n) if k not in late]
        heapq.heapify(events)
        joined, left = False, False
        sent = dropped = 0
        next_sample = 0.0
        while events:
            t, k = heapq.heappop(events)
            if t > seconds:
                continue
            if t >= next_sample:
                st_ = sw.sw_server_read_stats(srv)
                samples.append((t, int(st_["admitted"]), int(st_["waiting"])))
                next_sample = t + 0.1
            if not joined and t >= seconds / 3:
                for j in late:
                    open_stream(j)
                    heapq.heappush(events, (t + float(rng.exponential(1.0 / rate_hz)), j))
                joined = True
            if not left and t >= 2 * seconds / 3:
                for j in leaving:
                    sw.sw_server_close(srv, ids[j])
                left = True
            if left and k in leaving:
                continue
            delay = t0 + t - time.perf_counter()
            if delay > 0:
                time.sleep(delay)
            seq = seqs[k]
            st = sw.sw_server_submit(srv, ids[k], seq[pos[k] % len(seq)], 2 + pos[k])
            if st == 0:
                pos[k] += 1
                sent += 1
            else:
                dropped += 1
            heapq.heappush(events, (t + float(rng.exponential(1.0 / rate_hz)), k))
        sw.sw_server_wait(srv, 120000)
        res = []
        while True:
            got = sw.sw_server_poll(srv)
            if not got:
                break
            res += got
        stats = sw.sw_server_read_stats(srv)
    finally:
        sw.sw_server_destroy(srv)
        sw.sw_set_memory_budget(0)
    ok = [r for r in res if r["status"] == 0]
    lat = np.array([r["done_ms"] - r["submit_ms"] for r in ok]) if ok else np.zeros(1)
    span_s = (max(r["done_ms"] for r in ok) - min(r["submit_ms"] for r in ok)) / 1000.0 if ok else 1.0
    offered = rate_hz * n
    out = {"workload": f"{n_regular} streams of the uneven sizes + {n_large} large (640x480, 4096 nodes), "
                       f"Poisson arrivals at {rate_hz:.3g} Hz per stream for {seconds:g} s; "
                       f"{len(late)} join at 1/3, {len(leaving)} leave at 2/3; {gn} GN x {pcg} PCG + fusion",
           "path": "plain (one frame at a time)" if plain else
                   "continuous batching, adaptive (batch or stream by stream per step)" if adaptive else
                   "continuous batching (every step one batch)",
           "budget_gb": budget_gb, "frames_per_s": len(ok) / span_s, "offered_frames_per_s": offered,
           "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                          "max": float(lat.max())},
           "frames_done": len(ok), "frames_failed": len(res) - len(ok), "frames_dropped": dropped,
           "drop_rate": dropped / max(1, dropped + sent),
           "mean_batch": float(np.mean([r["batch_size"] for r in ok])) if ok else 0.0,
           "steps": int(stats["steps"]), "steps_alone": int(stats["steps_alone"]), "gpu_busy_frac": float(stats["busy_ms"]) / 1000.0 / max(span_s, 1e-9),
           "streams": n, "memory_gb_at_end": stats["memory_in_use"] / float(1 << 30)}
    if samples:
        out["admitted_max"] = max(a for _, a, _ in samples)
        out["waiting_max"] = max(w for _, _, w in samples)
        out["admitted_waiting_samples"] = [[round(t, 2), a, w] for t, a, w in samples[::5]]
    return out


def served_summary(r):
    return {k: r[k] for k in ("frames_per_s", "offered_frames_per_s", "latency_ms", "frames_done", "frames_dropped",
                              "drop_rate", "mean_batch", "steps", "steps_alone", "gpu_busy_frac")}


def run_served_sweep(sw, members, large, args, gn, pcg):
    """Continuous batching against the plain server on the same arrival
    traces: the saturating point first (its served frames/s is the batched
    capacity), then offered loads of 25, 50 and 75% of that capacity for
    the adaptive server (the default), the server that batches every step,
    and the plain one, and one run whose memory budget admits only part of
    the streams at a time (admission binds; the arrivals do not wait for
    it)."""
    n_streams = args.served_streams + args.served_large
    sat = run_served(sw, members, large, args.served_streams, args.served_large, args.served_seconds,
                     args.served_rate, args.served_budget_gb, gn, pcg)
    cap = sat["frames_per_s"]
    points = []
    for frac in (0.25, 0.5, 0.75):
        rate = frac * cap / n_streams
        b = run_served(sw, members, large, args.served_streams, args.served_large, args.served_seconds, rate,
                       args.served_budget_gb, gn, pcg, seed=1)
        ba = run_served(sw, members, large, args.served_streams, args.served_large, args.served_seconds, rate,
                        args.served_budget_gb, gn, pcg, seed=1, adaptive=False)
        pl = run_served(sw, members, large, args.served_streams, args.served_large, args.served_seconds, rate,
                        args.served_budget_gb, gn, pcg, seed=1, plain=True)
        points.append({"offered_frac_of_batched_capacity": frac, "rate_hz_per_stream": rate,
                       "batched": served_summary(b), "batched_every_step": served_summary(ba),
                       "plain": served_summary(pl)})
    # a budget of about half what the streams hold: admission binds
    need_gb = max(sat["memory_gb_at_end"], 0.1)
    tight = run_served(sw, members, large, args.served_streams, args.served_large, args.served_seconds,
                       0.5 * cap / n_streams, 0.5 * need_gb, gn, pcg, seed=2, wait_admission=False)
    out = dict(sat)
    out["load_sweep"] = points
    out["binding_budget"] = tight
    return out


def batch_workload(n_streams, frame_ids, scale=1.0):
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=max(1, min(os.cpu_count() or 4, n_streams))) as pool:
        out = dict(pool.map(_batch_member_data, [(k, frame_ids, scale) for k in range(n_streams)]))
    return [out[k] for k in range(n_streams)]


def run_batched(sw, torch, members, rounds, warmup, flush, stream):
    """The uneven streams advanced one frame per round, first one stream at a
    time (every call serialised on one CUDA stream: the plain solve), then as
    one batch (one launch per stage for all streams).  Device time per round
    by CUDA events; L2 flushed between rounds outside the events."""
    from types import SimpleNamespace
    handles, dev_frames, nnzb, n_s, n_n, n_pix = [], [], [], [], [], []
    for m in members:
        w, h_, fx, fy, cx, cy = m["cam"]
        cam = SimpleNamespace(width=w, height=h_, fx=fx, fy=fy, cx=cx, cy=cy)
        v4, n4, t2, node4 = m["arrays"]
        hd = sw.sw_create_stream(sw.params_for(cam, len(v4), len(node4)), stream)
        sw.sw_set_model(hd, v4, n4, t2, node4)
        handles.append(hd)
        dev_frames.append([torch.from_numpy(f).cuda() for f in m["frames"]])
        n_s.append(len(v4))
        n_n.append(len(node4))
        n_pix.append(w * h_)
    gn, pcg = members[0]["gn"], members[0]["pcg"]
    nf = len(members[0]["frames"])
    pp = list(range(nf)) + list(range(nf - 2, 0, -1))   # the frames back and forth, no jumps
    S = len(members)
    for hd, fr in zip(handles, dev_frames):       # structure sizes and a first frame
        sw.sw_upload_depth(hd, fr[0], 1)
        nnzb.append(sw.sw_debug_assemble(hd)[0])
    torch.cuda.synchronize()

    def timed(fn, n_rounds, n_warm):
        lat = []
        for r in range(n_warm + n_rounds):
            with torch.cuda.stream(stream):
                flush.fill_(r & 0xff)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn(r)
            b.record(stream)
            torch.cuda.synchronize()
            if r >= n_warm:
                lat.append(a.elapsed_time(b))
        return np.array(lat)

    # both runs play the same continuous sequence from the same fresh models:
    # round r is frame pp[r] (back and forth, no jumps) with frame id 2 + r
    def reset_models():
        for hd, m in zip(handles, members):
            sw.sw_set_model(hd, *m["arrays"])

    def plain_round(r):
        for hd, fr in zip(handles, dev_frames):
            sw.sw_upload_depth(hd, fr[pp[r % len(pp)]], 2 + r)
            sw.sw_solve_frame(hd, gn, pcg, want_stats=False)
            sw.sw_fuse_frame(hd)

    # the first pass over the streams (one frame of every stream) is played
    # untimed by both runs (the batched run tunes its PCG on it; the
    # autotune leaves the state as it found it); the later passes are timed
    reset_models()
    plain_round(0)
    lat_plain = timed(lambda r: plain_round(r + 1), rounds, warmup)
    reset_models()
    b = sw.sw_batch_create(handles, stream)

    def batch_round(r, stats=False):
        sw.sw_batch_upload_depth(b, [fr[pp[r % len(pp)]] for fr in dev_frames], [2 + r] * S)
        st = sw.sw_batch_solve(b, gn, pcg, want_stats=stats)
        sw.sw_batch_fuse(b)
        return st

    batch_round(0)
    tuned = sw.sw_batch_autotune(b, pcg)
    lat_batch = timed(lambda r: batch_round(r + 1), rounds, warmup)
    # live stage times of two more profiled batched rounds, and their associations
    sw.sw_batch_set_profiling(b, True)
    prof = {}
    n_corr_seen = [[] for _ in range(S)]
    for r in range(warmup + rounds + 1, warmup + rounds + 3):
        st = batch_round(r, stats=True)
        prof = sw.sw_batch_read_profile(b)
        for k in range(S):
            n_corr_seen[k] += st[k]["n_corr"]
    sw.sw_batch_set_profiling(b, False)
    n_corr = [int(np.mean(v)) for v in n_corr_seen]
    sw.sw_batch_destroy(b)
    for hd in handles:
        sw.sw_destroy_stream(hd)
    data_bytes = sum(stage_bytes(n_s[k], n_n[k], nnzb[k], n_corr[k], n_pix[k], pcg)["data_assembly"] for k in range(S))
    peak, src = measured_hbm_peak()
    t_data = prof["data_assembly"][0] / prof["data_assembly"][1] / 1000.0
    return {
        "workload": f"{S} streams of uneven size (depth 320x240..640x480, 40k-400k surfels, 256-4096 nodes, "
                    f"log-uniform; sphere / torus / wavy plane), {gn} GN x {pcg} PCG + fusion per frame",
        "streams": [m["name"] for m in members],
        "plain": {"frames_per_s": S * 1000.0 / float(lat_plain.mean()),
                  "round_ms_p50": float(np.percentile(lat_plain, 50)),
                  "round_ms_p99": float(np.percentile(lat_plain, 99))},
        "batched": {"frames_per_s": S * 1000.0 / float(lat_batch.mean()),
                    "round_ms_p50": float(np.percentile(lat_batch, 50)),
                    "round_ms_p99": float(np.percentile(lat_batch, 99))},
        "speedup": float(lat_plain.mean() / lat_batch.mean()),
        "autotune": {"pcg_rows_per_cta": tuned[0], "pcg_us_per_launch": tuned[1]},
        "stages_ms_per_round": {k: v[0] for k, v in prof.items()},
        "data_assembly_roofline": {"bound": "hbm", "achieved": data_bytes / t_data / 1e9, "peak": peak,
                                   "unit": "GB/s", "frac": data_bytes / t_data / 1e9 / peak,
                                   "bytes_per_launch": data_bytes, "us_per_launch": t_data * 1e6,
                                   "peak_source": src},
        "l2": "flushed between rounds (512 MiB write outside the events)",
    }


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-streams", type=int, default=16, help="streams of the uneven batched workload (0: skip)")
    ap.add_argument("--batch-rounds", type=int, default=5)
    ap.add_argument("--clocks-csv", default="", help="keep the nvidia-smi clock samples here ({rank} is replaced)")
    ap.add_argument("--served-streams", type=int, default=64, help="regular streams of the serving run (0: skip)")
    ap.add_argument("--served-large", type=int, default=8)
    ap.add_argument("--served-seconds", type=float, default=3.0)
    ap.add_argument("--served-rate", type=float, default=30.0)
    ap.add_argument("--served-budget-gb", type=float, default=120.0)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    import synth
    scene = synth.plain_full(seed=0)
    # one continuous sequence for every pass (warm-up, timed, profiled, end to
    # end), played back and forth past its last frame, so that tracking never
    # jumps; frame ids keep counting up
    prof_steps = min(args.steps, 8)
    n_frames = args.warmup + args.steps + prof_steps + args.steps
    last = scene.n_frames - 1
    period = 2 * (last - 1)

    def frame_at(k):
        m = k % period
        return 1 + (m if m < last else period - m)
    ts = [frame_at(k) for k in range(n_frames)]
    frames = render_frames(0, sorted(set(ts)), os.cpu_count() or 4)
    frame_of = dict(zip(sorted(set(ts)), frames))
    want_members = (args.batch_streams > 0 or args.served_streams > 0) and rank == 0
    members = batch_workload(max(args.batch_streams, 16), [2, 3, 4], 1.0) if want_members else []
    large = large_workload(2, [2, 3, 4]) if args.served_large > 0 and args.served_streams > 0 and rank == 0 else []

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

    def step(k, host, stats=False):
        t = ts[k]
        sw.sw_upload_depth(h, host_frames[t] if host else dev_frames[t], k + 1)
        st = sw.sw_solve_frame(h, gn, pcg, want_stats=stats)
        sw.sw_fuse_frame(h)
        return st

    # warm-up (also captures the solve graph), with the PCG granularity
    # autotuned on the first frame's system
    step(0, False)
    tuned_rows, tuned_us = sw.sw_autotune(h, pcg)
    pcg_mode = sw.sw_debug_pcg_mode(h)   # 3: the cluster PCG
    for k in range(1, args.warmup):
        step(k, False)
    torch.cuda.synchronize()

    # device-resident timed region
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks_csv = args.clocks_csv.replace("{rank}", str(rank)) if args.clocks_csv else os.path.join(
        tempfile.gettempdir(), f"sw_clocks_rank{rank}.csv")
    with Clocks(clocks_csv) as clk:
        torch.cuda.synchronize()
        clk.start()
        for k in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(k & 0xff)
                starts[k].record(stream)
            step(args.warmup + k, False)
            ends[k].record(stream)
        torch.cuda.synchronize()
        clk.stop()
    if dist:
        dist.barrier()
    lat = np.array([s.elapsed_time(e) for s, e in zip(starts, ends)])
    ms = float(lat.sum()) / args.steps
    if dist:
        ms = max_over_ranks(ms, dist, torch, "cuda")
    clocks = clk.summary()

    # stage timing, live: CUDA events recorded inside the captured solve graph
    # on the library's stream, over a second timed region of the same steps
    sw.sw_set_profiling(h, True)
    base = args.warmup + args.steps
    n_corr_seen = []
    stage_ms = {k: 0.0 for k in sw.PROFILE_STAGES}
    stage_n = {k: 0 for k in sw.PROFILE_STAGES}
    for k in range(prof_steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xff)
        st = step(base + k, False, stats=True)
        n_corr_seen += st["n_corr"]
        pr = sw.sw_read_profile(h)
        for name, (t_ms, n_l) in pr.items():
            stage_ms[name] += t_ms
            stage_n[name] += n_l
    sw.sw_set_profiling(h, False)
    n_corr = int(np.mean(n_corr_seen))   # correspondences per Gauss-Newton iteration
    nnzb = sw.sw_debug_assemble(h)[0]
    roof = roofline(stage_ms, stage_n, len(v4), len(node4), nnzb, n_corr, c.width * c.height, pcg)
    # the PCG is bound by synchronisation, not HBM: its latency bound is the
    # hops it must take (cluster PCG: two cluster barriers per iteration and
    # two at set-up) times one hop measured alone
    if pcg_mode == 3:
        ctas = sw.sw_debug_pcg_cluster(h, 0, 16, 0)[0]
        hop_us = sw.sw_debug_cluster_barrier_us(ctas)
        hops = 2 * pcg + 2
        meas = roof["stages"]["pcg"]["us_per_launch"]
        roof["stages"]["pcg"]["latency_bound"] = {
            "hops_per_launch": hops, "hop_us": hop_us, "bound_us": hops * hop_us, "measured_us": meas,
            "frac": hops * hop_us / meas,
            "note": "cluster barriers of the cluster PCG (2 per iteration, 2 at set-up) x one barrier of the same "
                    "cluster measured alone; the stage also holds the preconditioner launch"}
        if roof["dominant"]["kernel"] == "pcg":
            roof["dominant"]["latency_bound"] = roof["stages"]["pcg"]["latency_bound"]

    # end to end through the C ABI: host depth in, node state out, every step
    pos = np.empty((len(node4), 4), np.float32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e_lat = []
    for k in range(args.steps):
        s0 = time.perf_counter()
        step(base + prof_steps + k, True)
        pos, dq = sw.sw_read_nodes(h)
        e_lat.append(time.perf_counter() - s0)
    torch.cuda.synchronize()
    e2e_ms = 1000.0 * (time.perf_counter() - t0) / args.steps

    # rigid pre-alignment (a separate call, not part of the configuration's
    # frame): ICP iterations on the next frame, timed on the library's stream
    rigid = None
    k_r = base + prof_steps + args.steps - 1
    sw.sw_upload_depth(h, dev_frames[ts[k_r]], k_r + 2)
    rig_stats = sw.sw_rigid_align(h, 3)                 # warm-up, and the association count
    torch.cuda.synchronize()
    r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    r0.record(stream)
    for _ in range(5):
        sw.sw_rigid_align(h, 3, want_stats=False)
    r1.record(stream)
    torch.cuda.synchronize()
    rigid_it_us = 1000.0 * r0.elapsed_time(r1) / 15.0
    rig_bytes = 64.0 * len(v4) + 32.0 * float(np.mean([n for n, _ in rig_stats])) + 29 * 4.0 * (len(v4) / 256.0)
    peak, _src = measured_hbm_peak()
    rigid = {"iterations_timed": 15, "us_per_iteration": rigid_it_us,
             "correspondences": [int(n) for n, _ in rig_stats],
             "bytes_per_iteration": rig_bytes, "achieved_gbs": rig_bytes / rigid_it_us / 1e3,
             "frac": rig_bytes / rigid_it_us / 1e3 / peak}
    # splat visibility (Sec. 7, sw_params.visibility): the same frames on a
    # stream that predicts visibility before each solve, timed the same way
    hv = sw.sw_create_stream(sw.params_for(c, len(v4), len(node4), visibility=1), stream)
    sw.sw_set_model(hv, v4, n4, t2, node4)

    def vstep(k):
        sw.sw_upload_depth(hv, dev_frames[ts[k]], k + 1)
        sw.sw_solve_frame(hv, gn, pcg)
        sw.sw_fuse_frame(hv)
    for k in range(args.warmup):
        vstep(k)
    torch.cuda.synchronize()
    v_lat = []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        vstep(args.warmup + k)
        e1.record(stream)
        torch.cuda.synchronize()
        v_lat.append(e0.elapsed_time(e1))
    sw.sw_set_profiling(hv, True)
    k_v = args.warmup + args.steps
    sw.sw_upload_depth(hv, dev_frames[ts[k_v]], k_v + 1)
    v_stats = sw.sw_solve_frame(hv, gn, pcg, want_stats=True)
    sw.sw_fuse_frame(hv)
    v_prof = sw.sw_read_profile(hv)
    sw.sw_set_profiling(hv, False)
    sw.sw_destroy_stream(hv)
    visibility = {"frames_per_s": 1000.0 / float(np.mean(v_lat)), "ms_per_step": float(np.mean(v_lat)),
                  "visibility_ms": v_prof["visibility"][0], "n_corr_per_gn_iter": v_stats["n_corr"],
                  "n_corr_without": n_corr,
                  "note": "same workload and timing as the headline, with sw_params.visibility = 1: the "
                          "selected live surfels drawn as opaque disk splats before each solve, only "
                          "surfels that keep a pixel associated"}
    # the configuration's literal precision split: FP64 inner products in the
    # PCG (SW_PRECISION_MIXED_F64DOTS) instead of the default double-float
    # pairs, on the same frames, timed the same way
    hp64 = sw.sw_create_stream(sw.params_for(c, len(v4), len(node4), precision=sw.SW_PRECISION_MIXED_F64DOTS), stream)
    sw.sw_set_model(hp64, v4, n4, t2, node4)

    def pstep(k):
        sw.sw_upload_depth(hp64, dev_frames[ts[k]], k + 1)
        sw.sw_solve_frame(hp64, gn, pcg, want_stats=False)
        sw.sw_fuse_frame(hp64)
    pstep(0)
    sw.sw_autotune(hp64, pcg)
    for k in range(1, args.warmup):
        pstep(k)
    torch.cuda.synchronize()
    p_lat = []
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(k & 0xff)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pstep(args.warmup + k)
        e1.record(stream)
        torch.cuda.synchronize()
        p_lat.append(e0.elapsed_time(e1))
    precision_f64dots = {"frames_per_s": 1000.0 / float(np.mean(p_lat)),
                         "latency_ms": {"p50": float(np.percentile(p_lat, 50)), "p99": float(np.percentile(p_lat, 99))},
                         "pcg_mode": sw.sw_debug_pcg_mode(hp64),
                         "note": "same workload, frames and timing as the headline with FP64 PCG inner products "
                                 "(the configuration's precision split); the headline accumulates them in "
                                 "double-float pairs"}
    sw.sw_destroy_stream(hp64)
    # appending (a separate call after fusion, not part of the configuration's
    # frame): steady state on the full model, where the candidates are the
    # few pixels no surfel covers, frame after frame; the first call loads
    # the kernels and is not reported
    sw.sw_destroy_stream(h)
    room = len(v4) + c.width * c.height

    def append_case(keep, n_calls, keep_nodes=None, node_room=0):
        nodes = node4 if keep_nodes is None else node4[keep_nodes]
        ha = sw.sw_create_stream(sw.params_for(c, room, len(nodes) + node_room), stream)
        sw.sw_set_model(ha, v4[keep], n4[keep], t2[keep], nodes)
        out = []
        for k in range(n_calls):
            sw.sw_upload_depth(ha, dev_frames[ts[k]], k + 1)
            sw.sw_solve_frame(ha, gn, pcg)
            sw.sw_fuse_frame(ha)
            torch.cuda.synchronize()
            a0 = time.perf_counter()
            a_st = sw.sw_append_frame(ha)
            a_st["call_ms"] = 1000.0 * (time.perf_counter() - a0)
            out.append(a_st)
        sw.sw_destroy_stream(ha)
        return out
    appends = append_case(np.ones(len(v4), bool), 3)
    # and a model with 30% of its surfels cut away (the early-frame regime)
    x_cut = np.quantile(scene.surfel_v[:, 0], 0.7)
    cut_st = append_case(scene.surfel_v[:, 0] < x_cut, 3)   # the first fills the hole, the next ones the edges
    # and with the nodes of that region cut too, and room for 256 more: the
    # node graph is extended over the appended surfels
    ext_st = append_case(scene.surfel_v[:, 0] < x_cut, 1, scene.node_p[:, 0] < x_cut - scene.node_sigma[0], 256)[0]
    # the paper's whole per-frame pipeline, upload + solve + fusion + appending,
    # frame after frame on the cut model (wall clock with the device drained:
    # it includes the model rebuilds and the solve graph's re-capture after
    # each change)
    hp = sw.sw_create_stream(sw.params_for(c, room, len(node4)), stream)
    keep = scene.surfel_v[:, 0] < x_cut
    sw.sw_set_model(hp, v4[keep], n4[keep], t2[keep], node4)
    pipe = []
    for k in range(2 + args.steps):
        torch.cuda.synchronize()
        a0 = time.perf_counter()
        sw.sw_upload_depth(hp, dev_frames[ts[k]], k + 1)
        sw.sw_solve_frame(hp, gn, pcg, want_stats=False)
        sw.sw_fuse_frame(hp)
        a_st = sw.sw_append_frame(hp)
        torch.cuda.synchronize()
        pipe.append((1000.0 * (time.perf_counter() - a0), a_st["appended"], a_st["n_surfels"], a_st["resorted"]))
    sw.sw_destroy_stream(hp)
    steady_pipe = pipe[2:]   # the first frames fill the cut-away hole
    pipeline = {"frames_per_s": 1000.0 / float(np.mean([m for m, _, _, _ in steady_pipe])),
                "ms_per_frame": float(np.mean([m for m, _, _, _ in steady_pipe])),
                "appended_per_frame": float(np.mean([a for _, a, _, _ in steady_pipe])),
                "frames_with_appends": int(sum(1 for _, a, _, _ in steady_pipe if a > 0)),
                "frames_resorted": int(sum(1 for _, _, _, r in steady_pipe if r == 1)),
                "frames_pattern_rebuilt": int(sum(1 for _, _, _, r in steady_pipe if r == 2)),
                "first_frames": [{"ms": m, "appended": a, "surfels": n, "resorted": r} for m, a, n, r in pipe[:2]],
                "note": "upload + solve + fusion + sw_append_frame per frame, wall clock, on the model cut by "
                        "30%; steady frames after the first two"}
    appending = {"steady": appends[1:], "model_cut_30pct": cut_st, "model_and_nodes_cut_30pct": ext_st,
                 "pipeline": pipeline,
                 "note": "kernel_ms: device time of the appending kernels (events); rebuild_ms: host-side "
                         "model rebuild (set sort, JtJ pattern, runner); call_ms: the whole call"}
    batched = run_batched(sw, torch, members[:args.batch_streams], args.batch_rounds, 2, flush, stream) \
        if members and args.batch_streams > 0 else None
    served = run_served_sweep(sw, members, large, args, gn, pcg) if members and args.served_streams > 0 else None

    if rank != 0:
        return
    line = {
        "metric": METRIC, "value": job_frames_per_s(ms, world), "unit": "frames/s", "n_gpus": world,
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
        # kernels of this library per step: depth (frame id + maps), solve
        # (stats reset, system clear, 3 per Gauss-Newton iteration: the
        # assembly of both terms, preconditioner, PCG), fusion (3)
        "gpu_launches": args.steps * (2 + 2 + 3 * gn + 3),
        "roofline": roof["dominant"],
        "stages_ms_per_step": {k: v / prof_steps for k, v in stage_ms.items()},
        "stage_roofline": roof["stages"],
        "autotune": {"pcg_rows_per_cta": tuned_rows, "pcg_us_per_launch": tuned_us},
        "rigid_align": rigid,
        "appending": appending,
        "visibility": visibility,
        "precision_f64dots": precision_f64dots,
        "pcg_mode": pcg_mode,
    }
    if batched:
        line["multi_stream"] = batched
    if served:
        line["served"] = served
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_sample()
    print(json.dumps(line))


if __name__ == "__main__":
    main()
