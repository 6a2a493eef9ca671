"""Benchmark of the visibility-bitmask gather on GB300.

Default workload: the 4K precision form (3840x2160, FP32 depth + FP16 normal and
radiance, 4 slices, 32 steps per side, N_b = 32, 4 ambient cones against a seeded
3-band SH environment, R = 2 m, t = 0.5 m) on a seeded procedural scene.
One step = one gather over one frame.  Metric: Gsamples/s (2 N_d N_s samples per
pixel, all pixels) and ms/frame.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--workload 4k|1080p|256] [--nb 32|64]

Under torchrun (N > 1) every rank gathers its own frames (independent replicas,
no collective on the data path); value = all ranks' samples / max-over-ranks time.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import scenegen  # noqa: E402


def _jsonable(o):
    """numpy scalars in the result line as plain numbers."""
    if isinstance(o, np.integer):
        return int(o)
    if isinstance(o, np.floating):
        return float(o)
    if isinstance(o, np.bool_):
        return bool(o)
    raise TypeError(f"not JSON serializable: {type(o).__name__}")

SM_COUNT_GB300 = 152
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ssilvb", choices=["ssilvb", "reference"])
    ap.add_argument("--workload", default="4k",
                    choices=["4k", "1080p", "256", "batch", "serve", "trends", "issue_peak"])
    ap.add_argument("--serve-seconds", type=float, default=2.0)
    ap.add_argument("--nb", type=int, default=32)
    ap.add_argument("--radius", type=float, default=None, help="override the workload's radius R (m)")
    ap.add_argument("--ns", type=int, default=None, help="override the workload's steps per side")
    ap.add_argument("--nd", type=int, default=None, help="override the workload's slices per pixel")
    ap.add_argument("--no-gi", action="store_true", help="override: AO and ambient only (no indirect-light fetches)")
    ap.add_argument("--planar", action="store_true",
                    help="FP16 normal and radiance as two F16X4 planes instead of one interleaved F16X8 plane")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the other sector counts, the batch and the serving measurements")
    return ap.parse_args()


def make_workload(name, nb, radius=None, ns=None, nd=None, gi=None):
    """The named workload, with optional overrides of R, N_s and N_d (profiling the shapes of the
    paper's Table 1 and 2 on the same scenes); an override is named in the workload string."""
    import dataclasses
    if name == "4k":
        w = scenegen.workload_4k(sector_count=nb)
    elif name == "1080p":
        w = scenegen.workload_1080p()
    else:
        w = scenegen.workload_256()
    over = {k: v for k, v in (("radius", radius), ("steps_per_side", ns), ("num_slices", nd), ("gi", gi))
            if v is not None}
    if over:
        w = dataclasses.replace(w, params=dataclasses.replace(w.params, **over),
                                name=w.name + " " + " ".join(f"{k}={v}" for k, v in over.items()))
    return w


KERNEL_SOURCES = ["gather_kernel.cuh", "launch_impl.cuh", "launch_nb32.cu", "launch_nb64.cu", "launch_nb128.cu",
                  "internal.h"]  # internal.h: the default launch choice (blocks per SM)


def kernel_sources_sha256():
    """Hash of the device code (the kernel, its instantiating units and the default launch
    choice) and the nvcc flags: measured DRAM counters apply only to this code; other host-side
    changes leave them valid."""
    import hashlib

    import paper_2301_11376_gb300 as ssilvb
    h = hashlib.sha256(" ".join(ssilvb.NVCC_FLAGS).encode())
    csrc = os.path.join(ROOT, "paper_2301_11376_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()


def measured_traffic(key):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the ncu capture
    recorded in profiles/traffic.json, or None when the kernel sources changed since."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            rec = json.load(f).get(key)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("sources_sha256") != kernel_sources_sha256():
        return None
    return rec.get("dram_bytes_per_launch")


def samples_per_frame(w):
    H, W = w.gbuf.depth.shape
    return H * W * 2 * w.params.num_slices * w.params.steps_per_side


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm = [float(r[1]) for r in self.rows if len(r) >= 9 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) >= 9 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows if len(r) >= 9 for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(sm)}


def algorithmic_ops_per_frame(w):
    """Algorithmic lane-ops of one frame of workload w: the binary32 replica's op count (one per IEEE
    add/mul/fma/div/sqrt, compare, select, conversion, shift, logic op, popcount) on a uniform pixel
    sample scaled to the frame, frozen in profiles/opcounts.json by `python -m oracle.freeze_opcounts`
    (a CPU test keeps it current).  (None, None) for a workload the table does not hold."""
    try:
        with open(os.path.join(ROOT, "profiles", "opcounts.json")) as f:
            rec = json.load(f).get(w.name)
    except (OSError, ValueError):
        rec = None
    if rec is None:
        return None, None
    return rec["ops_per_frame"], rec["counts_per_frame"]


def cpu_model():
    """The host CPU's model string (lscpu, else /proc/cpuinfo, else the machine name)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model Name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def _time_cpu_program(prob, program, H, W, per_px, threads, target_s, rng):
    """Gsamples/s of one CPU program (the FP64 oracle or the binary32 replica, as they stand) on
    `threads` threads: a short calibration, then one run on a uniform pixel sample sized to take
    about target_s."""
    import oracle
    oracle.threads(threads)
    run = (lambda xy: oracle.fp64(prob, xy)) if program == "fp64" else (lambda xy: oracle.fp32(prob, xy))
    n = 64 * threads
    while True:
        idx = rng.choice(H * W, size=min(n, H * W), replace=False)
        xy = np.stack([idx % W, idx // W], 1).astype(np.int32)
        t0 = time.perf_counter()
        res = run(xy)
        dt = time.perf_counter() - t0
        if dt >= 0.25 * target_s or n >= H * W:
            break
        n = min(H * W, max(2 * n, int(n * target_s / max(dt, 1e-3))))
    return {"program": "FP64 oracle" if program == "fp64" else "binary32 replica", "threads": threads,
            "value": len(idx) * per_px / dt / 1e9, "unit": "Gsamples/s", "pixels": int(len(idx)),
            "samples": int(len(idx) * per_px), "seconds": dt,
            "ms_per_frame_extrapolated": dt / len(idx) * H * W * 1e3}, idx, res


def _accuracy(gpu, idx, res, fp64):
    """The GPU's outputs on the pixels a timed CPU run evaluated: largest and mean absolute
    difference over AO, GI and ambient, and the share of pixels whose largest difference exceeds
    1e-4 (against the free-running FP64 oracle, decisions within rounding of a boundary may move a
    sector between samples; the tests gate every pixel against FP64 on the binary32 decisions)."""
    g0, g1 = gpu
    d = np.abs(g0[idx].astype(np.float64) - res[0])
    if g1 is not None:
        d = np.concatenate([d[:, :4], np.abs(g1[idx].astype(np.float64) - res[1])[:, :3]], axis=1)
    worst = d.max(axis=1)
    return {"against": "FP64 oracle (free-running)" if fp64 else "binary32 replica", "pixels": int(len(idx)),
            "max_abs": float(worst.max()), "mean_abs": float(d.mean()),
            "share_above_1e-4": float((worst > 1e-4).mean())}


def cpu_baseline(w, target_s=6.0, gpu=None):
    """Both CPU programs of the oracle, as they stand, on the host cores: the FP64 oracle and the
    binary32 replica, each on 1 thread and on every core (OpenMP over pixels), on bounded uniform
    pixel samples of the workload.  value = the FP64 oracle on every core.  gpu: optional host
    copies (out0, out1) of the GPU's outputs for the same workload, compared with the all-core
    runs' outputs on their pixels."""
    import oracle
    H, W = w.gbuf.depth.shape
    prob = oracle.Problem(w.gbuf, w.params, w.noise, w.sh)
    per_px = 2 * w.params.num_slices * w.params.steps_per_side
    cores = os.cpu_count() or 1
    default_threads = oracle.threads()
    rng = np.random.default_rng(7)
    runs, accuracy = [], []
    try:
        for program in ("fp64", "fp32"):
            for threads in sorted({1, cores}):
                r, idx, res = _time_cpu_program(prob, program, H, W, per_px, threads, target_s, rng)
                runs.append(r)
                if gpu is not None and threads == cores:
                    accuracy.append(_accuracy(gpu, idx, res, program == "fp64"))
    finally:
        oracle.threads(default_threads)
    head = [r for r in runs if r["program"] == "FP64 oracle" and r["threads"] == cores][0]
    out = {"value": head["value"], "unit": "Gsamples/s", "cores": cores, "kind": "oracle",
           "sample": f"FP64 oracle on {cores} threads, {head['pixels']} uniformly drawn pixels of the {W}x{H} frame "
                     f"({head['samples']} samples, {head['seconds']:.1f} s); every run below on its own sample",
           "cpu_model": cpu_model(), "nproc": cores, "runs": runs}
    if accuracy:
        out["gpu_accuracy_on_these_pixels"] = accuracy
    return out


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v):
    if world <= 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def line_config(w, world):
    """The `config` of the result line for a single-frame workload (shared by both arms)."""
    return {"workload": w.name, "samples_per_frame": samples_per_frame(w),
            "l2": "flushed (256 MB write) between timed steps",
            "storage": "f32 depth, f16 normal+radiance" if w.gbuf.normal.dtype == np.float16 else "f32",
            "parallelism": f"replicas x{world}"}


def run_reference(args, world, rank):
    """Reference arm: the CPU oracle (FP64, as it stands) on every host core.  Each step is a bounded
    uniform pixel sample of the workload; ms_per_step is that step's measured time, and the line
    states the per-frame time extrapolated from it (the only other place this file runs the
    oracle)."""
    if rank != 0:
        return
    w = make_workload(args.workload, args.nb, args.radius, args.ns, args.nd, False if args.no_gi else None)
    import oracle
    H, W = w.gbuf.depth.shape
    prob = oracle.Problem(w.gbuf, w.params, w.noise, w.sh)
    per_px = 2 * w.params.num_slices * w.params.steps_per_side
    cores = oracle.threads()
    n = min(H * W, 4096 * cores)  # pixels per step: a bounded sample so the whole run takes seconds
    rng = np.random.default_rng(11)
    times = []
    for s in range(args.warmup + args.steps):
        idx = rng.choice(H * W, size=n, replace=False)
        xy = np.stack([idx % W, idx // W], 1).astype(np.int32)
        t0 = time.perf_counter()
        oracle.fp64(prob, xy)
        dt = time.perf_counter() - t0
        if s >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = args.steps * n * per_px / total / 1e9
    out = {"impl": "reference", "metric": "Gsamples/s (ms/frame at 4K)", "value": value, "unit": "Gsamples/s",
           "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": line_config(w, args.gpus),
           "sampled": {"pixels_per_step": n, "pixels_per_frame": H * W,
                       "ms_per_frame_extrapolated": total / args.steps * (H * W / n) * 1e3,
                       "note": "a step is a uniform sample of the frame's pixels; value is samples per second"},
           "cpu_baseline": {"value": value, "unit": "Gsamples/s", "cores": cores, "kind": "oracle",
                            "sample": f"FP64 oracle, {cores} threads, {n} random pixels per step of the {W}x{H} frame",
                            "cpu_model": cpu_model()},
           "e2e": {"value": value, "unit": "Gsamples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out, default=_jsonable))


def batch_workload(n_frames=64, base_seed=1000, sizes=None):
    """64 seeded frames of uneven sizes (640x360 .. 2560x1440, or `sizes`), per-frame N_d 1-4, N_s
    8-32, t 0.1-1.0 m; 64 spheres + 16 panels, FP32 storage, N_b 32, R 2 m, 4x4 IGN noise."""
    out = []
    for seed, W, H, nd, ns, t in scenegen.batch_recipe(n_frames, base_seed, sizes):
        g = scenegen.render(seed, W, H, 64, 16)
        out.append((g, scenegen.Params(nd, ns, 2.0, t)))
    return out


def batch_measure(ctx, dev, steps, warmup, base_seed=1000, world=1, sizes=None):
    """The 64-frame uneven batch (640x360..2560x1440, per-frame N_d 1-4, N_s 8-32, t 0.1-1 m, FP32,
    N_b 32) through ssilvb_gather_batch in its two forms (one persistent kernel over a tile queue
    launched through a CUDA graph; one graph of per-frame kernels) and as the autotuner picks, against
    the plain per-frame launch with and without a host synchronisation per frame.  CUDA events on the
    launching stream, L2 flushed between timed steps."""
    import torch
    frames_np = batch_workload(64, base_seed, sizes)
    noise = scenegen.ign_table()
    stream = torch.cuda.current_stream(dev)
    frames, keep, hold = [], None, []
    samples = 0
    for g, prm in frames_np:
        H, W = g.depth.shape
        d = torch.from_numpy(g.depth).to(dev)
        n = torch.from_numpy(g.normal).to(dev)
        r = torch.from_numpy(g.radiance).to(dev)
        o0, _, _ = ssilvb_mod().alloc_outputs(H, W, prm, dev)
        f, keep = ctx.frame(d, n, r, g.camera, prm, o0, None, None, noise=noise, keep=keep)
        frames.append(f)
        hold.append((d, n, r, o0, g, prm))
        samples += H * W * 2 * prm.num_slices * prm.steps_per_side
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    tuned = ctx.autotune(frames, stream)

    def timed(fn, k):
        ts = []
        for i in range(k):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return ts

    def batched(mode):
        def fn():
            ctx.set_tuning(batch_mode=mode)
            ctx.gather_batch(frames, stream)
        return fn

    def plain_nosync():
        for d, n, r, o0, g, prm in hold:
            ctx.gather(d, n, r, g.camera, prm, o0, None, None, noise=noise, stream=stream)

    def plain_sync():
        for d, n, r, o0, g, prm in hold:
            ctx.gather(d, n, r, g.camera, prm, o0, None, None, noise=noise, stream=stream)
            stream.synchronize()

    forms = {"autotuned": batched(0), "persistent_graph": batched(1), "graph_of_frame_kernels": batched(2),
             "plain_no_sync": plain_nosync, "plain_host_sync": plain_sync}
    for fn in forms.values():
        timed(fn, warmup)
    res = {name: timed(fn, steps) for name, fn in forms.items()}
    ctx.set_tuning()
    med = {name: statistics.median(v) for name, v in res.items()}
    sz = scenegen.BATCH_SIZES if sizes is None else sizes
    out = {"workload": f"batch of 64 uneven frames ({sz[0][0]}x{sz[0][1]}..{sz[-1][0]}x{sz[-1][1]}), N_d 1-4, "
                       "N_s 8-32, t 0.1-1.0 m, fp32, nb32",
           "samples_per_batch": samples, "steps": steps, "warmup": warmup,
           "l2": "flushed (256 MB write) between timed steps",
           "tuning": {"occupancy": tuned.occupancy, "rows_per_tile": tuned.rows_per_tile,
                      "use_graph": tuned.use_graph, "batch_mode": tuned.batch_mode,
                      "block_order": tuned.block_order},
           "accuracy": "each frame bit-identical to its single-frame gather; masks bit-exact against the binary32 "
                       "replica and outputs within 1e-4 of FP64 (tests/test_gpu_batch.py)"}
    for name, m in med.items():
        out[name] = {"ms_per_batch": m, "frames_per_s": 64 * world / (m / 1e3),
                     "gsamples_per_s": world * samples / (m / 1e3) / 1e9}
    out["speedup_vs_plain_no_sync"] = med["plain_no_sync"] / med["autotuned"]
    out["speedup_vs_plain_host_sync"] = med["plain_host_sync"] / med["autotuned"]
    out["timed_sum_ms"] = {name: sum(v) for name, v in res.items()}
    return out


def ssilvb_mod():
    import paper_2301_11376_gb300 as ssilvb
    return ssilvb


def run_batch_bench(args, world, rank, local):
    import torch
    ssilvb = ssilvb_mod()
    ssilvb.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctx = ssilvb.Context(local)
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    res = batch_measure(ctx, dev, args.steps, args.warmup, 1000 + 64 * rank, world)
    barrier(world)
    clk = clocks.stop()
    t_dev = max_over_ranks(world, res["autotuned"]["ms_per_batch"] / 1e3)
    if rank != 0:
        return
    out = {"metric": "Gsamples/s (batched frames/s vs plain per-frame launch)",
           "value": world * res["samples_per_batch"] / t_dev / 1e9, "unit": "Gsamples/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_dev * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": res["workload"], "l2": res["l2"]}, "batch": res, "clocks": clk,
           "gpu_launches": args.steps}
    print(json.dumps(out, default=_jsonable))


def run_trend_sweep(args, world, rank, local):
    """Sweeps shaped like the paper's Table 1 (AO only, 1080p, one slice per pixel, N_b 32:
    radius/steps pairs, bitmask t = 0.5 m vs infinite thickness = horizon mode; plus N_b 128)
    and Table 2 (indirect diffuse, t = 0.2 m, constant vs quadratic steps, half resolution).
    Reproduces trends only; the paper's numbers are from an RTX 2080 on another scene."""
    import torch

    import paper_2301_11376_gb300 as ssilvb
    ssilvb.build()
    if rank != 0:
        return
    dev = torch.device("cuda", local)
    ctx = ssilvb.Context(local)
    noise = scenegen.ign_table()
    full = scenegen.render(2, 1920, 1080, 64, 16)
    half = scenegen.render(2, 960, 540, 64, 16)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def dev_gb(g):
        return tuple(torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in (g.depth, g.normal, g.radiance))

    gbs = {"full": (full, dev_gb(full)), "half": (half, dev_gb(half))}

    def time_one(res, prm, reps=12):
        g, (d, n, r) = gbs[res]
        H, W = g.depth.shape
        o0, _, _ = ssilvb.alloc_outputs(H, W, prm, dev)
        ts = []
        for i in range(reps):
            flush.fill_(float(i))
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            ctx.gather(d, n, r, g.camera, prm, o0, None, None, noise=noise)
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts[3:])

    rows = []
    for radius, ns, paper_gtao, paper_bm in [(0.8, 8, 0.49, 0.51), (1.0, 12, 0.75, 0.77), (1.0, 16, 0.95, 0.97),
                                            (2.0, 16, 1.12, 1.13), (3.0, 16, 1.12, 1.13)]:
        row = {"table": 1, "radius": radius, "steps_per_side": ns}
        for name, t, nb in [("horizon_t_inf", math.inf, 32), ("bitmask_nb32", 0.5, 32), ("bitmask_nb128", 0.5, 128)]:
            prm = scenegen.Params(1, ns, radius, t, sector_count=nb, gi=False)
            row[name + "_ms"] = time_one("full", prm)
        row["paper_rtx2080_ms"] = {"gtao": paper_gtao, "bitmask": paper_bm}
        rows.append(row)
    for label, ns, radius, mode, res, paper in [("a", 8, 1.0, 0, "full", 0.9), ("b", 8, 4.0, 0, "full", 1.7),
                                                ("c", 16, 4.0, 0, "full", 2.3), ("d", 16, 4.0, 1, "full", 2.6),
                                                ("e", 32, 4.0, 1, "full", 4.0), ("f", 16, 4.0, 1, "half", 0.97)]:
        prm = scenegen.Params(1, ns, radius, 0.2, step_mode=mode)
        rows.append({"table": 2, "config": label, "steps_per_side": ns, "radius": radius,
                     "steps": "quadratic" if mode else "constant", "resolution": res,
                     "ms": time_one(res, prm), "paper_rtx2080_sampling_ms": paper})
    out = {"metric": "trend sweep (ms per 1080p frame)", "value": rows[2]["bitmask_nb32_ms"], "unit": "ms",
           "higher_is_better": False, "n_gpus": 1, "data": "synthetic",
           "config": {"workload": "1920x1080 seed 2, 64 spheres + 16 panels, fp32, N_d 1 with 4x4 IGN rotation",
                      "l2": "flushed between timed runs"}, "rows": rows}
    print(json.dumps(out, default=_jsonable))


def serve_pool(dev, rank=0):
    """Resident G-buffers of the serving stream: 2 seeded scenes per size, 1280x720 .. 3840x2160."""
    from paper_2301_11376_gb300 import serve
    pool = serve.ResidentPool(dev)
    keys = []
    for si, (W, H) in enumerate(scenegen.SERVE_SIZES):
        for k in range(2):
            seed = 2_000_000 + 16 * si + k + 1000 * rank
            pool.add((W, H, k), scenegen.render(seed, W, H, 64, 16))
            keys.append((W, H, k))
    return pool, keys


def serve_measure(ctx, pool, keys, seconds, rate_sps, budget_ms=50.0, batch_ms=4.0, rank=0):
    """The Poisson serving stream (mean 2000 req/s; 720p-4K, N_d 1-8, N_b 32/64, N_s 8/16/32) and the
    same recipe below capacity (300 req/s), each through the continuous-batching server and through
    the plain per-frame launch with a host synchronisation per request, both under the same
    latency-aware admission (budget_ms) and the same host-side completion clock."""
    from paper_2301_11376_gb300 import serve
    warm = serve.poisson_requests(5, 48, 1e-5, keys, None)
    serve.Server(ctx, pool, arena_bytes=4 << 30).run(warm)
    serve.PlainServer(ctx, pool).run(warm[:8])
    out = {"workload": "Poisson arrivals, frames 1280x720..3840x2160 (2 resident scenes per size), N_d 1-8, "
                       "N_b 32/64, N_s 8/16/32, fp32, R 2 m, t 0.5 m, 4x4 IGN noise",
           "budget_ms": budget_ms, "batch_span_ms": batch_ms,
           "admission": "shed at arrival when the predicted FIFO latency (plus the batch span for the batching "
                        "server) exceeds the budget (serve.LatencyAdmission)",
           "clock": "host time when the completion is first observed, both servers",
           "accuracy": "every served result bit-identical to the same request alone, outputs within 1e-4 of FP64 "
                       "(tests/test_gpu_serve.py)"}
    for label, rps, seed in (("load_2000_req_per_s", 2000.0, 77), ("load_300_req_per_s", 300.0, 91)):
        reqs = serve.poisson_requests(seed + rank, int(seconds * rps), 1.0 / rps, keys, None)
        a = serve.Server(ctx, pool, arena_bytes=4 << 30, max_inflight=4, max_batch=16, budget_ms=budget_ms,
                         rate=rate_sps, batch_ms=batch_ms).run(reqs).summary()
        b = serve.PlainServer(ctx, pool, budget_ms=budget_ms, rate=rate_sps).run(reqs).summary()
        out[label] = {"requests": len(reqs), "server": a, "plain_per_frame_launch": b,
                      "goodput_ratio": a["goodput_frames_per_s"] / max(b["goodput_frames_per_s"], 1e-9),
                      "goodput_samples_ratio": a["goodput_gsamples_per_s"] / max(b["goodput_gsamples_per_s"], 1e-9),
                      "frames_per_s_ratio": a["frames_per_s"] / max(b["frames_per_s"], 1e-9)}
    return out


def run_serve_bench(args, world, rank, local):
    import torch
    ssilvb = ssilvb_mod()
    ssilvb.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ctx = ssilvb.Context(local)
    pool, keys = serve_pool(dev, rank)
    clocks = Clocks(local)
    clocks.start()
    barrier(world)
    res = serve_measure(ctx, pool, keys, args.serve_seconds, 4.5e11, rank=rank)
    barrier(world)
    clk = clocks.stop()
    fps = max_over_ranks(world, -res["load_2000_req_per_s"]["server"]["goodput_frames_per_s"])  # slowest rank
    if rank != 0:
        return
    out = {"metric": "served frames/s within the latency budget and p99 latency vs plain per-frame launch",
           "value": -fps * world, "unit": "frames/s", "n_gpus": world, "steps": 1, "warmup": 1,
           "ms_per_step": res["load_2000_req_per_s"]["server"]["wall_s"] * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": res["workload"], "budget_ms": res["budget_ms"]}, "serve": res, "clocks": clk,
           "gpu_launches": res["load_2000_req_per_s"]["server"]["batches"]}
    print(json.dumps(out, default=_jsonable))

# Issue-rate probe: the denominators of the ALU roofline measured on this GPU (scalar FP32 FMA,
# packed f32x2 FMA, integer ops), each from 8 independent chains per thread on 8 blocks of 256
# threads per SM.  Nothing here touches the gather.
ISSUE_PROBE_CU = r"""
#include <cstdio>
#include <cuda_runtime.h>
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
    float2 d;
    asm volatile("{.reg .b64 ra, rb, rc, rd;\n\tmov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
                 "mov.b64 rc, {%6, %7};\n\tfma.rn.f32x2 rd, ra, rb, rc;\n\tmov.b64 {%0, %1}, rd;}"
                 : "=f"(d.x), "=f"(d.y) : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y), "f"(c.x), "f"(c.y));
    return d;
}
__global__ void k_ffma(float *out, int n, float m) {
    float a[8];
    for (int i = 0; i < 8; ++i) a[i] = threadIdx.x * 1e-3f + i;
    for (int it = 0; it < n; ++it)
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = fmaf(a[i], m, 0.5f);
    float s = 0; for (int i = 0; i < 8; ++i) s += a[i];
    if (s == 12345.0f) out[0] = s;
}
__global__ void k_ffma2(float *out, int n, float m) {
    float2 a[8];
    for (int i = 0; i < 8; ++i) a[i] = make_float2(threadIdx.x * 1e-3f + i, i * 0.5f);
    const float2 mm = make_float2(m, m), h = make_float2(0.5f, 0.25f);
    for (int it = 0; it < n; ++it)
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = pfma(a[i], mm, h);
    float s = 0; for (int i = 0; i < 8; ++i) s += a[i].x + a[i].y;
    if (s == 12345.0f) out[0] = s;
}
__global__ void k_int(int *out, int n, int m) {
    int a[8];
    for (int i = 0; i < 8; ++i) a[i] = threadIdx.x + i;
    for (int it = 0; it < n; ++it)
#pragma unroll
        for (int i = 0; i < 8; ++i) a[i] = (a[i] ^ m) + i;
    int s = 0; for (int i = 0; i < 8; ++i) s += a[i];
    if (s == 12345) out[0] = s;
}
int main() {
    int sms; cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, 0);
    float *out; if (cudaMalloc(&out, 16) != cudaSuccess) return 1;
    const int n = 1 << 14, blocks = sms * 8, threads = 256;
    const double elems = (double)blocks * threads * n * 8;
    cudaEvent_t e0, e1; cudaEventCreate(&e0); cudaEventCreate(&e1);
    float t[3] = {0, 0, 0};
    for (int rep = 0; rep < 2; ++rep) {  // the first pass warms the clocks up
        cudaEventRecord(e0); k_ffma<<<blocks, threads>>>(out, n, 0.999f); cudaEventRecord(e1); cudaEventSynchronize(e1);
        cudaEventElapsedTime(&t[0], e0, e1);
        cudaEventRecord(e0); k_ffma2<<<blocks, threads>>>(out, n, 0.999f); cudaEventRecord(e1); cudaEventSynchronize(e1);
        cudaEventElapsedTime(&t[1], e0, e1);
        cudaEventRecord(e0); k_int<<<blocks, threads>>>((int *)out, n, 7); cudaEventRecord(e1); cudaEventSynchronize(e1);
        cudaEventElapsedTime(&t[2], e0, e1);
    }
    printf("%d %.6f %.6f %.6f %.1f\n", sms, t[0], t[1], t[2], elems);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}
"""


def run_issue_peak(args, world, rank, local):
    """ALU roofline denominators measured here, beside the derived peak the roofline uses."""
    if rank != 0:
        return
    import subprocess
    import tempfile
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "issue_probe.cu"), os.path.join(d, "issue_probe")
        with open(src, "w") as f:
            f.write(ISSUE_PROBE_CU)
        subprocess.run(["nvcc", "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe, src], check=True)
        clocks = Clocks(local)
        clocks.start()
        r = subprocess.run([exe], check=True, capture_output=True, text=True)
        clk = clocks.stop()
    sms, t_ffma, t_ffma2, t_int, elems = r.stdout.split()
    sms, elems = int(sms), float(elems)
    derived = sms * FP32_LANES_PER_SM * 2.070e9 / 1e12
    out = {"metric": "ALU issue-rate probe (roofline denominators)", "unit": "T lane-ops/s", "n_gpus": 1,
           "derived_peak": derived, "derived_note": f"{sms} SMs x 128 lanes x 2.070 GHz",
           "ffma_fp32_ops": elems / float(t_ffma) / 1e9,
           "ffma2_instructions": elems / float(t_ffma2) / 1e9, "ffma2_fp32_ops": 2 * elems / float(t_ffma2) / 1e9,
           "int_xor_add_ops": 2 * elems / float(t_int) / 1e9, "clocks": clk}
    out["value"] = out["ffma_fp32_ops"]
    print(json.dumps(out, default=_jsonable))


def main():
    args = parse()
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    if args.workload == "batch":
        run_batch_bench(args, world, rank, local)
        return
    if args.workload == "serve":
        run_serve_bench(args, world, rank, local)
        return
    if args.workload == "trends":
        run_trend_sweep(args, world, rank, local)
        return
    if args.workload == "issue_peak":
        run_issue_peak(args, world, rank, local)
        return
    import torch

    import paper_2301_11376_gb300 as ssilvb
    ssilvb.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    w = make_workload(args.workload, args.nb, args.radius, args.ns, args.nd, False if args.no_gi else None)
    H, W = w.gbuf.depth.shape
    spf = samples_per_frame(w)
    g = w.gbuf
    d = torch.from_numpy(g.depth).to(dev)
    # FP16 storage: by default one interleaved plane (F16X8: a sample's normal and radiance in one
    # 16-byte record, the same bytes per pixel as two F16X4 planes); --planar: the two planes
    interleaved = g.normal.dtype == np.float16 and not args.planar
    n_host = g.interleaved_f16() if interleaved else np.ascontiguousarray(g.normal)
    r_host = None if interleaved else np.ascontiguousarray(g.radiance)
    n = torch.from_numpy(n_host).to(dev)
    r = torch.from_numpy(r_host).to(dev) if r_host is not None else None
    out0, out1, _ = ssilvb.alloc_outputs(H, W, w.params, dev)
    ctx = ssilvb.Context(local)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2

    def step():
        ctx.gather(d, n, r, g.camera, w.params, out0, out1, None, noise=w.noise, sh=w.sh, stream=stream)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    ctx.synchronize(stream)
    torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = Clocks(local)
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        flush.fill_(float(i))  # evict the G-buffer from L2 between timed steps (outside the events)
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - wall0
    clk = clocks.stop()
    ctx.synchronize(stream)
    kern_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    # the same gather with the L2 left warm between steps (reported beside the L2-flushed headline)
    warm_ms = []
    for i in range(3 + min(args.steps, 10)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        torch.cuda.synchronize()
        if i >= 3:
            warm_ms.append(a.elapsed_time(b))
    gpu_host = None
    if not args.no_cpu_baseline and rank == 0:  # this workload's outputs, compared on the CPU baseline's pixels
        gpu_host = (out0.cpu().numpy().reshape(-1, 4), out1.cpu().numpy().reshape(-1, 4) if out1 is not None else None)
    t_dev = sum(kern_ms) / 1e3
    t_max = max_over_ranks(world, t_dev)
    value = world * args.steps * spf / t_max / 1e9
    ms = t_max / args.steps * 1e3

    # e2e: the same gather through the host-buffer entry point (copies inside the timed region)
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hd, hn = pin(g.depth), pin(n_host)
        hr = pin(r_host) if r_host is not None else None
        ho0 = torch.empty((H, W, 4), dtype=torch.float32).pin_memory()
        ho1 = torch.empty((H, W, 4), dtype=torch.float32).pin_memory() if out1 is not None else None
        # a stream of frames through the pipelined host-buffer call (one frame's copies overlap the
        # next frame's gather); every step still copies its inputs in and its outputs back
        outs = [(ho0, ho1), (torch.empty_like(ho0).pin_memory(),
                             torch.empty_like(ho1).pin_memory() if ho1 is not None else None)]
        # warm-up: the staging of the synchronous lane, then W frames through both pipelined lanes
        ctx.gather_host(hd, hn, hr, g.camera, w.params, ho0, ho1, None, noise=w.noise, sh=w.sh, stream=stream)
        for i in range(max(2, args.warmup)):
            ctx.gather_host(hd, hn, hr, g.camera, w.params, *outs[i % 2], None, noise=w.noise, sh=w.sh, stream=stream,
                            asynchronous=True)
        ctx.synchronize(stream)
        ke = max(3, args.steps)  # the same number of frames as the device-timed region
        barrier(world)
        t0 = time.perf_counter()
        for i in range(ke):  # frames in flight together write different output buffers
            o0, o1 = outs[i % 2]
            ctx.gather_host(hd, hn, hr, g.camera, w.params, o0, o1, None, noise=w.noise, sh=w.sh, stream=stream,
                            asynchronous=True)
        ctx.synchronize(stream)
        te = max_over_ranks(world, time.perf_counter() - t0)
        # the same frames one synchronous call at a time (each returns with its outputs on the host)
        t0 = time.perf_counter()
        for _ in range(ke):
            ctx.gather_host(hd, hn, hr, g.camera, w.params, ho0, ho1, None, noise=w.noise, sh=w.sh, stream=stream)
        ts = max_over_ranks(world, time.perf_counter() - t0)
        h2d = hd.numel() * 4 + hn.numel() * hn.element_size() + (hr.numel() * hr.element_size() if hr is not None else 0)
        d2h = ho0.numel() * 4 + (ho1.numel() * 4 if ho1 is not None else 0)
        e2e = {"value": world * ke * spf / te / 1e9, "unit": "Gsamples/s", "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "ms_per_step": te / ke * 1e3,
               "api": "ssilvb_gather_host_async x steps, then ssilvb_synchronize",
               "synchronous_call": {"value": world * ke * spf / ts / 1e9, "ms_per_step": ts / ke * 1e3}}

    # The rest of the metric at N = 1: the 4K workload at its other sector counts, the uneven batch
    # against the plain per-frame launch, and the serving stream against the plain per-frame launch.
    extras = None
    if world == 1 and not args.no_extras and args.workload == "4k":
        extras = {}
        xclk = Clocks(local)
        xclk.start()
        extras["sector_counts"] = {}
        for nb in (64, 128):
            prm = scenegen.Params(w.params.num_slices, w.params.steps_per_side, w.params.radius, w.params.thickness,
                                  sector_count=nb, ambient_cones=w.params.ambient_cones)
            ts = []
            for i in range(args.warmup + min(args.steps, 10)):
                flush.fill_(float(i))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.gather(d, n, r, g.camera, prm, out0, out1, None, noise=w.noise, sh=w.sh, stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                if i >= args.warmup:
                    ts.append(a.elapsed_time(b))
            wn = scenegen.Workload(w.name.replace("nb32", f"nb{nb}"), g, prm, w.noise, w.sh)
            ops_nb, _ = algorithmic_ops_per_frame(wn)
            m = statistics.median(ts)
            extras["sector_counts"][f"nb{nb}"] = {
                "ms_per_frame": m, "gsamples_per_s": spf / (m / 1e3) / 1e9, "steps": len(ts),
                "roofline_frac": (ops_nb / (m / 1e3) / (SM_COUNT_GB300 * FP32_LANES_PER_SM * 2.070e9)
                                  if ops_nb is not None else None),
                "ops_per_frame": ops_nb,
                "accuracy": "masks bit-exact against the binary32 replica on the whole frame "
                            "(tests/test_gpu_parity.py)"}
        if g.normal.dtype == np.float16:
            # the same workload with the other FP16 layout, for comparison (same results bit for bit)
            other = (torch.from_numpy(np.ascontiguousarray(g.normal)).to(dev),
                     torch.from_numpy(np.ascontiguousarray(g.radiance)).to(dev)) if interleaved else \
                (torch.from_numpy(g.interleaved_f16()).to(dev), None)
            ts = []
            for i in range(args.warmup + min(args.steps, 10)):
                flush.fill_(float(i))
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                ctx.gather(d, other[0], other[1], g.camera, w.params, out0, out1, None, noise=w.noise, sh=w.sh,
                           stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                if i >= args.warmup:
                    ts.append(a.elapsed_time(b))
            del other
            extras["storage_layouts"] = {
                "f16x8_interleaved_ms": ms if interleaved else statistics.median(ts),
                "f16x4_planar_ms": statistics.median(ts) if interleaved else ms,
                "note": "FP16 normal and radiance as one interleaved plane (a sample's normal and radiance in one "
                        "16-byte record) or two planes; the same values, bit-identical results"}
        extras["batch"] = batch_measure(ctx, dev, min(args.steps, 10), max(3, min(args.warmup, 5)))
        # outside the workload configs, for the regime: frames too small to fill the GPU, where
        # per-launch overhead and host round trips dominate and one batch call pays
        extras["batch"]["small_frames_outside_configs"] = batch_measure(
            ctx, dev, min(args.steps, 10), max(3, min(args.warmup, 5)), sizes=scenegen.SMALL_BATCH_SIZES)
        pool, keys = serve_pool(dev)
        extras["serve"] = serve_measure(ctx, pool, keys, args.serve_seconds, value * 1e9)
        extras["clocks"] = xclk.stop()
    if rank != 0:
        return
    ops, counts = algorithmic_ops_per_frame(w)
    peak_ops = SM_COUNT_GB300 * FP32_LANES_PER_SM * 2.070e9
    achieved = ops / (ms / 1e3) if ops is not None else None
    roof = {"bound": "alu", "achieved": achieved / 1e12 if ops is not None else None, "peak": peak_ops / 1e12,
            "unit": "Tops/s", "frac": achieved / peak_ops if ops is not None else None,
            "traffic": (measured_traffic(f"{args.workload} nb{args.nb}")
                        if args.radius is None and args.ns is None and args.nd is None and not args.no_gi
                        and not args.planar else None),
            "traffic_unit": "bytes per launch (ncu dram read + write)",
            "algorithmic_bytes": int(H * W * (4 + 2 * g.normal.dtype.itemsize * 4 + 16 + (16 if out1 is not None else 0))),
            "kernel": "gather_class_kernel", "ops_per_launch": ops,
            "ops_per_sample": ops / spf if ops is not None else None,
            "ops_source": "profiles/opcounts.json (binary32 replica op count, frozen)",
            "peak_note": "152 SMs x 128 FP32 lanes x 2.070 GHz max SM clock (derived)"}
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    alg_gbs = roof["algorithmic_bytes"] / (ms / 1e3) / 1e9
    roof["hbm_context"] = {"algorithmic_GBps": alg_gbs, "peak_GBps": hbm_peak, "frac": alg_gbs / hbm_peak,
                           "peak_source": "measured" if "hbm_gbs" in peaks else "fallback"}
    cpu = None if args.no_cpu_baseline else cpu_baseline(w, gpu=gpu_host)
    out = {"metric": "Gsamples/s (ms/frame at 4K)", "value": value, "unit": "Gsamples/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": line_config(w, world),
           "layout": ("F16X8 (normal and radiance interleaved)" if interleaved else
                      "F16X4 planes" if g.normal.dtype == np.float16 else "F32X4 planes"),
           "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": args.steps,
           "kernel_ms": {"min": min(kern_ms), "p10": float(np.percentile(kern_ms, 10)),
                         "median": statistics.median(kern_ms), "p90": float(np.percentile(kern_ms, 90)),
                         "max": max(kern_ms), "l2": "flushed between steps"},
           "kernel_ms_warm_l2": {"median": statistics.median(warm_ms), "min": min(warm_ms), "steps": len(warm_ms),
                                 "l2": "not flushed: the G-buffer left in L2 by the previous step"},
           "wall_s_timed_region": wall}
    if extras is not None:
        out.update({k: extras[k] for k in ("sector_counts", "storage_layouts", "batch", "serve") if k in extras})
        out["extras_clocks"] = extras["clocks"]
    print(json.dumps(out, default=_jsonable))


if __name__ == "__main__":
    main()
