#!/usr/bin/env python3
"""Throughput benchmark: Mpix/s cleaned at niter=4 on synthetic CCD frames.

Default workload: 64 uneven frames (16 each of 800^2, 1024^2, 2048x4096,
4096^2; per-frame gain and read noise), one crb_clean_batch call per step with
the niter loop replayed from a CUDA graph. A step is the whole hot path (niter
iterations of detection + replacement) over that batch. Inputs (1.72 GB)
exceed the 126 MB L2, so no flush is needed.

Printed (one JSON line from rank 0):
  value        device-timed batched throughput, inputs resident in HBM, graph
               replay, no per-kernel events in the timed region;
  e2e          the same through the public API with host buffers (pinned H2D
               of the inputs, D2H of cleaned frames and masks inside the timed
               region);
  per_frame    the plain path: one crb_clean call per frame, no batching;
  roofline     the dominant kernel kind, timed with CUDA events around every
               launch in a separate profiled pass of the same steps, against
               the measured issue rates of its operation mix;
  serving      Poisson arrivals of 10,000 frames at 1000 and 2000 frames/s;
  cpu_baseline the CPU oracle on a bounded sample of the workload, all host
               cores and one core;
  parity_sample the same sample cleaned on the GPU against the FP64 oracle:
               mask flips and fragile pixels.
With --impl reference the CPU oracle itself is the timed arm (this method has
no runnable reference implementation), on the same sample.
Multi-GPU (torchrun): independent replicas, one per GPU, weak scaling.
"""

from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

# A dense estimate of the detection work per pixel and iteration (two
# 25-input median selections of ~200 min/max each plus ~25 arithmetic
# operations); reported for context only, since the kernel evaluates the
# medians only where they can change a flag.
DENSE_OPS_PER_PIX_ITER = 425.0
# Algorithmic HBM bytes per pixel and iteration: read J (4 B), write I_k (4 B),
# flag bits in and out (0.25 B).
ALG_BYTES_PER_PIX_ITER = 8.25
# Per tested pixel of the bound pass: min/max operations -- the sliding column
# median (12 per two rows: the middle pair of four shared values, then one
# clamp per row), the minimum of the five column medians (4), the clamp of that
# minimum at 0 (1) -- and other FP32 operations: L+ (4 differences, 4 quadrant
# sums, 4 clips taken as t+|t|, 3 sums, 1 scale = 16) and the two threshold
# tests (gain*m, +rn^2, L+^2, *gain^2, two scaled thresholds, two compares = 8).
BOUND_TEST_MINMAX = 6 + 4 + 1
# Per pixel of iteration 1 the dense bound pass also takes med3 (the 3x3 median) from sorted columns:
# its column's three rows sorted (6), then the largest of three column minima (2), the median of three
# column medians (4), the smallest of three column maxima (2) and the median of those three (4).
M3_DENSE_MINMAX = 6 + 2 + 4 + 2 + 4
# DRAM bytes (read + write) per step and per input pixel of each kernel kind's
# launches, from an ncu capture of one step on three 4096x4096 frames of the
# batch mix (the summaries are kept with the profiles), applied to the
# workload's pixels; a kind whose kernels changed since their capture has none.
TRAFFIC_PER_PIXEL = {"bound": 858694144 / 50331648}
# Algorithmic FP32 operations per unit of each kernel kind: (min/max, other).
KIND_OPS = {
    "bound": (BOUND_TEST_MINMAX, 24),
    "s": (192, 22),       # med25; L+ 16, N: mul, add, sqrt, div; S: mul, div
    "sprime": (192, 1),   # med25 of S; the difference
    "m3": (33, 0),        # med9
}


# The headline metric, printed alike by both arms.
METRIC = "Mpix/s cleaned at niter=4, batched vs per-frame on 1 GB300; p50/p99 latency"


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the machine type)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
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
    import platform
    return platform.machine()


def cpu_sample(recipes, max_frames=4):
    """The bounded sample the CPU legs time: one 800x800 frame per size class of the workload (at most
    max_frames), generated from that class's recipe (sky, gain, read noise, star and cosmic-ray
    densities scaled to the smaller area)."""
    seen, out = set(), []
    for r in recipes:
        if (r["w"], r["h"]) in seen:
            continue
        seen.add((r["w"], r["h"]))
        rr = dict(r)
        rr.update(w=min(r["w"], 800), h=min(r["h"], 800))
        scale = rr["w"] * rr["h"] / (r["w"] * r["h"])
        rr.update(nstars=max(1, int(round(r["nstars"] * scale))), ncr=max(1, int(round(r["ncr"] * scale))))
        out.append(rr)
        if len(out) >= max_frames:
            break
    return out


def sample_desc(sample):
    sizes = ", ".join(f"{r['w']}x{r['h']} (gain {r['gain']:.2f}, read noise {r['readnoise']:.2f})" for r in sample)
    return f"{len(sample)} frames, one per size class of the workload, from that class's recipe: {sizes}"


def time_oracle(frames, threads, min_s):
    """The FP64 oracle over the frames, taken in turn, until min_s seconds have passed (at least one
    frame); returns (Mpix/s, frames timed, seconds)."""
    import oracle
    oracle.set_threads(threads)
    pix, t_tot, n = 0, 0.0, 0
    while t_tot < min_s or n == 0:
        img, P = frames[n % len(frames)]
        t0 = time.perf_counter()
        oracle.clean(img, P, 4)
        t_tot += time.perf_counter() - t0
        pix += img.size
        n += 1
    return pix / t_tot / 1e6, n, t_tot


def cpu_baseline(sample, all_s=4.0, one_s=10.0):
    """The oracle (FP64) timed on this host: all cores, then one core, on the bounded sample."""
    import oracle
    from synth import workloads as wl
    frames = [(wl.make(r), oracle.Params(gain=r["gain"], readnoise=r["readnoise"])) for r in sample]
    nproc = os.cpu_count() or 1
    v_all, n_all, t_all = time_oracle(frames, nproc, all_s)
    cores = oracle.max_threads()
    v_one, n_one, t_one = time_oracle(frames, 1, one_s)
    oracle.set_threads(nproc)
    return {"value": v_all, "unit": "Mpix/s", "cores": cores, "kind": "oracle",
            "sample": f"{sample_desc(sample)}; niter=4, FP64; {n_all} frames in {t_all:.1f} s on {cores} threads",
            "single_thread": {"value": v_one, "unit": "Mpix/s", "cores": 1,
                              "sample": f"the same frames, {n_one} in {t_one:.1f} s on 1 thread"},
            "nproc": nproc, "cpu_model": cpu_model()}


def parity_sample(torch, sample, pipeline="queue"):
    """The sample cleaned on the GPU in one batched call (the headline's kernels) against the oracle:
    bit-identical to its FP32 run; against FP64, mask flips (all on fragile pixels) and fragile pixels."""
    import oracle
    from paper_1008_2192_gb300 import Cleaner
    from synth import workloads as wl
    imgs = [wl.make(r) for r in sample]
    gains = [r["gain"] for r in sample]
    rns = [r["readnoise"] for r in sample]
    cl = Cleaner(niter=4, pipeline=pipeline)
    outs, masks = cl.clean_batch([torch.from_numpy(a).cuda() for a in imgs], gains, rns)
    cl.sync()
    flips = off = fragile = 0
    exact = True
    for a, o, m, g, r in zip(imgs, outs, masks, gains, rns):
        o, m = o.cpu().numpy(), m.cpu().numpy()
        P = oracle.Params(gain=g, readnoise=r)
        r32 = oracle.clean(a, P, 4, precision="f32")
        exact &= bool(np.array_equal(m, r32.mask) and np.array_equal(o, r32.clean))
        r64 = oracle.clean(a, P, 4, fragile=True)
        fl = m != r64.mask
        flips += int(fl.sum())
        off += int((fl & (r64.fragile == 0)).sum())
        fragile += int(r64.fragile.sum())
    cl.close()
    return {"frames": len(imgs), "pixels": int(sum(a.size for a in imgs)), "pipeline": pipeline,
            "bit_exact_vs_fp32_oracle": exact, "flips_vs_fp64": flips, "flips_off_fragile": off,
            "fragile": fragile}


def arm_config(args, desc, recipes):
    """The config object both arms print for a workload."""
    npix = sum(r["w"] * r["h"] for r in recipes)
    return {"workload": desc, "frames": len(recipes), "mpix_per_step": npix / 1e6, "niter": 4,
            "params": "sigclip 4.5, sigfrac 0.5, objlim 1.0",
            "l2": "inputs 1.7 GB > L2, no flush" if args.workload == "batch64" else "see workload",
            "parallelism": "replicas"}


def network_minmax():
    """min/max instruction counts of the generated selection networks (3-input forms count once)."""
    import re
    path = os.path.join(ROOT, "paper_1008_2192_gb300", "csrc", "_gen", "networks.cuh")
    counts = {}
    with open(path) as f:
        for line in f:
            m = re.match(r"// rank \d+ \(0-based\) of (\d+) values; \d+ two-input min/max, (\d+) instructions", line)
            if m:
                counts[int(m.group(1))] = int(m.group(2))
            m = re.match(r"// row group: (\d+) medians of 5x5 windows; \d+ two-input min/max, (\d+) instructions", line)
            if m:
                counts["row25"] = int(m.group(2)) / int(m.group(1))  # per median
    return counts


def max_over_ranks(ms, world, device="cpu"):
    """The slowest rank's time (every rank gets it); the time itself with one rank."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(npix_per_rank, steps, ms_max, world):
    """Mpix/s of the whole job: every rank cleans its own copy of the workload (replicas), timed by the
    slowest rank."""
    return world * npix_per_rank * steps / (ms_max * 1e-3) / 1e6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="crb", choices=["crb", "reference"])
    ap.add_argument("--workload", default="batch64",
                    choices=["batch64", "single4096", "single800", "mosaic16384", "triple4096", "serving",
                             "poisson750", "poisson_batch64"])
    ap.add_argument("--rates", default="50,200,500,1000,2000", help="serving: arrival rates, frames/s")
    ap.add_argument("--serve-frames", type=int, default=0, help="serving: frames per rate (0: 10,000)")
    ap.add_argument("--tile-shape", type=int, default=0)
    ap.add_argument("--no-extras", action="store_true", help="skip e2e / per-frame / cpu legs")
    return ap.parse_args()


def recipes_for(name):
    from synth import workloads as wl
    if name == "batch64":
        return wl.batch_64(), "64 uneven frames: 16x800x800, 16x1024x1024, 16x2048x4096, 16x4096x4096"
    if name == "single4096":
        return [wl.single_4096()], "one 4096x4096 frame, 5000 stars, 40000 cosmic rays"
    if name == "triple4096":  # a small case above L2 size, for profiler captures
        return wl.batch_64(sizes=[(4096, 4096)], per_size=3), "three 4096x4096 frames of the batch mix"
    if name == "single800":
        return [wl.single_800()], "one 800x800 frame, 200 stars, 1500 cosmic rays"
    return [wl.mosaic_16384()], "one 16384x16384 mosaic, 2e5 stars, 6e5 cosmic rays"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.t:
            self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def serve_run(torch, rate, nframes, seed=0, budget=64 << 30, max_inflight=2, max_batch=64, fuse2=False):
    """Poisson arrivals at `rate` frames/s, sizes uniform over the batch sizes, through crb_server.

    A pool of 2 resident frames per size stands in for arriving data (their content does not change the
    work per pixel much); outputs are recycled as frames finish. Latency = completion - scheduled arrival.
    """
    from paper_1008_2192_gb300 import Server
    from synth import workloads as wl
    t_arr, recipes = wl.serving_stream(nframes, rate, seed=seed)
    pool = {}
    for r in recipes:
        key = (r["w"], r["h"])
        if key not in pool:
            imgs = []
            for j in range(2):
                rr = dict(r, index=900000 + len(pool) * 2 + j)
                imgs.append(torch.from_numpy(wl.make(rr)).cuda())
            pool[key] = {"imgs": imgs, "free": [], "n_alloc": 0}
    srv = Server(niter=4, budget_bytes=budget, max_inflight=max_inflight, max_batch=max_batch, fuse2=fuse2)
    lat = [None] * nframes
    pix = 0
    busy = {}
    i = 0
    t0 = time.perf_counter()
    pending = None
    done_n = 0
    t_last = t0
    while done_n < nframes:
        for tag, l_srv, st in srv.poll(block_ms=0):
            if st != 0:
                raise RuntimeError(f"served frame {tag} failed with status {st}")
            key, bufs, t_sub = busy.pop(tag)
            pool[key]["free"].append(bufs)
            lat[tag] = (t_sub - (t0 + t_arr[tag])) + l_srv
            done_n += 1
            t_last = time.perf_counter()
        now = time.perf_counter() - t0
        if pending is None and i < nframes and now >= t_arr[i]:
            pending = i
            i += 1
        if pending is not None:
            r = recipes[pending]
            key = (r["w"], r["h"])
            p = pool[key]
            if not p["free"] and p["n_alloc"] < 16:
                img0 = p["imgs"][0]
                p["free"].append((torch.empty_like(img0), torch.empty(img0.shape, dtype=torch.uint8, device="cuda")))
                p["n_alloc"] += 1
            if p["free"]:
                bufs = p["free"].pop()
                img = p["imgs"][pending % 2]
                if srv.submit(img, bufs[0], bufs[1], tag=pending, gain=r["gain"], readnoise=r["readnoise"]):
                    busy[pending] = (key, bufs, time.perf_counter())
                    pix += img.numel()
                    pending = None
                    continue
                p["free"].append(bufs)
        time.sleep(0.0002)
    stats = srv.stats()
    srv.close()
    span = t_last - t0
    lat = np.array(lat)
    return {"rate_hz": rate, "frames": nframes, "mpix_per_s": pix / span / 1e6,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "waves": stats["waves"], "max_wave": stats["max_wave"], "peak_resident_gb": stats["peak_resident_bytes"] / 1e9}


def run_serving(args):
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    rates = [float(x) for x in args.rates.split(",")]
    res = []
    for rate in rates:
        n = args.serve_frames or 10000
        res.append(serve_run(torch, rate, n))
    best = max(res, key=lambda r: r["mpix_per_s"])
    line = {"metric": "Mpix/s served at niter=4 (continuous batching, 1 GB300); p50/p99 latency",
            "value": best["mpix_per_s"], "unit": "Mpix/s", "n_gpus": 1, "steps": len(rates), "warmup": 0,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "Poisson arrivals, sizes uniform over 800x800, 1024x1024, 2048x4096, 4096x4096; "
                                   "64 GB budget, 2 wave slots, waves of up to 64 frames"},
            "serving": res}
    print(json.dumps(line), flush=True)


def run_reference(args):
    """The reference arm: the FP64 CPU oracle, timed on this host's cores, each step one pass over the
    bounded sample of the workload that the CPU baseline uses."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from synth import workloads as wl
    if args.workload.startswith("poisson"):
        run_reference_poisson(args)
        return
    recipes, desc = recipes_for(args.workload)
    sample = cpu_sample(recipes)
    frames = [(wl.make(r), oracle.Params(gain=r["gain"], readnoise=r["readnoise"])) for r in sample]
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)

    def step():
        for img, P in frames:
            oracle.clean(img, P, 4)

    for _ in range(max(0, min(args.warmup, 1))):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t0
    pix = sum(img.size for img, _ in frames)
    value = args.steps * pix / dt / 1e6
    sample_txt = f"each step: {sample_desc(sample)}; niter=4, FP64 oracle, {oracle.max_threads()} threads"
    config = arm_config(args, desc, recipes)
    config["sample"] = sample_txt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mpix/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config,
            "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": sample_txt, "nproc": threads, "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# FP64 arithmetic of the POISSON work function: one multiply per uniform drawn (the product; the
# uniform's exact scaling by 2^-53 is built from its bits and the comparison with e^-mu is made on
# the bit patterns), and per pixel 32 for e^-mu: the reduction (3 multiplies, 1 rounding, 2
# subtractions) and the degree-13 Horner polynomial (13 multiplies, 13 additions).
POISSON_FP64_EXP = 32
# Nominal dense FP64 rate of a GB300 (no measured figure): 1.25 TFLOP/s counting a multiply-add as two
# operations, i.e. 0.625 T single FP64 operations per second.
POISSON_FP64_PEAK = 0.625e12


def run_poisson(args):
    """The POISSON work function (Sec. 6.3.2): the paper's 750x750 image of 24.3, or 64 frames of the batch
    sizes at the same mean; device buffers, CUDA events; the oracle timed on the host cores beside it."""
    import torch
    import oracle
    from paper_1008_2192_gb300 import poisson_batch_into
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    mu = 24.3
    if args.workload == "poisson750":
        sizes, desc = [(750, 750)], "the paper's POISSON test image: 750x750, every pixel 24.3"
    else:
        sizes = [(800, 800)] * 16 + [(1024, 1024)] * 16 + [(2048, 4096)] * 16 + [(4096, 4096)] * 16
        desc = "64 frames of the batch sizes (16x800x800, 16x1024x1024, 16x2048x4096, 16x4096x4096), every pixel 24.3"
    imgs = [torch.full((h, w), mu, dtype=torch.float32, device="cuda") for (w, h) in sizes]
    outs = [torch.empty_like(a) for a in imgs]
    seeds = list(range(len(imgs)))
    npix = sum(w * h for (w, h) in sizes)
    stream = torch.cuda.current_stream()

    def step():
        poisson_batch_into(imgs, outs, seeds)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    clk = clocks.stop()
    draws = sum(float(o.double().sum().item()) + o.numel() for o in outs)  # k + 1 uniforms per pixel
    fp64 = draws + POISSON_FP64_EXP * npix
    # end to end: pinned host input, copies in and out inside the timed region
    h_in = [a.cpu().pin_memory() for a in imgs]
    h_out = [torch.empty(a.shape, dtype=torch.float32).pin_memory() for a in imgs]

    def e2e_step():
        for hi, di in zip(h_in, imgs):
            di.copy_(hi, non_blocking=True)
        step()
        for ho, do in zip(h_out, outs):
            ho.copy_(do, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    k2 = max(2, min(args.steps, 20))
    a.record(stream)
    for _ in range(k2):
        e2e_step()
    b.record(stream)
    torch.cuda.synchronize()
    e2e_ms = a.elapsed_time(b) / k2
    # the oracle on the host cores: the 750x750 image (the first frame)
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    h0 = np.full((750, 750), mu, np.float32)
    oracle.poisson(h0, 0)
    t0 = time.perf_counter()
    reps = 0
    while time.perf_counter() - t0 < 3.0:
        oracle.poisson(h0, reps)
        reps += 1
    cpu = reps * h0.size / (time.perf_counter() - t0) / 1e6
    achieved = fp64 / (ms * 1e-3)
    line = {"metric": "Mpix/s of the POISSON work function (mean 24.3, 1 GB300)", "value": npix / (ms * 1e-3) / 1e6,
            "unit": "Mpix/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc, "frames": len(sizes), "mpix_per_step": npix / 1e6,
                       "l2": "inputs below L2" if npix * 8 < 120e6 else "inputs above L2, no flush"},
            "gpu_launches": args.steps * ((len(sizes) + 255) // 256), "clocks": clk,
            "roofline": {"bound": "alu", "kernel": "poisson_kernel", "achieved": achieved / 1e12,
                         "peak": POISSON_FP64_PEAK / 1e12, "unit": "T FP64 ops/s",
                         "frac": achieved / POISSON_FP64_PEAK, "traffic": None,
                         "peak_source": "nominal FP64 rate (1.25 TFLOP/s counting a multiply-add as two)",
                         "achieved_is": "1 FP64 multiply per uniform drawn (counted from the deviates) + 32 FP64 "
                                        "operations per pixel for e^-mu, / device time per step"},
            "e2e": {"value": npix / (e2e_ms * 1e-3) / 1e6, "unit": "Mpix/s", "h2d_bytes_per_step": npix * 4,
                    "d2h_bytes_per_step": npix * 4, "api": "crb_poisson_batch with pinned host copies around it"},
            "cpu_baseline": {"value": cpu, "unit": "Mpix/s", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"the 750x750 image of 24.3, {reps} calls in ~3 s"},
            "paper_context": "CRBLASTER with POISSON on the 750x750 image: 79.738 s on one TILE64 tile "
                             "(0.0071 Mpix/s), Sec. 6.3.2"}
    print(json.dumps(line), flush=True)


def run_reference_poisson(args):
    """The reference arm of the POISSON workloads: the oracle on the 750x750 image of 24.3 per step."""
    import oracle
    oracle.set_threads(os.cpu_count() or 1)
    img = np.full((750, 750), 24.3, np.float32)
    for i in range(max(0, min(args.warmup, 1))):
        oracle.poisson(img, i)
    t0 = time.perf_counter()
    for i in range(args.steps):
        oracle.poisson(img, i)
    dt = time.perf_counter() - t0
    value = args.steps * img.size / dt / 1e6
    line = {"impl": "reference", "metric": "Mpix/s of the POISSON work function (mean 24.3, 1 GB300)",
            "value": value, "unit": "Mpix/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": "each step: the 750x750 image of 24.3 (the paper's POISSON test image)"},
            "cpu_baseline": {"value": value, "unit": "Mpix/s", "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": "the 750x750 image of 24.3 per step"},
            "e2e": {"value": value, "unit": "Mpix/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "serving":
        run_serving(args)
        return
    if args.workload.startswith("poisson"):
        run_poisson(args)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()

    from paper_1008_2192_gb300 import Cleaner
    from paper_1008_2192_gb300.api import alu_peak, fadd_peak
    from synth import workloads as wl

    recipes, desc = recipes_for(args.workload)
    frames = [wl.make(r) for r in recipes]
    gains = [r["gain"] for r in recipes]
    rns = [r["readnoise"] for r in recipes]
    npix = sum(f.size for f in frames)
    niter = wl.CLEAN_PARAMS["niter"]

    h_imgs = [torch.from_numpy(f).pin_memory() for f in frames]
    d_imgs = [t.cuda() for t in h_imgs]
    d_outs = [torch.empty_like(t) for t in d_imgs]
    d_masks = [torch.empty(t.shape, dtype=torch.uint8, device="cuda") for t in d_imgs]
    stream = torch.cuda.current_stream()

    ops2, ops3 = alu_peak()
    # the headline: one batched call per step, its work replayed from a CUDA graph, with the launch
    # configuration the autotuner picked for this batch in the first warm-up call
    cl = Cleaner(gain=7.0, readnoise=5.0, niter=niter, tile_shape=args.tile_shape, use_graphs=True, autotune=True)

    def step(c=cl):
        c.clean_batch_into(d_imgs, d_outs, d_masks, gains, rns)

    for _ in range(max(args.warmup, 0)):
        step()
    cl.sync()

    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    cl.sync()
    launches = cl.last_launches()
    tuned = cl.tuned_config()

    # the profiled pass: the same steps with CUDA events around every launch (no graph), for the
    # per-kernel breakdown and the roofline of the dominant kernel kind
    clp = Cleaner(gain=7.0, readnoise=5.0, niter=niter, tile_shape=args.tile_shape, profile=True, autotune=True)
    step(clp)
    clp.sync()
    clp.profile_read(reset=True)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    for _ in range(args.steps):
        step(clp)
    pe1.record(stream)
    torch.cuda.synchronize()
    prof_ms = pe0.elapsed_time(pe1)
    kinds = clp.profile_kernels(reset=True)
    work = clp.last_work()  # every step cleans the same batch
    clp.close()
    det_ms = sum(v[0] for k, v in kinds.items() if k in ("bound", "need", "s", "sprime", "m3need", "m3", "cand",
                                                          "grow", "tile_detect"))
    rep_ms = sum(v[0] for k, v in kinds.items() if k in ("replace", "mask", "tile_replace"))

    ms_max = max_over_ranks(ms, world, "cuda")
    value = whole_job_value(npix, args.steps, ms_max, world)

    extras = {}
    if not args.no_extras:
        # end to end through the public API with host buffers
        h_outs = [torch.empty(f.shape, dtype=torch.float32).pin_memory() for f in frames]
        h_masks = [torch.empty(f.shape, dtype=torch.uint8).pin_memory() for f in frames]

        def serial_step():  # copies, then the clean, then copies back
            for hs, ds in zip(h_imgs, d_imgs):
                ds.copy_(hs, non_blocking=True)
            cl.clean_batch_into(d_imgs, d_outs, d_masks, gains, rns)
            for ho, do, hm, dm in zip(h_outs, d_outs, h_masks, d_masks):
                ho.copy_(do, non_blocking=True)
                hm.copy_(dm, non_blocking=True)

        cl_host = Cleaner(gain=7.0, readnoise=5.0, niter=niter, tile_shape=args.tile_shape)

        def e2e_step():  # crb_clean_batch_host: chunks with copies overlapping the cleans
            cl_host.clean_batch_host_into(h_imgs, h_outs, h_masks, gains, rns, stream)

        def timed_steps(fn, k2, reps=3):
            """Median over `reps` runs of k2 steps (after two warm-up steps) of the time per step."""
            fn()
            fn()
            torch.cuda.synchronize()
            barrier()
            times = []
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                for _ in range(k2):
                    fn()
                b.record(stream)
                torch.cuda.synchronize()
                times.append(a.elapsed_time(b) / k2)
            return sorted(times)[len(times) // 2]

        k2 = max(2, min(args.steps, 5))
        e2e_ms = timed_steps(e2e_step, k2)
        serial_ms = timed_steps(serial_step, k2)
        extras["e2e"] = {"value": world * npix / (e2e_ms * 1e-3) / 1e6, "unit": "Mpix/s",
                         "h2d_bytes_per_step": int(npix * 4), "d2h_bytes_per_step": int(npix * 5),
                         "api": "crb_clean_batch_host (pinned host buffers, chunks overlapping copies and cleans)",
                         "serial_value": world * npix / (serial_ms * 1e-3) / 1e6}
        del cl_host
        # the plain per-frame path: one crb_clean per frame
        cl_plain = Cleaner(gain=7.0, readnoise=5.0, niter=niter, tile_shape=args.tile_shape)
        plain = [Cleaner(gain=g, readnoise=r, niter=niter, tile_shape=args.tile_shape) for g, r in
                 zip(gains, rns)] if len(frames) > 1 else [cl_plain]

        def plain_step():
            for c, di, do, dm in zip(plain, d_imgs, d_outs, d_masks):
                c.clean_into(di, do, dm)

        pf_ms = timed_steps(plain_step, k2)
        extras["per_frame"] = {"value": world * npix / (pf_ms * 1e-3) / 1e6, "unit": "Mpix/s",
                               "ms_per_step": pf_ms}
        # serving: continuous batching of Poisson arrivals, 10,000 frames per rate (p50/p99 latency)
        del plain, cl_plain
        torch.cuda.empty_cache()
        extras["serving"] = [serve_run(torch, rate, 10000) for rate in (1000.0, 2000.0)]

    peaks = measured_peaks()
    fadd = fadd_peak()
    net = network_minmax()
    units = {"bound": sum(w[5] for w in work), "s": sum(w[0] for w in work), "sprime": sum(w[1] for w in work),
             "m3": sum(w[2] for w in work)}
    per_step = {k: v[0] / args.steps for k, v in kinds.items()}
    tot = sum(per_step.values())
    kernels = {k: {"ms_per_step": round(v, 4), "share": round(v / max(tot, 1e-9), 4)}
               for k, v in sorted(per_step.items(), key=lambda kv: -kv[1]) if v > 0}
    dom = max(per_step, key=lambda k: per_step[k])
    if dom in KIND_OPS:
        mm, fp = KIND_OPS[dom]
        mm_n, fp_n = mm * units[dom], fp * units[dom]  # per step
        if dom == "bound":  # iteration 1's dense pass also takes med3 at every pixel
            mm_n += M3_DENSE_MINMAX * work[0][5]
            mm = f"{mm} (+{M3_DENSE_MINMAX} in iteration 1)"
        ops = mm_n + fp_n
        achieved = ops / (per_step[dom] * 1e-3) / 1e12
        peak = ops / (mm_n / ops2 + fp_n / fadd) / 1e12  # the kernel's op mix at the measured issue rates
        traffic = TRAFFIC_PER_PIXEL.get(dom)
        roofline = {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "Tops/s",
                    "frac": achieved / peak,
                    "traffic": traffic * npix if traffic else None,
                    "traffic_is": "DRAM bytes of the kernel kind's launches per step (ncu capture scaled by pixels)",
                    "peak_source": f"measured: crb_alu_peak min/max {ops2 / 1e12:.2f} T/s and crb_fadd_peak "
                                   f"{fadd / 1e12:.2f} T/s, weighted by the kernel's {mm} min/max + {fp} other FP32 "
                                   "operations per unit",
                    "achieved_is": f"({mm} + {fp}) FP32 operations x units the kernel processed (counted live) / "
                                   "its device time (CUDA events around each launch in the profiled pass)",
                    "units_per_step": units[dom]}
    else:
        roofline = {"bound": "latency", "kernel": dom, "achieved": None, "peak": None, "unit": None, "frac": None,
                    "traffic": None}
    # context: the selection networks over all detection kernels
    # the queue kernels take S and S' medians by groups of four adjacent windows
    m25 = net["row25"] if tuned[2] == "queue" else net[25]
    minmax = sum(w[0] * m25 + w[1] * m25 + w[2] * net[9] + w[3] * (7 * net[7] + 12) + w[4] * net[49]
                 + w[5] * BOUND_TEST_MINMAX for w in work)
    roofline.update({
        "kernels": kernels,
        "profiled_pass": {"steps": args.steps, "ms_per_step": prof_ms / args.steps,
                          "how": "the timed steps again, no graph, CUDA events around every launch"},
        "work_per_iteration": [{"S": w[0], "Sprime": w[1], "med3": w[2], "cand_tests": w[3],
                                "cand_full_median": w[4], "bound_tests": w[5]} for w in work],
        "detect_minmax_tops": minmax / (det_ms / args.steps * 1e-3) / 1e12,
        "detect_ms_per_step": det_ms / args.steps, "replace_ms_per_step": rep_ms / args.steps,
        "hbm_frac_alg": (ALG_BYTES_PER_PIX_ITER * npix * niter / ((det_ms + rep_ms) / args.steps) / 1e6)
        / peaks.get("hbm_gbs", 6782.4)})

    if rank == 0:
        config = arm_config(args, desc, recipes)
        config.update({"parallelism": f"replicas x{world}", "tile_shape": args.tile_shape,
                       "graph": "the work of the call captured once and replayed",
                       "autotuned": {"pipeline": tuned[2], "segment_lists_from_iteration": tuned[1],
                                     "blocks_per_sm": tuned[0]}})
        line = {"metric": METRIC, "value": value, "unit": "Mpix/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": config,
                "gpu_launches": args.steps * launches, "clocks": clk, "roofline": roofline}
        line.update(extras)
        if not args.no_extras:
            sample = cpu_sample(recipes)
            ps = parity_sample(torch, sample)
            line["parity_sample"] = ps
            line["flips_vs_fp64"] = ps["flips_vs_fp64"]
            line["fragile"] = ps["fragile"]
            line["cpu_baseline"] = cpu_baseline(sample)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
