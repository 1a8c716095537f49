#!/usr/bin/env python3
"""Throughput of the renderer on the 1M-Gaussian 1920x1080 workload.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step renders one full frame (preprocess -> cull -> sort -> render) of the
1M-Gaussian cluster scene for one of 16 seeded camera poses (cycled), with
the scene resident in HBM.  Each step is timed with CUDA events on the
launching stream and L2 is flushed (a 256 MB write) between steps, outside the
events.  Prints one JSON line (rank 0).  With torchrun (N > 1) every rank
renders its own replica (frames are independent: weak scaling, no
collective); the job value is the sum of frames over max-over-ranks time.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of pixels of the same frames and reports the same metric.
"""
from __future__ import annotations

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

METRIC = "1080p frames/s @1M Gaussians (fwd)"  # fwd+bwd under "fwd_bwd", served p50/p99 under "serving"
WORKLOAD = "scene1m: 1,000,000 Gaussians (64 clusters + 10% shell, SH 3), 1920x1080, 16 poses"

# Algorithmic FP32 operations per pixel x Gaussian evaluation of the render
# kernel: the two affine 3-vectors num, d in (x, y) and their squared norms
# (~24), the reciprocal and rho^2, exp2 and its scale, the alpha clamp and
# compares (~3), t* (~4) and the blend (~8): about 40.
OPS_PER_EVAL = 40
# Mean DRAM bytes (read + write) of one render launch over the 16 poses of the
# workload, from an ncu capture of the current kernel (dram__bytes_read.sum +
# dram__bytes_write.sum, cold cache; profiles/render_kernel_scene1m_1080p.md).
RENDER_DRAM_BYTES = 16.18e6
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=32)
    ap.add_argument("--warmup", type=int, default=4)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-train", action="store_true", help="skip the 500k-Gaussian training-step timing")
    ap.add_argument("--no-hbm-large", action="store_true", help="skip preprocess and sort at 16M / 64M")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--capacity", type=int, default=48 << 20)
    ap.add_argument("--serve", default="40:10",
                    help="serving traces as rate_hz:seconds pairs ('' = skip serving)")
    ap.add_argument("--serve-warmup", type=float, default=0.0,
                    help="seconds at the start of each trace whose requests run but are not counted")
    ap.add_argument("--serve-policies", default="all", help="'all' or 'server,plain'")
    ap.add_argument("--serve-only", action="store_true",
                    help="run only the serving comparison and print its JSON (no frame timing)")
    ap.add_argument("--serve-capacity", type=int, default=1 << 28)
    ap.add_argument("--serve-budget-gb", type=float, default=48.0)
    ap.add_argument("--sort-keys", type=int, default=0,
                    help="only time aaag_radix_sort on this many random keys with values and exit")
    ap.add_argument("--sort-bits", type=int, default=32)
    ap.add_argument("--pre-gaussians", type=int, default=0,
                    help="only time aaag_preprocess of an N-Gaussian synthetic scene (the hbm.large scene)")
    ap.add_argument("--sort-reps", type=int, default=5)
    return ap.parse_args()


def run_sort_only(args):
    """Time the radix sort entry point (aaag_radix_sort) alone: N uniform
    random keys (low B bits) with their indices as values, R timed calls
    after one warm-up; prints ms per sort and bytes moved per second (each
    pass reads and writes key and value, plus one histogram read)."""
    import torch
    from paper_2504_12811_gb300 import aaag, build as B
    B.build()
    dev = torch.device("cuda", 0)
    n, bits = args.sort_keys, args.sort_bits
    g = torch.Generator(device=dev)
    g.manual_seed(1)
    k0 = torch.randint(0, 1 << min(bits, 31), (n,), device=dev, dtype=torch.int64, generator=g).to(torch.int32)
    v0 = torch.arange(n, device=dev, dtype=torch.int32)
    keys, vals = k0.clone(), v0.clone()
    ka, va = torch.empty_like(keys), torch.empty_like(vals)
    sb = aaag.aaag_radix_sort_scratch_bytes(n)
    scratch = torch.zeros(sb, dtype=torch.uint8, device=dev)
    st = aaag.current_stream()
    ms = []
    alt = 0
    for rep in range(args.sort_reps + 1):
        keys.copy_(k0)
        vals.copy_(v0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        alt = aaag.aaag_radix_sort(keys.data_ptr(), vals.data_ptr(), ka.data_ptr(), va.data_ptr(), n, bits,
                                   scratch.data_ptr(), sb, st)
        e1.record()
        torch.cuda.synchronize()
        if rep:
            ms.append(e0.elapsed_time(e1))
    out = ka if alt else keys
    ok = bool((out[1:].to(torch.int64) >= out[:-1].to(torch.int64)).all())
    passes = (bits + 7) // 8
    t = sum(ms) / len(ms)
    print(json.dumps({"keys": n, "key_bits": bits, "ms": t, "gbs": n * (16 * passes + 4) / (t / 1e3) / 1e9,
                      "sorted": ok}))
    if not ok:
        raise SystemExit("not sorted")


def run_serving(args, dev):
    """Served-request latency: the continuous-batching server against the
    plain per-frame renderer, on the same Poisson trace of mixed requests over
    three resident scenes, for each (rate, seconds) in --serve."""
    import torch
    from paper_2504_12811_gb300 import scenes, serve
    t = time.time()
    sc = scenes.serving_scenes()
    gen_s = time.time() - t
    out = {"scenes": {k: v.n for k, v in sc.items()},
           "mix": "equal thirds: 640x480 60deg, 1920x1080 60deg, stereo 2x1832x1920 110deg; "
                  "poses uniform in [-0.8,0.8]^3 inside the scene, uniform look directions",
           "latency": "host-observed completion (images of every view copied to pinned host memory) "
                      "minus arrival",
           "warmup_s": args.serve_warmup,
           "generation_s": gen_s, "runs": []}
    for spec in [x for x in args.serve.split(",") if x]:
        rate, seconds = (float(v) for v in spec.split(":"))
        trace = scenes.serving_trace(rate, seconds, seed=2)
        n_views = sum(len(r.cams) for r in trace)
        server = serve.Server(sc, int(args.serve_budget_gb * 2**30), 1920, 1920, args.serve_capacity,
                              max_batch_views=8, device=dev)
        n_slots = len(server.slots)
        all_policies = args.serve_policies == "all"
        lat_u = lat_f = lat_b = None
        try:
            server.warm(trace)
            t = time.time()
            lat = server.serve_streams(trace, urgent_pixels=1920 * 1080, heavy_pixels=1920 * 1080)
            ours_wall = time.time() - t
            if all_policies:
                t = time.time()
                lat_u = server.serve_streams(trace, urgent_pixels=640 * 480)
                urgent_wall = time.time() - t
                t = time.time()
                lat_f = server.serve_streams(trace)
                fifo_wall = time.time() - t
                t = time.time()
                lat_b = server.serve(trace)
                batch_wall = time.time() - t
        finally:
            server.close()
        del server
        torch.cuda.empty_cache()
        t = time.time()
        lat_p = serve.plain_renderer(sc, trace, 1920, 1920, args.serve_capacity, device=dev)
        plain_wall = time.time() - t
        torch.cuda.empty_cache()
        # requests of the warm-up seconds run but are not counted
        keep = [k for k, r in enumerate(trace) if r.arrival >= args.serve_warmup]
        kept_views = sum(len(trace[k].cams) for k in keep)
        span = max(seconds - args.serve_warmup, 1e-9)

        def summary(lat_s, wall):
            # rate over the counted requests: their number over the time from the
            # first counted arrival to the last counted completion
            done = max(trace[k].arrival + lat_s[k] for k in keep)
            busy = max(done - args.serve_warmup, span)
            return serve.latency_summary([lat_s[k] for k in keep], busy, kept_views)
        run = {"rate_hz": rate, "seconds": seconds, "warmup_s": args.serve_warmup, "requests": len(keep),
               "views": kept_views,
               "server": dict(summary(lat, ours_wall), slots=n_slots, budget_gb=args.serve_budget_gb, wall_s=ours_wall,
                              mode="per-request pipelines; stereo requests one at a time in arrival order, "
                                   "the others overtake them on high-priority streams"),
               "plain_per_frame": dict(summary(lat_p, plain_wall), wall_s=plain_wall)}
        if all_policies:
            run["server_priority_only"] = dict(summary(lat_u, urgent_wall), wall_s=urgent_wall,
                                               mode="per-request pipelines, 640x480 requests on high-priority streams")
            run["server_no_priority"] = dict(summary(lat_f, fifo_wall), wall_s=fifo_wall, mode="per-request pipelines")
            run["server_batches"] = dict(summary(lat_b, batch_wall), wall_s=batch_wall,
                                         mode="batch barrier, 8 views, 2 in flight")
        out["runs"].append(run)
    return out


def run_hbm_preprocess(dev, flush, n, reps=5):
    """aaag_preprocess of an n-Gaussian synthetic scene generated on the
    device (means uniform in a 20 m box, log-scales N(-4, 1), opacity logits
    N(0, 2), SH 3), seen from inside at 1920x1080: mean ms of `reps` calls
    after one warm-up (L2 flushed before each), bytes per second counted as in
    the headline's `hbm` entry, visible count."""
    import numpy as np
    import torch
    from paper_2504_12811_gb300 import aaag, scenes
    g = torch.Generator(device=dev)
    g.manual_seed(21)
    ds = aaag.DeviceScene.__new__(aaag.DeviceScene)
    ds.means = torch.rand(n, 3, device=dev, generator=g) * 20.0 - 10.0
    ds.log_scales = torch.randn(n, 3, device=dev, generator=g) - 4.0
    q = torch.randn(n, 4, device=dev, generator=g)
    ds.quats = (q / q.norm(dim=1, keepdim=True)).contiguous()
    ds.opacity_logits = torch.randn(n, device=dev, generator=g) * 2.0
    ds.sh = torch.randn(n, 48, device=dev, generator=g) * 0.05
    ds.vhat_train = torch.full((n,), 1e30, device=dev)
    ds.sh_degree, ds.n = 3, n
    cam = aaag.make_camera(scenes.make_camera((0.5, -0.3, -1.0), target=(0, 0, 0), width=1920, height=1080,
                                              fov_x_deg=60.0))
    ws = aaag.Workspace(n, 1920, 1080, 1 << 20, device=dev)
    st = torch.cuda.current_stream(dev).cuda_stream
    prm = aaag.make_params()
    sc = ds.struct()
    ms = []
    for rep in range(reps + 1):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        aaag.aaag_preprocess(sc, cam, prm, ws.handle, st)
        e1.record()
        torch.cuda.synchronize()
        if rep:
            ms.append(e0.elapsed_time(e1))
    vis = int(aaag.stats(ws, check=False)["n_visible"])
    pre_ms = float(np.mean(ms))
    pre_gbs = (n * 36 + vis * (16 + 192 + 64 + 16 + 4)) / (pre_ms / 1e3) / 1e9
    del ws, ds
    torch.cuda.empty_cache()
    return pre_ms, pre_gbs, vis


def run_hbm_large(dev, flush, hbm_peak, n=16_000_000, n_keys=64 << 20):
    """Preprocess and sort at sizes where bandwidth, not launch latency, can
    bound them: preprocess of a 16M-Gaussian synthetic scene (run_hbm_preprocess)
    and a radix sort of 64M random 32-bit keys with values, both through the
    C-ABI; bytes counted as in the headline's `hbm` entry."""
    import numpy as np
    import torch
    from paper_2504_12811_gb300 import aaag
    pre_ms, pre_gbs, vis = run_hbm_preprocess(dev, flush, n)
    g = torch.Generator(device=dev)
    g.manual_seed(22)
    st = aaag.current_stream()
    keys = torch.randint(0, 2**31 - 1, (n_keys,), device=dev, dtype=torch.int64, generator=g).to(torch.int32)
    vals = torch.arange(n_keys, device=dev, dtype=torch.int32)
    k0, v0 = keys.clone(), vals.clone()
    ka, va = torch.empty_like(keys), torch.empty_like(vals)
    sb = aaag.lib().aaag_radix_sort_scratch_bytes(n_keys)
    scratch = torch.empty(sb, dtype=torch.uint8, device=dev)
    ms = []
    for rep in range(6):
        keys.copy_(k0)
        vals.copy_(v0)
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        aaag.aaag_radix_sort(keys.data_ptr(), vals.data_ptr(), ka.data_ptr(), va.data_ptr(), n_keys, 32,
                             scratch.data_ptr(), sb, st)
        e1.record()
        torch.cuda.synchronize()
        if rep:
            ms.append(e0.elapsed_time(e1))
    sort_ms = float(np.mean(ms))
    sort_gbs = n_keys * (8 * 4 * 2 + 4) / (sort_ms / 1e3) / 1e9   # 4 passes r+w of key+value, histogram read
    del keys, vals, k0, v0, ka, va, scratch
    torch.cuda.empty_cache()
    return {"preprocess": {"gaussians": n, "visible": int(vis), "ms": pre_ms, "gbs": pre_gbs,
                           "frac": pre_gbs / hbm_peak},
            "sort": {"keys": n_keys, "key_bits": 32, "ms": sort_ms, "gbs": sort_gbs, "frac": sort_gbs / hbm_peak},
            "note": "inputs larger than L2; L2 flushed before each timed call"}


def run_train_step(args, dev, flush):
    """Forward + backward of each of the 4 views of the 500k-Gaussian
    training workload (1280x832, SH 3): the rendering work of one training
    step over those views.  This scene is dense enough that most pixels hold
    more waiting contributors than the per-pixel buffer: they take further
    depth-peeling passes (exact order)."""
    import numpy as np
    import torch
    from paper_2504_12811_gb300 import aaag, scenes
    t0 = time.time()
    scene, cams = scenes.workload("train500k")
    t_gen = time.time() - t0
    W, H = cams[0].width, cams[0].height
    ds = aaag.DeviceScene(scene, device=dev)
    ws = aaag.Workspace(scene.n, W, H, 64 << 20, device=dev)
    rgb = torch.empty(3, H, W, device=dev)
    alpha = torch.empty(H, W, device=dev)
    grads = [torch.empty_like(t) for t in (ds.means, ds.log_scales, ds.quats, ds.opacity_logits, ds.sh)]
    gs = aaag.aaag_grads(*[t.data_ptr() for t in grads])
    g = torch.Generator(device=dev)
    g.manual_seed(11)
    drgb = torch.randn(3, H, W, device=dev, generator=g)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream
    prm = aaag.make_params()
    sc = ds.struct()
    cc = [aaag.make_camera(c) for c in cams]

    def step():
        for c in cc:
            aaag.aaag_render_frame(sc, c, prm, ws.handle, rgb.data_ptr(), alpha.data_ptr(), sptr)
            aaag.aaag_render_backward(sc, ws.handle, rgb.data_ptr(), drgb.data_ptr(), None, gs, sptr)
    for _ in range(2):
        step()
    st = aaag.stats(ws, check=False)
    n = 8
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n)]
    for k in range(n):
        flush.zero_()
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    return {"workload": "train500k: 500,000 Gaussians (uniform cube, SH 3), 4 views of 1280x832",
            "ms_per_step": ms, "views_per_s": 4e3 / ms, "status": st["status"],
            "pairs_last_view": st["n_pairs"], "misorders_last_view": st["misorders"],
            "extra_passes_last_view": st["extra_passes"],
            "blended_last_view": st["blended"], "scene_generation_s": t_gen}


def max_over_ranks(x: float) -> float:
    """The largest value of x over the ranks of the process group (x itself
    without one): the job's time is that of its slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = (torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl"
           else torch.device("cpu"))
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, ms: float) -> float:
    """Whole-job throughput: the units all ranks processed (each the same
    count) per second of the slowest rank's time."""
    import torch.distributed as dist
    world = dist.get_world_size() if dist.is_available() and dist.is_initialized() else 1
    return units_per_rank * world / (max_over_ranks(ms) / 1e3)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi SM clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.samples.append(parts)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for name, v in zip(names, s[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def load_workload():
    from paper_2504_12811_gb300 import scenes
    t = time.time()
    scene, poses = scenes.workload("scene1m")
    return scene, poses, time.time() - t


def cpu_model() -> str:
    """CPU model name of this host (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def oracle_frame_seconds(scene, cam, fraction=1.0, seed=0):
    """Seconds of the oracle (as it stands) for one frame of `cam`: its
    preparation of every Gaussian plus every pixel, or a seeded random
    `fraction` of the pixels with the pixel time scaled to the full frame."""
    import numpy as np
    import oracle as O
    t0 = time.time()
    prep = O.prepare(scene, cam)
    t_prep = time.time() - t0
    py, px = np.mgrid[0:cam.height, 0:cam.width]
    px, py = px.ravel(), py.ravel()
    if fraction < 1.0:
        sel = np.random.default_rng(seed).choice(px.size, max(1, int(px.size * fraction)), replace=False)
        px, py = px[sel], py[sel]
    t1 = time.time()
    O.render_pixels(scene, cam, px, py, prep=prep)
    return t_prep + (time.time() - t1) * (cam.width * cam.height) / px.size


def cpu_baseline(scene, poses, seconds, unit_pixels):
    """Time the oracle as it stands on the host cores.

    Headline unit (1M Gaussians, 1920x1080): preparation of pose 0 plus a
    bounded random pixel sample, extrapolated to the frame.  Beside it, full
    frames of the oracle-sized workloads (4,096 Gaussians: 128x128 at
    distance 3; 480x270 zoom-out; 128x128 near-camera; the 2048x2048
    120-degree view on a 1/64 pixel sample), on all cores and on one core
    (the one-core zoom-out on a 1/8 sample).  Returns (frames/s, sample
    description, threads, frame seconds, per-workload figures)."""
    import numpy as np
    import torch
    import oracle as O
    from paper_2504_12811_gb300 import scenes
    cam = poses[0]
    t0 = time.time()
    prep = O.prepare(scene, cam)
    t_prep = time.time() - t0
    rng = np.random.default_rng(123)
    done, t_pix = 0, 0.0
    batch = 16
    while t_pix < seconds and done < 4096:
        px = rng.integers(0, cam.width, batch)
        py = rng.integers(0, cam.height, batch)
        t1 = time.time()
        O.render_pixels(scene, cam, px, py, prep=prep)
        t_pix += time.time() - t1
        done += batch
    per_pixel = t_pix / done
    frame_s = t_prep + per_pixel * unit_pixels
    desc = (f"scene1m pose 0, extrapolated: oracle preparation of all {scene.n} Gaussians ({t_prep:.2f} s) + "
            f"{done} random pixels ({t_pix:.2f} s) scaled to {unit_pixels} pixels")
    threads = torch.get_num_threads()
    small = {}
    plan = (("small", 1.0, 1.0), ("near", 1.0, 1.0), ("zoomout", 1.0, 0.125), ("widefov", 1.0 / 64, None))
    for wl, frac_all, frac_one in plan:
        sc, cams = scenes.workload(wl)
        c = cams[0]
        entry = {"gaussians": sc.n, "size": f"{c.width}x{c.height}"}
        s_all = oracle_frame_seconds(sc, c, frac_all)
        entry["all_cores"] = {"frames_per_s": 1.0 / s_all, "threads": threads, "pixel_fraction": frac_all}
        if frac_one is not None:
            torch.set_num_threads(1)
            try:
                s_one = oracle_frame_seconds(sc, c, frac_one)
            finally:
                torch.set_num_threads(threads)
            entry["one_core"] = {"frames_per_s": 1.0 / s_one, "threads": 1, "pixel_fraction": frac_one}
        small[wl] = entry
    return 1.0 / frame_s, desc, threads, frame_s, small


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import torch
    scene, poses, _ = load_workload()
    W, H = poses[0].width, poses[0].height
    import numpy as np
    import oracle as O
    rng = np.random.default_rng(5)
    # each step: oracle preparation for the pose + a bounded pixel sample
    pix = 16
    frame_times = []
    for step in range(args.warmup + args.steps):
        cam = poses[step % len(poses)]
        t0 = time.time()
        prep = O.prepare(scene, cam)
        t_prep = time.time() - t0
        px = rng.integers(0, W, pix)
        py = rng.integers(0, H, pix)
        t1 = time.time()
        O.render_pixels(scene, cam, px, py, prep=prep)
        t_pix = time.time() - t1
        if step >= args.warmup:
            frame_times.append(t_prep + t_pix / pix * W * H)
    mean_frame = sum(frame_times) / len(frame_times)
    value = 1.0 / mean_frame
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": mean_frame * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "frames/s", "cores": torch.get_num_threads(),
                         "kind": "oracle",
                         "sample": f"per step: oracle preparation of all Gaussians for the pose + {pix} "
                                   f"random pixels, frame time extrapolated to {W * H} pixels"},
        "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch
    from paper_2504_12811_gb300 import aaag, build as B

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    B.build()
    scene, poses, t_gen = load_workload()
    W, H = poses[0].width, poses[0].height
    ds = aaag.DeviceScene(scene, device=dev)
    ws = aaag.Workspace(scene.n, W, H, args.capacity, device=dev)
    rgb = torch.empty(3, H, W, device=dev)
    alpha = torch.empty(H, W, device=dev)
    stream = torch.cuda.Stream(dev)       # graph capture needs a non-default stream
    torch.cuda.set_stream(stream)
    sptr = stream.cuda_stream
    prm = aaag.make_params()
    cams = [aaag.make_camera(c) for c in poses]
    scene_struct = ds.struct()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def frame(i, ev=None):
        if ev is not None:
            ev[0].record(stream)
        aaag.aaag_preprocess(scene_struct, cams[i % len(cams)], prm, ws.handle, sptr)
        if ev is not None:
            ev[1].record(stream)
        aaag.aaag_cull(ws.handle, sptr)
        if ev is not None:
            ev[2].record(stream)
        aaag.aaag_sort(ws.handle, sptr)
        if ev is not None:
            ev[3].record(stream)
        aaag.aaag_render(ws.handle, rgb.data_ptr(), alpha.data_ptr(), sptr)
        if ev is not None:
            ev[4].record(stream)

    # warm-up (also checks capacity / timeouts once)
    for i in range(max(args.warmup, 3)):
        frame(i)
    st = aaag.stats(ws, check=False)
    if st["status"] != "OK":
        raise SystemExit(f"warm-up frame failed: {st}")

    # per-pose statistics (evaluations are needed for the roofline)
    per_pose = []
    for i in range(len(poses)):
        frame(i)
        per_pose.append(aaag.stats(ws, check=True))

    # the timed steps: each frame is one launch of the captured frame graph
    # (preprocess, cull, sort, render), re-aimed at the step's camera
    all_stages = (aaag.AAAG_STAGE_PREPROCESS | aaag.AAAG_STAGE_CULL | aaag.AAAG_STAGE_SORT |
                  aaag.AAAG_STAGE_RENDER)
    graph = aaag.aaag_graph_create(scene_struct, cams[0], prm, ws.handle, all_stages, rgb.data_ptr(),
                                   alpha.data_ptr(), sptr)
    for i in range(max(args.warmup, 3)):
        aaag.aaag_graph_launch(graph, cams[i % len(cams)], sptr)
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    wall0 = time.time()
    for k in range(args.steps):
        flush.zero_()                                  # evict L2 between steps
        gev[k][0].record(stream)
        aaag.aaag_graph_launch(graph, cams[(args.warmup + k) % len(cams)], sptr)
        gev[k][1].record(stream)
    torch.cuda.synchronize()
    wall = time.time() - wall0
    if world > 1:
        torch.distributed.barrier()
    clocks = sampler.stop()
    st_g = aaag.stats(ws, check=False)
    if st_g["status"] != "OK":
        raise SystemExit(f"timed frame failed: {st_g}")
    step_ms = np.array([a.elapsed_time(b) for a, b in gev])
    total_ms = float(step_ms.sum())
    aaag.aaag_graph_destroy(graph)

    # stage breakdown: the same steps through the per-stage calls, events
    # between the stages (these launches are not graphed)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        frame(args.warmup + k, evs[k])
    torch.cuda.synchronize()
    stage = np.array([[evs[k][j].elapsed_time(evs[k][j + 1]) for j in range(4)] for k in range(args.steps)])
    total_ms = max_over_ranks(total_ms)
    value = job_rate(args.steps, total_ms)

    # ---- ablations (Sec. 5): the same frames with one switch each
    ablation = {}
    abl_steps = max(16, min(args.steps, 64))
    for name, flags in (("full", 0), ("no_cull", aaag.AAAG_FLAG_NO_CULL),
                        ("no_resort", aaag.AAAG_FLAG_NO_RESORT), ("no_filter", aaag.AAAG_FLAG_NO_FILTER),
                        ("kbuffer", aaag.AAAG_FLAG_KBUFFER), ("no_3d", aaag.AAAG_FLAG_EVAL_2D)):
        p_abl = aaag.make_params(flags=flags)
        def abl_frame(i):
            aaag.aaag_preprocess(scene_struct, cams[i % len(cams)], p_abl, ws.handle, sptr)
            aaag.aaag_cull(ws.handle, sptr)
            aaag.aaag_sort(ws.handle, sptr)
            aaag.aaag_render(ws.handle, rgb.data_ptr(), alpha.data_ptr(), sptr)
        for i in range(3):
            abl_frame(i)
        ok = aaag.stats(ws, check=False)["status"] == "OK"
        aev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(abl_steps)]
        for k in range(abl_steps):
            flush.zero_()
            aev[k][0].record(stream)
            abl_frame(k)
            aev[k][1].record(stream)
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in aev]))
        ablation[name] = {"ms_per_frame": ms, "frames_per_s": 1e3 / ms, "status_ok": ok}
    for name in ablation:
        ablation[name]["vs_full"] = ablation[name]["ms_per_frame"] / ablation["full"]["ms_per_frame"]

    # ---- training sampling frequency (Eq. 5) of every Gaussian over 128 cameras
    rng_v = np.random.default_rng(3)
    from paper_2504_12811_gb300 import scenes as S
    tcams = [aaag.make_camera(c) for c in S.orbit_cameras(rng_v, 128, 30.0, W, H, 60.0)]
    vout = torch.empty(scene.n, device=dev)
    aaag.aaag_vhat_train(ds.means.data_ptr(), scene.n, tcams, vout.data_ptr(), sptr)
    v0, v1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    v0.record(stream)
    for _ in range(5):
        aaag.aaag_vhat_train(ds.means.data_ptr(), scene.n, tcams, vout.data_ptr(), sptr)
    v1.record(stream)
    torch.cuda.synchronize()
    vhat_ms = v0.elapsed_time(v1) / 5

    # ---- forward + backward (gradients w.r.t. every scene parameter)
    grads = [torch.empty_like(t) for t in (ds.means, ds.log_scales, ds.quats, ds.opacity_logits, ds.sh)]
    gstruct = aaag.aaag_grads(*[t.data_ptr() for t in grads])
    g = torch.Generator(device=dev)
    g.manual_seed(7)
    drgb = torch.randn(3, H, W, device=dev, generator=g)
    dalpha = torch.randn(H, W, device=dev, generator=g)
    bwd_steps = max(4, args.steps // 2)
    bev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(bwd_steps)]
    torch.cuda.synchronize()
    for k in range(bwd_steps):
        flush.zero_()
        bev[k][0].record(stream)
        frame(args.warmup + k)
        bev[k][1].record(stream)
        aaag.aaag_render_backward(scene_struct, ws.handle, rgb.data_ptr(), drgb.data_ptr(), dalpha.data_ptr(),
                                  gstruct, sptr)
        bev[k][2].record(stream)
    torch.cuda.synchronize()
    st_b = aaag.stats(ws, check=False)
    fb_ms = np.array([[bev[k][0].elapsed_time(bev[k][1]), bev[k][1].elapsed_time(bev[k][2])]
                      for k in range(bwd_steps)])
    fwd_bwd_fps = job_rate(bwd_steps, float(fb_ms.sum()))

    # ---- roofline of the dominant kernel (render, FP32 ALU bound)
    ev_by_step = [per_pose[(args.warmup + k) % len(poses)]["evaluations"] for k in range(args.steps)]
    render_ms = stage[:, 3]
    achieved_tflops = float(np.sum(np.array(ev_by_step) * OPS_PER_EVAL) / (render_ms.sum() / 1e3) / 1e12)
    sm_max = clocks.get("sm_max_mhz") or 2070.0
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    peak_tflops = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    # preprocess + cull + sort: algorithmic bytes vs measured HBM peak
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm_peak = float(peaks["hbm_gbs"])
        hbm_src = "measured"
    except (OSError, KeyError, ValueError):
        hbm_peak, hbm_src = 6800.0, "fallback"
    pre_bytes, sort_bytes = [], []
    kv = ws.view()
    passes = (kv.tile_bits + kv.depth_bits + 7) // 8     # radix passes of the pair keys
    for k in range(args.steps):
        s = per_pose[(args.warmup + k) % len(poses)]
        V, K = s["n_visible"], s["n_pairs"]
        # every Gaussian: means, log-scales, opacity, v_train read (32 B), chunk
        # count written (4 B); every visible one: quaternion and SH read
        # (16 + 192 B), record, aux word and count written (64 + 16 + 4 B)
        pre_bytes.append(scene.n * 36 + V * (16 + 192 + 64 + 16 + 4))
        sort_bytes.append(K * (8 * passes * 2 + 4) + K * 8)   # passes r+w of key+val, histogram read, ranges
    pre_gbs = float(np.sum(pre_bytes) / (stage[:, 0].sum() / 1e3) / 1e9)
    sort_gbs = float(np.sum(sort_bytes) / (stage[:, 2].sum() / 1e3) / 1e9)

    # ---- end to end through the C-ABI with host buffers.  Every step copies
    # its scene from pinned host memory and reads its image back; with two
    # device copies of the scene and of the image, the upload of step k+1 and
    # the read-back of step k-1 overlap the frame of step k (three streams).
    names = ("means", "log_scales", "quats", "opacity_logits", "sh", "vhat_train")
    host = {name: getattr(ds, name).cpu().pin_memory() for name in names}
    dsc = [ds, aaag.DeviceScene(scene, device=dev)]
    sstructs = [d.struct() for d in dsc]
    d_rgb = [rgb, torch.empty_like(rgb)]
    d_alpha = [alpha, torch.empty_like(alpha)]
    h_rgb = [torch.empty(3, H, W, pin_memory=True) for _ in range(2)]
    h_alpha = [torch.empty(H, W, pin_memory=True) for _ in range(2)]
    up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    d2h = (h_rgb[0].numel() + h_alpha[0].numel()) * 4
    e2e_steps = max(8, min(args.steps, 32))
    uploaded = [torch.cuda.Event() for _ in range(e2e_steps)]
    rendered = [torch.cuda.Event() for _ in range(e2e_steps)]
    read = [torch.cuda.Event() for _ in range(e2e_steps)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(up)
    for k in range(e2e_steps):
        b = k & 1
        if k >= 2:
            up.wait_event(rendered[k - 2])       # scene copy b is free
        with torch.cuda.stream(up):
            for name in names:
                getattr(dsc[b], name).copy_(host[name], non_blocking=True)
        uploaded[k].record(up)
        stream.wait_event(uploaded[k])
        if k >= 2:
            stream.wait_event(read[k - 2])       # image copy b is free
        aaag.aaag_preprocess(sstructs[b], cams[k % len(cams)], prm, ws.handle, sptr)
        aaag.aaag_cull(ws.handle, sptr)
        aaag.aaag_sort(ws.handle, sptr)
        aaag.aaag_render(ws.handle, d_rgb[b].data_ptr(), d_alpha[b].data_ptr(), sptr)
        rendered[k].record(stream)
        down.wait_event(rendered[k])
        with torch.cuda.stream(down):
            h_rgb[b].copy_(d_rgb[b], non_blocking=True)
            h_alpha[b].copy_(d_alpha[b], non_blocking=True)
        read[k].record(down)
    e1.record(down)
    torch.cuda.synchronize()
    e2e_value = job_rate(e2e_steps, e0.elapsed_time(e1))

    # set_frame + preprocess test + preprocess; cull: offsets + test + emit;
    # sort: histogram + radix passes + ranges; render: tile order + render
    launches_per_frame = 3 + 3 + (2 + passes) + 2
    mean = lambda key: float(np.mean([p[key] for p in per_pose]))
    line = {
        "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "launch": "one CUDA-graph launch per frame (aaag_graph_launch, all four stages)",
                   "l2": "flushed between steps (256 MB write outside the timed events)",
                   "pair_capacity": args.capacity},
        "stage_ms": {name: float(stage[:, j].mean()) for j, name in
                     enumerate(("preprocess", "cull", "sort", "render"))},
        "stage_ms_note": "per-stage calls without the graph: their sum exceeds ms_per_step by the launch gaps",
        "per_frame": {"visible": mean("n_visible"), "pairs": mean("n_pairs"),
                      "evaluations": mean("evaluations"), "blended": mean("blended"),
                      "misorders": mean("misorders"), "tiles_tested": mean("tiles_tested")},
        "evals_per_s": float(np.sum(ev_by_step) / (total_ms / 1e3)),
        "ablation": ablation,
        "vhat_train": {"gaussians": scene.n, "cameras": len(tcams), "ms": vhat_ms},
        "fwd_bwd": {"value": fwd_bwd_fps, "unit": "frames/s", "forward_ms": float(fb_ms[:, 0].mean()),
                    "backward_ms": float(fb_ms[:, 1].mean()), "steps": bwd_steps,
                    "replay_mismatch": int(st_b["replay_mismatch"])},
        "roofline": {"kernel": "render", "bound": "alu", "achieved": achieved_tflops, "peak": peak_tflops,
                     "unit": "TFLOP/s", "frac": achieved_tflops / peak_tflops, "traffic": RENDER_DRAM_BYTES,
                     "peak_source": f"{sms} SMs (device query) x {FP32_LANES_PER_SM} FP32 lanes x 2 x "
                                    f"{sm_max:.0f} MHz (max SM clock, nvidia-smi)",
                     "ops_per_evaluation": OPS_PER_EVAL},
        "hbm": {"preprocess_gbs": pre_gbs, "sort_gbs": sort_gbs, "peak_gbs": hbm_peak,
                "peak_source": hbm_src, "preprocess_frac": pre_gbs / hbm_peak,
                "sort_frac": sort_gbs / hbm_peak},
        "e2e": {"value": e2e_value, "unit": "frames/s", "steps": e2e_steps,
                "note": "scene uploaded and image read back every step; upload, frame and read-back of "
                        "consecutive steps overlap on three streams",
                "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": launches_per_frame * (args.steps + 0),
        "clocks": clocks,
        "wall_s_timed": wall,
        "scene_generation_s": t_gen,
    }
    if not args.no_hbm_large:
        line["hbm"]["large"] = run_hbm_large(dev, flush, hbm_peak)
    if not args.no_train:
        line["train_step"] = run_train_step(args, dev, flush)
    if args.serve:
        line["serving"] = run_serving(args, dev)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        v, desc, cores, frame_s, small = cpu_baseline(scene, poses, args.cpu_seconds, W * H)
        line["cpu_baseline"] = {"value": v, "unit": "frames/s", "cores": cores, "kind": "oracle",
                                "sample": desc, "nproc": os.cpu_count(), "cpu_model": cpu_model(),
                                "oracle_sized_frames": small,
                                "note": "frames/s of the FP64 oracle; a pixel_fraction below 1 times that "
                                        "share of the pixels and scales the pixel time to the frame"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.serve_only:
        import torch
        from paper_2504_12811_gb300 import build as B
        B.build()
        print(json.dumps({"serving": run_serving(args, torch.device("cuda", 0))}), flush=True)
    elif args.sort_keys:
        run_sort_only(args)
    elif args.pre_gaussians:
        import torch
        from paper_2504_12811_gb300 import build as B
        B.build()
        dev = torch.device("cuda", 0)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        pre_ms, pre_gbs, vis = run_hbm_preprocess(dev, flush, args.pre_gaussians)
        print(json.dumps({"gaussians": args.pre_gaussians, "visible": vis, "ms": pre_ms, "gbs": pre_gbs}))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
