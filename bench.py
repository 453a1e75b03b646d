#!/usr/bin/env python
"""Benchmark of the sparse-voxel rasterizer hot path on one GB300 per rank.

Workload (default ``shell1m``): the ~1M-voxel adaptive octree around a noisy
sphere shell (levels 4..9, seed 0), one 1280x840 orbit camera per rank, K = 3,
t_stop = 1e-4.  A step is one pass of the whole path: svr_preprocess,
svr_bin_sort (no host sync), svr_render_fwd and svr_render_bwd with seeded
upstream gradients, everything resident in HBM.  The reported value is
forward+backward steps/s over all ranks; the forward alone (preprocess, sort,
render) is timed too.  On one GPU the line also carries ``large_batched``:
eight 2560x1440 views of a ~8M-voxel octree (levels 4..11) rendered forward
+ backward in one graph-captured batch vs one launch sequence per view, with
the device memory in use (``--no-large`` skips it).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU
oracle on a bounded pixel sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "fwd frames/s & fwd+bwd steps/s, 1M voxels 1280x840; % HBM roofline"
L2_FLUSH_BYTES = 256 << 20           # > 129 MB L2
FP32_LANES_PER_SM = 128
# FP32 operations of the path per unit of counted work (an FMA counts once): a
# candidate's slab test is 6 multiplies, 4 min/max and 2 compares; a composited
# segment is its setup plus, per sample, the trilinear interpolation, explin,
# the exponential and the depth and transmittance updates; the backward adds,
# per sample, the chain through explin and the 8 trilinear weights.
OPS_CAND = 12                         # slab test of one candidate entry
OPS_HIT = {1: 42, 2: 71, 3: 100}      # one composited segment (forward)
OPS_HIT_BWD = {1: 98, 2: 156, 3: 214}  # one segment in the backward (recompute + gradient)
BATCH_SIZES = ((640, 480), (1280, 840), (1920, 1080))
# The DRAM traffic of the dominant kernel comes from an ncu capture recorded
# in its profile summary as one line
#   traffic: kernel=<name> bytes_per_launch=<n> source_sha1=<sha1 of the kernel's sources>
# and is reported only while the kernel's sources still hash to that value.
KERNEL_SOURCES = ("paper_2412_04459_gb300/csrc/render.cu", "paper_2412_04459_gb300/csrc/svr_internal.cuh")
TRAFFIC_RECORD = "profiles/render_bwd_shell1m.md"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--workload", choices=["shell1m", "dense5", "shell8m"], default="shell1m",
                    help="shell8m: the large batched workload (8 x 2560x1440 views of ~8M voxels), "
                         "timed on its own")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-pixels", type=int, default=24576,
                    help="pixels of the CPU oracle's timed sample (about 10-20 s on 16 cores)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 16-view batched vs per-view comparison")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the large batched workload (8 x 2560x1440 views of ~8M voxels; its scene "
                         "takes about a minute to generate)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the timings of the normal / pruning / subdivision outputs, the "
                         "anti-aliasing kernels and the training step")
    return ap.parse_args()


def workload(name, rank):
    import synth
    if name == "dense5":
        scene = synth.dense_scene(5, seed=0)
        cam = synth.dense_view_camera()
        return scene, cam, dict(K=1, t_stop=1e-4), "dense level-5 octree, 32768 voxels, 128x128, K=1"
    scene = synth.shell_scene(seed=0)
    cam = rank_camera(rank)
    desc = (f"adaptive octree around a noisy sphere shell, {scene.n_vox} voxels (levels 4-9), "
            "1280x840 orbit camera, K=3, t_stop=1e-4, forward+backward")
    return scene, cam, dict(K=3, t_stop=1e-4), desc


# ------------------------------------------------------------ multi-rank

def max_over_ranks(values, world, device=None):
    """Element-wise maximum of per-rank timings over all ranks (the slowest
    rank sets the step time).  Every rank calls it; world == 1 is a no-op."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


def whole_job_rate(world, ms_per_step):
    """Steps/s of the whole job: each of the `world` ranks renders its own
    view per step (weak scaling, replicas), so the job finishes `world`
    steps in the slowest rank's step time."""
    return world * 1000.0 / ms_per_step


def rank_camera(rank, width=1280, height=840):
    """The view rank `rank` renders: one seeded orbit camera per rank."""
    import synth
    return synth.orbit_camera(100 + rank, width, height)


# ----------------------------------------------------------------- clocks

class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# -------------------------------------------------------------- reference

def run_reference(args, rank, world):
    """The FP64 CPU oracle on a bounded pixel sample of the same workload."""
    import oracle
    import synth
    if rank != 0:
        return
    scene, cam, kw, desc = workload(args.workload, 0)
    rng = np.random.default_rng(123)
    n_px = min(256, cam.width * cam.height)
    px = np.stack([rng.integers(0, cam.width, n_px), rng.integers(0, cam.height, n_px)], 1)
    g_rgb = rng.normal(size=(n_px, 3))
    g_d = rng.normal(size=n_px)
    g_a = rng.normal(size=n_px)
    threads = os.cpu_count() or 1
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.render_grad(scene, cam, g_rgb, g_d, g_a, K=kw["K"], t_stop=kw["t_stop"], pixels=px,
                           threads=threads)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    frac = n_px / (cam.width * cam.height)
    per_step = float(np.mean(times)) / frac
    value = 1.0 / per_step
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": desc, "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": value, "unit": "steps/s", "cores": threads, "kind": "oracle",
                             "sample": f"{n_px} random pixels per step (forward+analytic backward), "
                                       "scaled to the full frame"},
            "e2e": {"value": value, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- native

def cpu_baseline(args, scene, cam, kw):
    """The oracle as it stands, on a bounded pixel sample (forward + backward)."""
    import oracle
    rng = np.random.default_rng(7)
    n_px = min(args.cpu_pixels, cam.width * cam.height)
    px = np.stack([rng.integers(0, cam.width, n_px), rng.integers(0, cam.height, n_px)], 1)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.render_grad(scene, cam, rng.normal(size=(n_px, 3)), rng.normal(size=n_px),
                       rng.normal(size=n_px), K=kw["K"], t_stop=kw["t_stop"], pixels=px, threads=threads)
    dt = time.perf_counter() - t0
    frac = n_px / (cam.width * cam.height)
    return {"value": frac / dt, "unit": "steps/s", "cores": threads, "kind": "oracle",
            "sample": f"{n_px} random pixels, forward + analytic backward ({dt:.1f} s), scaled to the full frame"}


def run_native(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    import synth
    from paper_2412_04459_gb300 import DeviceScene, Frame
    from paper_2412_04459_gb300 import build as gbuild

    gbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    scene, cam, kw, desc = workload(args.workload, rank)
    dscene = DeviceScene.from_host(scene, device=dev)
    K, t_stop = kw["K"], kw["t_stop"]
    fr = Frame(dscene, cam, K=K, t_stop=t_stop)
    fr.render()                               # sizes the workspace (host sync once)
    P = fr.n_pairs
    fr.pair_capacity = max(fr.pair_capacity, int(P * 1.1) + 1024)
    fr.render()
    H, W = cam.height, cam.width
    g_rgb, g_depth, g_alpha = (torch.as_tensor(a, device=dev) for a in synth.upstream_grads(1, H, W))
    d_grid = torch.zeros(scene.n_pts, device=dev)
    d_sh = torch.empty(scene.n_vox, 48, device=dev)
    out = fr.forward()
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
    stream = torch.cuda.current_stream()

    # work counts of the forward (candidates examined, hits) for the roofline
    st = fr.forward_stats()
    counts = st["counts"].to(torch.int64).sum(dim=(0, 1)).cpu().numpy()
    n_cand, n_hit = int(counts[0]), int(counts[1])

    def ev():
        return torch.cuda.Event(enable_timing=True)

    calls = ("preprocess", "bin_sort", "render_fwd", "render_bwd")

    def step(rec=None):
        e = [ev() for _ in range(6)] if rec is not None else None
        if e: e[0].record(stream)
        fr.preprocess()
        if e: e[1].record(stream)
        fr.bin_sort(sync=False)
        if e: e[2].record(stream)
        fr.forward(out)
        if e: e[3].record(stream)
        d_grid.zero_()
        if e: e[4].record(stream)
        fr.backward(g_rgb, g_depth, g_alpha, out, d_grid, d_sh)
        if e: e[5].record(stream)
        if rec is not None:
            rec.append(e)

    for _ in range(args.warmup):
        flush.fill_(1.0)
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = ClockSampler(local_rank)
    clk.start()
    time.sleep(0.3)
    recs = []
    torch.cuda.synchronize()
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)                      # L2 flush between timed steps (outside the events)
        step(recs)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    spans = {"preprocess": (0, 1), "bin_sort": (1, 2), "render_fwd": (2, 3), "render_bwd": (4, 5)}
    per_call = {c: float(np.mean([r[a].elapsed_time(r[b]) for r in recs])) for c, (a, b) in spans.items()}
    ms_step = float(np.mean([r[0].elapsed_time(r[5]) for r in recs]))
    ms_fwd = float(np.mean([r[0].elapsed_time(r[3]) for r in recs]))
    ms_step, ms_fwd = max_over_ranks([ms_step, ms_fwd], world, dev)

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(args, scene, cam, kw, dev, world)
    batched = None
    if not args.no_batched and args.workload == "shell1m":
        batched = run_batched(args, scene, dscene, dev, kw)
    extras = None
    if not args.no_extras and args.workload == "shell1m":
        extras = run_extras(args, scene, dscene, cam, dev, kw, fr, out, (g_rgb, g_depth, g_alpha), P)

    # the large batched workload (8 x 2560x1440 views of ~8M voxels), on one GPU
    large = None
    if world == 1 and not args.no_large and args.workload == "shell1m":
        large = run_large_batched(args)

    if rank != 0:
        return
    value = whole_job_rate(world, ms_step)
    fwd_fps = whole_job_rate(world, ms_fwd)
    peaks = load_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm = props.multi_processor_count
    sm_mhz = (peaks or {}).get("sm_max_mhz", 2070.0)
    alu_peak = sm * FP32_LANES_PER_SM * sm_mhz * 1e6 / 1e12          # T FP32 lane-ops/s
    ops = n_cand * OPS_CAND + n_hit * OPS_HIT[K]
    achieved = ops / (per_call["render_fwd"] * 1e-3) / 1e12
    # the backward tests no candidates (it reads the forward's hit masks):
    # per hit, the segment's slab test, the forward recompute and the gradient
    ops_bwd = n_hit * (OPS_CAND + OPS_HIT_BWD[K])
    achieved_bwd = ops_bwd / (per_call["render_bwd"] * 1e-3) / 1e12
    hbm = (peaks or {}).get("hbm_gbs", 6800.0)
    frame_bytes = frame_algorithmic_bytes(scene, P, H, W)
    n_launch = launches_per_step(fr)
    traffic, traffic_from = recorded_traffic(f"k_render_bwd<{K}>")
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": desc, "voxels": scene.n_vox, "pairs": P, "image": f"{W}x{H}", "K": K,
                   "l2": "flushed between steps (256 MB write, outside the timed events)",
                   "parallelism": f"replicas x{world} (one view per rank)"},
        "fwd_frames_per_s": fwd_fps, "ms_fwd": ms_fwd, "ms_per_call": per_call,
        "roofline": {"bound": "alu", "kernel": "k_render_bwd", "achieved": achieved_bwd, "peak": alu_peak,
                     "unit": "T FP32 lane-ops/s", "frac": achieved_bwd / alu_peak, "traffic": traffic,
                     "traffic_from": traffic_from,
                     "work": {"hits": n_hit, "ops_per_hit": OPS_CAND + OPS_HIT_BWD[K]},
                     "timed": "svr_render_bwd call: k_render_bwd + k_voxel_bwd + 2 memsets",
                     "peak_from": f"{sm} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_mhz:.0f} MHz"},
        "roofline_fwd": {"bound": "alu", "kernel": "k_render_fwd", "achieved": achieved, "peak": alu_peak,
                         "unit": "T FP32 lane-ops/s", "frac": achieved / alu_peak,
                         "work": {"candidates": n_cand, "hits": n_hit, "ops_per_candidate": OPS_CAND,
                                  "ops_per_hit": OPS_HIT[K]}},
        "batched": batched,
        "next_rows": extras,
        "large_batched": large,
        "frame_hbm": {"algorithmic_bytes": frame_bytes, "achieved_gbs": frame_bytes / (ms_step * 1e-3) / 1e9,
                      "peak_gbs": hbm, "frac": frame_bytes / (ms_step * 1e-3) / 1e9 / hbm,
                      "peak_from": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6800 GB/s"},
        # the whole step against the larger of its two algorithmic times:
        # minimal HBM bytes at the measured copy bandwidth, render FP32 work at the ALU peak
        "frame_roofline": frame_roofline(frame_bytes, hbm, ops + ops_bwd, alu_peak, ms_step),
        "gpu_launches": n_launch * args.steps,
        "clocks": clocks,
        "e2e": e2e,
    }
    if not args.no_cpu_baseline and world >= 1:
        line["cpu_baseline"] = cpu_baseline(args, scene, cam, kw)
    print(json.dumps(line), flush=True)


def frame_roofline(frame_bytes, hbm_gbs, lane_ops, alu_peak_t, ms_step):
    """max(bytes / bandwidth, FP32 lane-ops / ALU peak) over the measured step time."""
    ms_bytes = frame_bytes / (hbm_gbs * 1e9) * 1e3
    ms_ops = lane_ops / (alu_peak_t * 1e12) * 1e3
    return {"ms_bytes": ms_bytes, "ms_ops": ms_ops, "bound": "alu" if ms_ops >= ms_bytes else "hbm",
            "frac": max(ms_bytes, ms_ops) / ms_step}


def run_e2e(args, scene, cam, kw, dev, world):
    """The training step as a user runs it through the public API: the
    voxel parameters stay resident on the GPU (they are the model); every
    step copies its input, the target image, from pinned host memory, renders
    (svr_preprocess, svr_bin_sort, svr_render_fwd), takes the MSE loss and its
    gradient (svr_l2_loss), runs svr_render_bwd and reads the loss back."""
    import torch
    from paper_2412_04459_gb300 import DeviceScene, Frame, l2_loss
    dsc = DeviceScene.from_host(scene, device=dev)
    fr = Frame(dsc, cam, K=kw["K"], t_stop=kw["t_stop"])
    fr.render()
    fr.pair_capacity = int(fr.n_pairs * 1.1) + 1024
    H, W = cam.height, cam.width
    rng = np.random.default_rng(9)
    target_host = torch.as_tensor(rng.uniform(0, 1, size=(3, H, W)).astype(np.float32)).pin_memory()
    targets = [torch.empty(3, H, W, device=dev) for _ in range(2)]
    loss_host = torch.empty(1).pin_memory()
    loss = torch.empty(1, device=dev)
    g_rgb = torch.empty(3, H, W, device=dev)
    out = fr.new_outputs()
    d_grid = torch.zeros(scene.n_pts, device=dev)
    d_sh = torch.empty(scene.n_vox, 48, device=dev)
    h2d = target_host.numel() * target_host.element_size()
    d2h = loss_host.numel() * loss_host.element_size()
    stream = torch.cuda.current_stream()
    # the next step's target is uploaded on a copy stream while this step
    # computes (two device buffers); every step still uploads its target
    copy_stream = torch.cuda.Stream(device=dev)
    copied = [torch.cuda.Event() for _ in range(2)]
    used = [torch.cuda.Event() for _ in range(2)]

    def upload(b):
        copy_stream.wait_event(used[b])
        with torch.cuda.stream(copy_stream):
            targets[b].copy_(target_host, non_blocking=True)
        copied[b].record(copy_stream)

    state = {"i": 0}

    def step():
        b = state["i"] & 1
        state["i"] += 1
        upload(b ^ 1)                      # the next step's input
        stream.wait_event(copied[b])
        fr.preprocess()
        fr.bin_sort(sync=False)
        fr.forward(out)
        l2_loss(out["rgb"], targets[b], g_rgb, loss)
        used[b].record(stream)
        d_grid.zero_()
        fr.backward(g_rgb, None, None, out, d_grid, d_sh)
        loss_host.copy_(loss, non_blocking=True)

    for b in range(2):
        used[b].record(stream)
    upload(0)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for _ in range(args.steps):
        step()
    e.record(stream)
    torch.cuda.synchronize()
    ms = max_over_ranks([s.elapsed_time(e) / args.steps], world, dev)[0]
    return {"value": whole_job_rate(world, ms), "unit": "steps/s", "h2d_bytes_per_step": int(h2d),
            "d2h_bytes_per_step": int(d2h), "ms_per_step": ms, "loss": float(loss_host[0]),
            "step": "target image H2D -> render -> MSE loss + gradient -> backward -> loss D2H; "
                    "voxel parameters resident; the next step's upload overlaps this step's compute"}


def run_batched(args, scene, dscene, dev, kw, n_views=16, steps=10):
    """16 orbit views with resolutions drawn from 640x480 / 1280x840 /
    1920x1080: fwd+bwd of all views as autotuned graph-captured batched
    launches vs one launch sequence per view."""
    import torch
    import synth
    from paper_2412_04459_gb300 import Frame
    from paper_2412_04459_gb300.autotune import BatchedRenderer, tune
    rng = np.random.default_rng(4)
    cams = [synth.orbit_camera(s, *BATCH_SIZES[int(rng.integers(len(BATCH_SIZES)))]) for s in range(n_views)]
    t0 = time.perf_counter()
    best = tune(dscene, cams, K=kw["K"], t_stop=kw["t_stop"], reps=3, use_cache=False)
    tune_s = time.perf_counter() - t0
    r = BatchedRenderer(dscene, cams, K=kw["K"], t_stop=kw["t_stop"], tile=best["tile"],
                        partitions=best["partitions"]).capture()
    g = torch.Generator(device=dev).manual_seed(5)
    for x in r.grads:
        x.normal_(generator=g)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)

    def timed(fn):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            flush.fill_(1.0)
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            fn()
            e.record()
            ts.append((s, e))
        torch.cuda.synchronize()
        return float(np.mean([s.elapsed_time(e) for s, e in ts]))

    ms_batched = timed(r.step)
    flags, pairs = r.status()
    del r
    # the same views, one preprocess/sort/forward/backward sequence each
    frames = []
    for c in cams:
        fr = Frame(dscene, c, K=kw["K"], t_stop=kw["t_stop"])
        fr.render()
        fr.pair_capacity = int(fr.n_pairs * 1.15) + 4096
        fr._alloc()
        o = fr.new_outputs()
        gg = [torch.randn(3 * c.width * c.height, device=dev), torch.randn(c.width * c.height, device=dev),
              torch.randn(c.width * c.height, device=dev)]
        frames.append((fr, o, gg))
    d_grid = torch.zeros(scene.n_pts, device=dev)
    d_sh = torch.empty(scene.n_vox, 48, device=dev)

    def per_view():
        d_grid.zero_()
        for fr, o, gg in frames:
            fr.preprocess()
            fr.bin_sort(sync=False)
            fr.forward(o)
            fr.backward(gg[0], gg[1], gg[2], o, d_grid, d_sh)

    ms_per_view = timed(per_view)
    del frames
    torch.cuda.empty_cache()
    pixels = sum(c.width * c.height for c in cams)
    return {"views": n_views, "pixels": pixels, "sizes": [f"{c.width}x{c.height}" for c in cams],
            "pairs": pairs, "flags": flags, "tile": best["tile"], "partitions": best["partitions"],
            "tuning_ms": best["ms"], "tuning_s": tune_s,
            "ms_batched_graph": ms_batched, "ms_per_view_launches": ms_per_view,
            "views_per_s_batched": n_views * 1000.0 / ms_batched,
            "views_per_s_per_view": n_views * 1000.0 / ms_per_view,
            "speedup": ms_per_view / ms_batched, "l2": "flushed before each timed step"}


def _event_ms(fn, reps, flush, warm=2, graph=True):
    """Mean CUDA-event time of fn() on the current stream, L2 flushed before
    each timed call (outside the events).  graph=True captures fn once in a
    CUDA graph and times its replays, so the host's launch overhead (Python
    and ctypes, tens of microseconds) does not count as GPU time."""
    import torch
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    if graph:
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            fn()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        with torch.cuda.graph(g):
            fn()
        fn = g.replay
        fn()
        torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.fill_(1.0)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        ts.append((a, b))
    torch.cuda.synchronize()
    return float(np.mean([a.elapsed_time(b) for a, b in ts]))


def run_extras(args, scene, dscene, cam, dev, kw, fr, out, grads, P, reps=10):
    """Timings of the rows built beyond the base path, on the bench frame:
    the forward and backward with all extra outputs (normal image, maximum
    blending weights, distortion loss; normal gradient, subdivision priority,
    distortion gradient) against the plain ones; the anti-aliasing
    downsampling of rgb, depth and alpha from 1.1x; Adam on all grid and SH
    parameters and the transmittance-concentration loss (bandwidth-bound:
    GB/s against the measured copy bandwidth); and whole training steps
    (train.TrainStep: render, MSE + L_T + distortion, backward, Adam) of the
    1280x840 view, forward-backward graph-replayed, with and without 1.1x
    supersampling."""
    import torch
    from paper_2412_04459_gb300 import _native as N
    from paper_2412_04459_gb300.raster import _ptr, _stream, downsample, downsample_bwd, supersampled_camera
    from paper_2412_04459_gb300.train import TrainStep, adam, t_concentration_loss
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)
    hbm = (load_peaks() or {}).get("hbm_gbs", 6800.0)
    H, W = cam.height, cam.width
    g_rgb, g_depth, g_alpha = grads
    res = {}
    # forward / backward with every extra output
    normal = torch.empty(3, H, W, device=dev)
    mw = torch.zeros(scene.n_vox, device=dev)
    dist = torch.empty(2, H, W, device=dev)
    ex = N.SvrRenderExtras()
    ex.normal, ex.max_weight, ex.distortion = normal.data_ptr(), mw.data_ptr(), dist.data_ptr()
    o = out

    def fwd_ex():
        N.check(N.lib().svr_render_fwd_ex(N.ref(fr.frame), _ptr(o["rgb"]), _ptr(o["depth"]), _ptr(o["alpha"]),
                                          _ptr(o["T_final"]), _ptr(o["last"]), N.ref(ex), _stream()), "fwd_ex")

    g_n = torch.randn(3, H, W, device=dev)
    g_d = torch.full((H, W), 0.1 / (H * W), device=dev)
    pr = torch.zeros(scene.n_vox, device=dev)
    bx = N.SvrRenderExtras()
    bx.d_normal, bx.priority, bx.distortion, bx.d_distortion = g_n.data_ptr(), pr.data_ptr(), dist.data_ptr(), \
        g_d.data_ptr()
    d_grid = torch.zeros(scene.n_pts, device=dev)
    d_sh = torch.empty(scene.n_vox, 48, device=dev)

    def bwd_ex():
        N.check(N.lib().svr_render_bwd_ex(N.ref(fr.frame), _ptr(g_rgb), _ptr(g_depth), _ptr(g_alpha),
                                          _ptr(o["T_final"]), _ptr(o["last"]), _ptr(d_grid), _ptr(d_sh), N.ref(bx),
                                          _stream()), "bwd_ex")

    res["extras"] = {"ms_fwd_plain": _event_ms(lambda: fr.forward(o), reps, flush),
                     "ms_fwd_all_extras": _event_ms(fwd_ex, reps, flush)}
    fwd_ex()
    res["extras"]["ms_bwd_plain"] = _event_ms(lambda: fr.backward(g_rgb, g_depth, g_alpha, o, d_grid, d_sh), reps,
                                              flush)
    fwd_ex()
    res["extras"]["ms_bwd_all_extras"] = _event_ms(bwd_ex, reps, flush)
    res["extras"]["outputs"] = ("normal image, per-voxel max blending weight, per-ray distortion loss; backward "
                                "with the normal and distortion gradients and the subdivision priority")
    # anti-aliasing: rgb, depth, alpha from 1.1x
    ss = supersampled_camera(cam, 1.1)
    src = torch.randn(5, ss.height, ss.width, device=dev)
    dst = torch.empty(5, H, W, device=dev)
    ms_ds = _event_ms(lambda: downsample(src, H, W, dst=dst), reps, flush)
    ms_dsb = _event_ms(lambda: downsample_bwd(dst, ss.height, ss.width, out=src), reps, flush)
    by = 4 * 5 * (ss.height * ss.width + H * W)
    res["antialias"] = {"from": f"{ss.width}x{ss.height}", "to": f"{W}x{H}", "planes": 5,
                        "ms_downsample": ms_ds, "ms_downsample_bwd": ms_dsb,
                        "gbs_downsample": by / ms_ds / 1e6, "frac_downsample": by / ms_ds / 1e6 / hbm,
                        "gbs_downsample_bwd": by / ms_dsb / 1e6, "frac_downsample_bwd": by / ms_dsb / 1e6 / hbm,
                        "bytes": by}
    # Adam over all parameters, L_T over the frame
    prm = [dscene.grid.clone(), dscene.sh.clone().reshape(-1)]
    st = [(torch.randn_like(x), torch.zeros_like(x), torch.zeros_like(x)) for x in prm]
    cnt = {"t": 0}

    def adam_all():
        cnt["t"] += 1
        adam(prm[0], st[0][0], st[0][1], st[0][2], cnt["t"], 0.025)
        adam(prm[1], st[1][0], st[1][1], st[1][2], cnt["t"], 0.01, 0.00025, period=48, head=3)

    ms_adam = _event_ms(adam_all, reps, flush)
    n_par = sum(x.numel() for x in prm)
    by_adam = 28 * n_par
    loss = torch.zeros(1, device=dev)
    ga = torch.empty(H, W, device=dev)
    ms_lt = _event_ms(lambda: t_concentration_loss(o["alpha"], 0.01, loss, ga), reps, flush)
    res["optimizer"] = {"params": n_par, "ms_adam": ms_adam, "gbs_adam": by_adam / ms_adam / 1e6,
                        "frac_adam": by_adam / ms_adam / 1e6 / hbm,
                        "bytes_adam": by_adam, "ms_t_concentration": ms_lt,
                        "note": "Adam moves 28 B per parameter (read param, grad, m, v; write param, m, v)"}
    # whole training steps
    tgt = [torch.rand(3, H, W, device=dev)]
    for name, h_ss in (("train_step", None), ("train_step_ss1.1", 1.1)):
        scn = type(dscene)(dscene.centre, dscene.level, dscene.corner_idx, dscene.grid.clone(), dscene.sh.clone(),
                           dscene.world_center, dscene.world_size, dscene.max_level)
        tsp = TrainStep(scn, [cam], tgt, K=kw["K"], t_stop=kw["t_stop"], h_ss=h_ss).capture()
        ms = _event_ms(tsp.step, reps, flush, graph=False)     # replays its own graph, then Adam
        res[name] = {"ms_per_step": ms, "steps_per_s": 1000.0 / ms,
                     "step": "batched render + MSE + 0.01 L_T + 0.1 distortion + backward (graph replay) + Adam",
                     "image": f"{tsp.render_cams[0].width}x{tsp.render_cams[0].height} rendered, {W}x{H} loss"}
        del tsp, scn
    torch.cuda.empty_cache()
    return res


def run_large_batched(args, n_views=8, width=2560, height=1440):
    """The large batched workload: ~8M voxels (three noisy shells, levels
    4..11, at most 4 levels between touching voxels), 8 orbit views at
    2560x1440, K = 3, forward + backward in graph-captured batched launches
    (tile size and partitions tuned among a few candidates) vs one launch
    sequence per view; device memory in use against 180 GB.  Returns the
    measurements as a dict (its parity against the oracle is a -m gpu test
    at the same size and launch configuration)."""
    import torch
    import synth
    from paper_2412_04459_gb300 import DeviceScene, Frame
    from paper_2412_04459_gb300 import build as gbuild
    from paper_2412_04459_gb300.autotune import BatchedRenderer, tune
    gbuild.build()
    dev = torch.device("cuda", 0)
    t0 = time.perf_counter()
    scene = synth.shell_scene(0, 8_000_000, spec=synth.scenes.SHELL_THREE)
    gen_s = time.perf_counter() - t0
    free0, total = torch.cuda.mem_get_info(dev)
    dscene = DeviceScene.from_host(scene, device=dev)
    cams = [synth.orbit_camera(200 + v, width, height) for v in range(n_views)]
    best = tune(dscene, cams, K=3, t_stop=1e-4, tiles=(16, 32), partitions=(1, 2), reps=2, use_cache=False)
    r = BatchedRenderer(dscene, cams, K=3, t_stop=1e-4, tile=best["tile"], partitions=best["partitions"]).capture()
    g = torch.Generator(device=dev).manual_seed(5)
    for x in r.grads:
        x.normal_(generator=g)
    flush = torch.empty(L2_FLUSH_BYTES // 4, device=dev)

    def timed(fn, steps):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(steps):
            flush.fill_(1.0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            ts.append((a, b))
        torch.cuda.synchronize()
        return float(np.mean([a.elapsed_time(b) for a, b in ts]))

    steps = max(3, min(args.steps, 10))
    clk = ClockSampler(0)
    clk.start()
    ms_batched = timed(r.step, steps)
    clocks = clk.stop()
    flags, pairs = r.status()
    free1, _ = torch.cuda.mem_get_info(dev)
    used = total - free1
    allocated = torch.cuda.memory_allocated(dev)
    ws_bytes = sum(fr.ws_bytes() for fr in r.frames)
    del r
    torch.cuda.empty_cache()
    # the same views as one launch sequence per view
    frames = []
    for c in cams:
        fr = Frame(dscene, c, K=3, t_stop=1e-4, tile=best["tile"])
        fr.render()
        fr.pair_capacity = int(fr.n_pairs * 1.15) + 4096
        fr.ws = None
        fr._alloc()
        o = fr.new_outputs()
        gg = [torch.randn(3 * c.width * c.height, device=dev), torch.randn(c.width * c.height, device=dev),
              torch.randn(c.width * c.height, device=dev)]
        frames.append((fr, o, gg))
    d_grid = torch.zeros(scene.n_pts, device=dev)
    d_sh = torch.empty(scene.n_vox, 48, device=dev)

    def per_view():
        d_grid.zero_()
        for fr, o, gg in frames:
            fr.preprocess()
            fr.bin_sort(sync=False)
            fr.forward(o)
            fr.backward(gg[0], gg[1], gg[2], o, d_grid, d_sh)

    ms_per_view = timed(per_view, steps)
    pixels = n_views * width * height
    line = {
        "metric": "large batched fwd+bwd views/s (8 x 2560x1440, ~8M voxels)", "value": n_views * 1000.0 / ms_batched,
        "unit": "views/s", "n_gpus": 1, "steps": steps, "ms_per_step": ms_batched, "higher_is_better": True,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"three noisy shells, {scene.n_vox} voxels (levels 4-11, at most 4 levels between "
                               f"touching voxels), {n_views} orbit views {width}x{height}, K=3, t_stop=1e-4, "
                               "forward+backward", "voxels": scene.n_vox, "grid_points": scene.n_pts,
                   "pixels": pixels, "pairs": pairs, "flags": flags, "tile": best["tile"],
                   "partitions": best["partitions"], "tuning_ms": best["ms"],
                   "l2": "flushed before each timed step"},
        "ms_per_view_launches": ms_per_view, "speedup_vs_per_view": ms_per_view / ms_batched,
        "memory": {"device_used_gb": used / 1e9, "allocated_gb": allocated / 1e9,
                   "before_scene_used_gb": (total - free0) / 1e9,
                   "workspace_gb": ws_bytes / 1e9, "budget_gb": 180.0, "frac_of_budget": used / 180e9,
                   "total_gb": total / 1e9},
        "parity": "tests/test_gpu_batched_oracle.py::test_large_workload_full_size_sampled",
        "scene_generation_s": gen_s, "clocks": clocks,
    }
    del frames, d_grid, d_sh, dscene
    torch.cuda.empty_cache()
    return line


def frame_algorithmic_bytes(scene, P, H, W):
    """Minimal HBM bytes of one forward+backward step (FP32 storage): scene
    read once, pairs written/sorted/read once, images written and read, the
    gradients written."""
    N = scene.n_vox
    pre = N * (12 + 1 + 32 + 32 + 192) + N * 64          # inputs + per-voxel record
    pairs = P * 12 * 2 + P * 12                          # emit, one sort read+write, render read
    img = H * W * (12 + 4 + 4 + 4 + 4)                   # rgb, depth, alpha, T_final, last
    bwd = H * W * (12 + 4 + 4 + 4 + 4) + P * 12 + N * (64 + 192) + scene.n_pts * 4 * 2
    return int(pre + pairs + img + bwd)


def launches_per_step(fr):
    """Kernels of ours launched per step (fills/memsets excluded): tile masks,
    preprocess, 2 tile-count scan kernels, work order, emission, chunk sort,
    run merge, block lists, forward, backward, voxel backward."""
    return 2 + 2 + 1 + 1 + 2 + 1 + 1 + 2


def sources_sha1(paths=KERNEL_SOURCES):
    import hashlib
    h = hashlib.sha1()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def recorded_traffic(kernel, record=TRAFFIC_RECORD):
    """(bytes per launch, note) of `kernel` from its profile summary's traffic
    line, or (None, why) if there is none or the sources changed since."""
    path = os.path.join(ROOT, record)
    if not os.path.exists(path):
        return None, "no ncu record"
    for line in open(path):
        line = line.strip()
        if not line.startswith("traffic:"):
            continue
        kv = dict(x.split("=", 1) for x in line[len("traffic:"):].split())
        if kv.get("kernel") != kernel:
            continue
        if kv.get("source_sha1") != sources_sha1():
            return None, "kernel sources changed since the ncu capture"
        return int(kv["bytes_per_launch"]), f"ncu capture recorded in {record}"
    return None, "no ncu record for this kernel"


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return None


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "shell8m":
        if rank == 0:
            print(json.dumps(run_large_batched(args)), flush=True)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    run_native(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
