"""Batched multi-view rendering with a CUDA-graph-captured step and an
offline autotuner.

BatchedRenderer renders a list of views of one scene forward and backward
through svr_render_batched.  The views can be split into `partitions`
sub-batches, each with its own sort and persistent launch (fewer key bits per
sort, more launches); `tile` is the tile edge (8, 16 or 32).  Each sub-batch's
call sequence is captured once in a CUDA graph and replayed per step.

tune() times every (tile, partitions) candidate on the actual scene and
cameras and returns the fastest; results are cached in a JSON file
($SVR_TUNE_CACHE, default ~/.cache/svr_autotune.json) keyed by the scene size,
the image sizes, K and the GPU name.
"""
from __future__ import annotations

import hashlib
import json
import os
from typing import Optional, Sequence

import numpy as np
import torch

from .raster import DeviceScene, Frame

TILES = (8, 16, 32)
PARTITIONS = (1, 2, 4)


def _split(n: int, parts: int):
    parts = max(1, min(parts, n))
    edges = np.linspace(0, n, parts + 1).round().astype(int)
    return [(int(a), int(b)) for a, b in zip(edges[:-1], edges[1:]) if b > a]


class BatchedRenderer:
    """Forward + backward of many views in graph-captured batched launches.

    Outputs and upstream gradients are flat buffers in the batch layout of the
    C ABI (view after view); `d_grid` accumulates over all views (zeroed by
    the step), `d_sh` holds the sum over views."""

    def __init__(self, scene: DeviceScene, cams: Sequence, K: int = 3, t_stop: float = 1e-4, tile: int = 16,
                 partitions: int = 1, bg=(0.0, 0.0, 0.0), backward: bool = True):
        self.scene = scene
        self.cams = list(cams)
        self.tile = tile
        self.backward = backward
        dev = scene.centre.device
        self.parts = _split(len(self.cams), partitions)
        self.frames = [Frame(scene, self.cams[a:b], K=K, t_stop=t_stop, tile=tile, bg=bg) for a, b in self.parts]
        # size each sub-batch's workspace from one synchronised render
        for fr in self.frames:
            fr.render()
            fr.pair_capacity = int(fr.n_pairs * 1.15) + 4096
            fr.ws = None        # the sizing render's workspace is larger than needed
            fr._alloc()
        pix = [c.width * c.height for c in self.cams]
        self.pixel_base = np.concatenate([[0], np.cumsum(pix)]).astype(np.int64)
        P = int(self.pixel_base[-1])
        self.out = dict(rgb=torch.empty(3 * P, device=dev), depth=torch.empty(P, device=dev),
                        alpha=torch.empty(P, device=dev), T_final=torch.empty(P, device=dev),
                        last=torch.empty(P, dtype=torch.int32, device=dev))
        self.grads = [torch.zeros(3 * P, device=dev), torch.zeros(P, device=dev), torch.zeros(P, device=dev)]
        self.d_grid = torch.zeros(scene.grid.shape[0], device=dev)
        self.d_sh = torch.zeros(scene.n_vox, 48, device=dev)
        self._d_sh_parts = [self.d_sh] + [torch.zeros_like(self.d_sh) for _ in self.frames[1:]]
        self.graph = None

    def _views(self, buf, a, b, per_pixel):
        lo, hi = int(self.pixel_base[a]), int(self.pixel_base[b])
        return buf[per_pixel * lo:per_pixel * hi]

    def _enqueue(self):
        self.d_grid.zero_()
        for (a, b), fr, dsh in zip(self.parts, self.frames, self._d_sh_parts):
            out = {k: self._views(v, a, b, 3 if k == "rgb" else 1) for k, v in self.out.items()}
            g = None
            if self.backward:
                g = (self._views(self.grads[0], a, b, 3), self._views(self.grads[1], a, b, 1),
                     self._views(self.grads[2], a, b, 1))
            fr.render_batched(out, g, self.d_grid, dsh)
        for dsh in self._d_sh_parts[1:]:
            self.d_sh.add_(dsh)

    def capture(self):
        """Warm up, then capture one step in a CUDA graph."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self._enqueue()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self._enqueue()
        return self

    def step(self):
        if self.graph is None:
            self.capture()
        self.graph.replay()

    def status(self):
        """(flags, pairs) summed over the sub-batches (synchronises)."""
        flags, pairs = 0, 0
        for fr in self.frames:
            f, n = fr.status()
            flags |= f
            pairs += n
        return flags, pairs


def _time(fn, reps: int) -> float:
    torch.cuda.synchronize()
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn()
    s.record()
    for _ in range(reps):
        fn()
    e.record()
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def _key(scene: DeviceScene, cams, K: int, backward: bool) -> str:
    sig = dict(n_vox=scene.n_vox, n_pts=int(scene.grid.shape[0]), max_level=scene.max_level, K=K,
               backward=backward, sizes=[(c.width, c.height) for c in cams],
               gpu=torch.cuda.get_device_name(scene.centre.device))
    return hashlib.sha1(json.dumps(sig, sort_keys=True).encode()).hexdigest()[:20]


def _cache_path() -> str:
    return os.environ.get("SVR_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "svr_autotune.json"))


def tune(scene: DeviceScene, cams: Sequence, K: int = 3, t_stop: float = 1e-4, backward: bool = True,
         tiles=TILES, partitions=PARTITIONS, reps: int = 3, use_cache: bool = True) -> dict:
    """Time every (tile, partitions) candidate; returns {"tile", "partitions",
    "ms": {"tile/partitions": ms}}.  Cached per configuration."""
    key = _key(scene, cams, K, backward)
    path = _cache_path()
    cache = {}
    if use_cache and os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
        if key in cache:
            return cache[key]
    times = {}
    for tile in tiles:
        for parts in partitions:
            if parts > len(cams):
                continue
            r = BatchedRenderer(scene, cams, K=K, t_stop=t_stop, tile=tile, partitions=parts,
                                backward=backward).capture()
            times[f"{tile}/{parts}"] = _time(r.step, reps)
            del r
            torch.cuda.empty_cache()
    best = min(times, key=times.get)
    tile, parts = (int(x) for x in best.split("/"))
    res = {"tile": tile, "partitions": parts, "ms": times}
    if use_cache:
        cache[key] = res
        try:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            with open(path, "w") as f:
                json.dump(cache, f, indent=1)
        except OSError:
            pass
    return res
