"""One optimisation step of the voxel parameters over a batch of views.

The objective of Sec. 3.2.3 restricted to the terms that act on the
rasterizer's outputs: MSE against the target images, lambda_T times the
transmittance-concentration loss and lambda_dist times the distortion loss
(the SSIM, per-point RGB and TV terms are outside the rasterization path),
with the supplementary's settings: lambda_T = 0.01, lambda_dist = 0.1, Adam
with learning rates 0.025 (grid densities), 0.01 (SH degree 0) and 0.00025
(higher SH degrees), momentum (0.1, 0.99), epsilon 1e-15.  Optionally the
views are rendered at h_ss times their size and averaged down (Sec. 3.1.2
anti-aliasing) before the MSE.

Every step of the path runs in libsvr.so: svr_preprocess_views,
svr_bin_sort, svr_render_fwd_ex (colour and the distortion loss of every
ray), svr_downsample, svr_l2_loss, svr_t_concentration_loss,
svr_weighted_mean, svr_downsample_bwd, svr_render_bwd_ex, svr_adam.  PyTorch
holds the buffers.  The forward-to-backward part can be captured in a CUDA
graph (capture()); Adam is launched after the replay because its bias
correction changes every step.
"""
from __future__ import annotations

from typing import Optional, Sequence

import numpy as np
import torch

from . import _native as N
from .raster import DeviceScene, Frame, _ptr, _stream, downsample, downsample_bwd, l2_loss, supersampled_camera

LAMBDA_T = 0.01
LAMBDA_DIST = 0.1
LR_GRID = 0.025
LR_SH_DC = 0.01
LR_SH_REST = 0.00025
BETAS = (0.1, 0.99)
EPS = 1e-15


def adam(param: torch.Tensor, grad: torch.Tensor, m: torch.Tensor, v: torch.Tensor, step: int, lr: float,
         lr_rest: Optional[float] = None, period: int = 1, head: int = 1, betas=BETAS, eps: float = EPS,
         stream=None):
    """svr_adam in place on param, m, v (all float32, contiguous, same size)."""
    for t in (param, grad, m, v):
        if not t.is_contiguous() or t.dtype != torch.float32:
            raise ValueError("adam: contiguous float32 tensors expected")
    N.check(N.lib().svr_adam(_ptr(param), _ptr(grad), _ptr(m), _ptr(v), param.numel(), period, head, float(lr),
                             float(lr if lr_rest is None else lr_rest), float(betas[0]), float(betas[1]), float(eps),
                             int(step), _stream(stream)), "svr_adam")


def t_concentration_loss(alpha: torch.Tensor, weight: float, loss: torch.Tensor,
                         grad: Optional[torch.Tensor] = None, stream=None):
    """Adds weight * L_T(alpha) to loss [1]; writes dL/dalpha into grad."""
    N.check(N.lib().svr_t_concentration_loss(_ptr(alpha), alpha.numel(), float(weight), _ptr(grad), _ptr(loss),
                                             _stream(stream)), "svr_t_concentration_loss")
    return grad


def weighted_mean(x: torch.Tensor, weight: float, loss: torch.Tensor, stream=None):
    N.check(N.lib().svr_weighted_mean(_ptr(x), x.numel(), float(weight), _ptr(loss), _stream(stream)),
            "svr_weighted_mean")


class TrainStep:
    """Renders `cams` (one batch: one sort, one launch per kernel), takes the
    losses against `targets` (a list of [3, H, W] float32 tensors, one per
    view) and updates scene.grid and scene.sh in place with Adam."""

    def __init__(self, scene: DeviceScene, cams: Sequence, targets: Sequence[torch.Tensor], K: int = 1,
                 t_stop: float = 1e-4, tile: int = 16, h_ss: Optional[float] = None, lambda_t: float = LAMBDA_T,
                 lambda_dist: float = LAMBDA_DIST, pair_capacity: Optional[int] = None, stats: bool = False):
        self.scene = scene
        self.cams = list(cams)
        self.h_ss = h_ss
        self.render_cams = [supersampled_camera(c, h_ss) for c in self.cams] if h_ss else self.cams
        dev = scene.centre.device
        self.frame = Frame(scene, self.render_cams, K=K, t_stop=t_stop, tile=tile, pair_capacity=pair_capacity)
        self.frame.render()                                   # sizes the workspace (one host sync)
        self.frame.pair_capacity = int(self.frame.n_pairs * 1.15) + 4096
        self.frame.ws = None
        self.frame._alloc()
        self.lambda_t, self.lambda_dist = float(lambda_t), float(lambda_dist)
        P = self.frame.n_pixels
        self.out = self.frame.new_outputs()
        self.dist = torch.zeros(2 * P, device=dev)
        # target-resolution images, concatenated view after view
        lo = [3 * c.width * c.height for c in self.cams]
        self.lo_base = np.concatenate([[0], np.cumsum(lo)]).astype(np.int64)
        self.target = torch.cat([t.reshape(-1).float() for t in targets]).contiguous()
        if self.target.numel() != int(self.lo_base[-1]):
            raise ValueError("targets do not match the cameras")
        self.rgb_lo = torch.empty_like(self.target) if h_ss else None
        self.g_rgb_lo = torch.empty_like(self.target)
        self.g_rgb = torch.empty(3 * P, device=dev) if h_ss else self.g_rgb_lo
        self.g_alpha = torch.empty(P, device=dev)
        self.g_dist = torch.full((P,), self.lambda_dist / P, device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.d_grid = torch.zeros_like(scene.grid)
        self.d_sh = torch.zeros_like(scene.sh)
        self.m_grid, self.v_grid = torch.zeros_like(scene.grid), torch.zeros_like(scene.grid)
        self.m_sh, self.v_sh = torch.zeros_like(scene.sh), torch.zeros_like(scene.sh)
        self.n_steps = 0
        self.graph = None
        # pruning and subdivision statistics gathered by every step's backward
        # (Sec. 3.2.2): the caller reads and zeroes them between octree edits
        self.max_weight = torch.zeros(scene.n_vox, device=dev) if stats else None
        self.priority = torch.zeros(scene.n_vox, device=dev) if stats else None

    # -- the pieces -----------------------------------------------------------
    def _views(self, buf, per_pixel):
        pb = self.frame.pixel_base
        return [buf[per_pixel * int(pb[v]):per_pixel * int(pb[v + 1])] for v in range(len(self.cams))]

    def forward_backward(self, stream=None):
        """Render, losses, backward (no optimizer): fills self.loss, d_grid, d_sh."""
        fr = self.frame
        fr.preprocess(self.scene.grid, self.scene.sh, stream=stream)
        fr.bin_sort(sync=False, stream=stream)
        ex = N.SvrRenderExtras()
        ex.distortion = self.dist.data_ptr()
        o = self.out
        N.check(N.lib().svr_render_fwd_ex(N.ref(fr.frame), _ptr(o["rgb"]), _ptr(o["depth"]), _ptr(o["alpha"]),
                                          _ptr(o["T_final"]), _ptr(o["last"]), N.ref(ex), _stream(stream)),
                "svr_render_fwd_ex")
        if self.h_ss:
            for v, (c, src) in enumerate(zip(self.cams, self._views(o["rgb"], 3))):
                a, b = int(self.lo_base[v]), int(self.lo_base[v + 1])
                downsample(src.view(3, fr.cams[v].height, fr.cams[v].width), c.height, c.width,
                           dst=self.rgb_lo[a:b].view(3, c.height, c.width), stream=stream)
            l2_loss(self.rgb_lo, self.target, self.g_rgb_lo, self.loss, stream=stream)
            for v, (c, dst) in enumerate(zip(self.cams, self._views(self.g_rgb, 3))):
                a, b = int(self.lo_base[v]), int(self.lo_base[v + 1])
                downsample_bwd(self.g_rgb_lo[a:b].view(3, c.height, c.width), fr.cams[v].height, fr.cams[v].width,
                               out=dst.view(3, fr.cams[v].height, fr.cams[v].width), stream=stream)
        else:
            l2_loss(o["rgb"], self.target, self.g_rgb_lo, self.loss, stream=stream)
        t_concentration_loss(o["alpha"], self.lambda_t, self.loss, self.g_alpha, stream=stream)
        rays = [d[:d.numel() // 2] for d in self._views(self.dist, 2)]     # plane 0 of every view
        P = fr.n_pixels
        for v, r in enumerate(rays):
            weighted_mean(r, self.lambda_dist * r.numel() / P, self.loss, stream=stream)
        self.d_grid.zero_()
        bx = N.SvrRenderExtras()
        bx.distortion = self.dist.data_ptr()
        bx.d_distortion = self.g_dist.data_ptr()
        if self.max_weight is not None:
            bx.max_weight = self.max_weight.data_ptr()
            bx.priority = self.priority.data_ptr()
        N.check(N.lib().svr_render_bwd_ex(N.ref(fr.frame), _ptr(self.g_rgb), None, _ptr(self.g_alpha),
                                          _ptr(o["T_final"]), _ptr(o["last"]), _ptr(self.d_grid), _ptr(self.d_sh),
                                          N.ref(bx), _stream(stream)), "svr_render_bwd_ex")

    def optimize(self, stream=None):
        self.n_steps += 1
        adam(self.scene.grid, self.d_grid, self.m_grid, self.v_grid, self.n_steps, LR_GRID, stream=stream)
        adam(self.scene.sh, self.d_sh, self.m_sh, self.v_sh, self.n_steps, LR_SH_DC, LR_SH_REST, period=48, head=3,
             stream=stream)

    def capture(self):
        """Capture forward_backward in a CUDA graph (after one eager warm-up)."""
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.forward_backward()
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.forward_backward()
        return self

    def step(self, stream=None):
        """forward_backward (graph replay if captured) then Adam; returns the
        loss tensor (device, [1]) of this step's parameters."""
        if self.graph is not None:
            self.graph.replay()
        else:
            self.forward_backward(stream=stream)
        self.optimize(stream=stream)
        return self.loss
