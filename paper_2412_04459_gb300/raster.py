"""Python front end of the sparse-voxel rasterizer.

Thin layer over the C ABI (include/svr.h): device memory and streams come
from PyTorch, every step of the path runs in libsvr.so's kernels.

    scene = DeviceScene.from_host(synth_scene)    # scene arrays on the GPU
    frame = Frame(scene, camera, K=3)             # workspace + per-view state
    out = frame.render()                          # preprocess, bin/sort, forward
    d_grid, d_sh = frame.backward(g_rgb, g_depth, g_alpha, out)

    batch = Frame(scene, [cam0, cam1, ...], K=3)  # several views, one sort, one launch
    out = batch.render(); batch.views(out)        # per-view images

    rgb, depth, alpha = rasterize(grid, sh, scene, camera, K=3)   # autograd
"""
from __future__ import annotations

import ctypes
import dataclasses
from typing import Optional

import numpy as np
import torch

from . import _native as N


def _ptr(t: Optional[torch.Tensor]):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream: Optional[torch.cuda.Stream] = None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def camera_struct(cam) -> N.SvrCamera:
    """svr_camera from any object with fx, fy, cx, cy, w2c [3, 4], width, height."""
    c = N.SvrCamera()
    c.fx, c.fy, c.cx, c.cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    w2c = np.asarray(cam.w2c, np.float32).reshape(-1)
    for i in range(12):
        c.w2c[i] = float(w2c[i])
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def params_struct(K: int = 1, t_stop: float = 1e-4, tile: int = 16, bg=(0.0, 0.0, 0.0)) -> N.SvrParams:
    p = N.SvrParams()
    p.K, p.t_stop, p.tile = int(K), float(t_stop), int(tile)
    for i in range(3):
        p.bg[i] = float(bg[i])
    return p


@dataclasses.dataclass
class DeviceScene:
    """Scene arrays resident on the GPU (the C ABI's svr_scene)."""
    centre: torch.Tensor      # float32 [N, 3]
    level: torch.Tensor       # uint8 [N]
    corner_idx: torch.Tensor  # int32 [N, 8]
    grid: torch.Tensor        # float32 [Pts]
    sh: torch.Tensor          # float32 [N, 48]
    world_center: tuple
    world_size: float
    max_level: int

    @property
    def n_vox(self) -> int:
        return int(self.level.shape[0])

    @staticmethod
    def from_host(scene, device="cuda", max_level: Optional[int] = None) -> "DeviceScene":
        def t(a, dtype):
            return torch.as_tensor(np.ascontiguousarray(a)).to(device=device, dtype=dtype)
        ml = max_level if max_level is not None else max(1, int(scene.max_level))
        return DeviceScene(t(scene.centre, torch.float32), t(scene.level, torch.uint8),
                           t(scene.corner_idx, torch.int32), t(scene.grid, torch.float32),
                           t(scene.sh, torch.float32),
                           tuple(float(x) for x in np.asarray(scene.world_center, np.float32)),
                           float(np.float32(scene.world_size)), ml)

    def struct(self, grid: Optional[torch.Tensor] = None, sh: Optional[torch.Tensor] = None) -> N.SvrScene:
        g = self.grid if grid is None else grid
        s = self.sh if sh is None else sh
        for name, x in (("centre", self.centre), ("level", self.level), ("corner_idx", self.corner_idx),
                        ("grid", g), ("sh", s)):
            if not x.is_cuda or not x.is_contiguous():
                raise ValueError(f"{name} must be a contiguous CUDA tensor")
        sc = N.SvrScene()
        for i in range(3):
            sc.world_center[i] = self.world_center[i]
        sc.world_size = self.world_size
        sc.n_vox = self.n_vox
        sc.n_pts = int(g.shape[0])
        sc.max_level = int(self.max_level)
        sc.centre = self.centre.data_ptr()
        sc.level = self.level.data_ptr()
        sc.corner_idx = self.corner_idx.data_ptr()
        sc.grid = g.data_ptr()
        sc.sh = s.data_ptr()
        return sc


def workspace_size(n_vox: int, pair_capacity: int, cams, K=1, t_stop=1e-4, tile=16, bg=(0, 0, 0),
                   batched: bool = False) -> int:
    p = params_struct(K, t_stop, tile, bg)
    if not batched:
        c = camera_struct(cams)
        n = N.lib().svr_workspace_size(int(n_vox), int(pair_capacity), N.ref(c), N.ref(p))
    else:
        arr = (N.SvrCamera * len(cams))(*[camera_struct(c) for c in cams])
        n = N.lib().svr_workspace_size_views(int(n_vox), int(pair_capacity), arr, len(cams), N.ref(p))
    if n == 0:
        raise N.SvrError(N.SVR_ERR_INVALID, "workspace size", "invalid arguments")
    return int(n)


class Frame:
    """One view (cams = a camera) or a batch of views (cams = a list) of a
    scene: the workspace, the svr_frame and the outputs.  Outputs of a batch
    are flat buffers in the C ABI's batch layout; Frame.views() splits them."""

    def __init__(self, scene: DeviceScene, cams, K: int = 1, t_stop: float = 1e-4, tile: int = 16,
                 bg=(0.0, 0.0, 0.0), pair_capacity: Optional[int] = None):
        self.scene = scene
        self.batched = isinstance(cams, (list, tuple))
        self.cams = list(cams) if self.batched else [cams]
        self.cam = self.cams[0]
        self.cstructs = (N.SvrCamera * len(self.cams))(*[camera_struct(c) for c in self.cams])
        self.pstruct = params_struct(K, t_stop, tile, bg)
        self.K = K
        self.tile = tile
        self.pixels = [c.width * c.height for c in self.cams]
        self.pixel_base = np.concatenate([[0], np.cumsum(self.pixels)]).astype(np.int64)
        self.n_pixels = int(self.pixel_base[-1])
        if pair_capacity is None:
            pair_capacity = max(1 << 16, 4 * scene.n_vox * len(self.cams))
        self.pair_capacity = int(pair_capacity)
        self.frame = N.SvrFrame()
        self.ws = None
        self.n_pairs = None
        self.grid = scene.grid
        self.sh = scene.sh

    # -- workspace -----------------------------------------------------------
    def ws_bytes(self) -> int:
        return workspace_size(self.scene.n_vox, self.pair_capacity, self.cams if self.batched else self.cam,
                              self.pstruct.K, self.pstruct.t_stop, self.pstruct.tile, tuple(self.pstruct.bg),
                              batched=self.batched)

    def _alloc(self):
        nbytes = self.ws_bytes()
        if self.ws is None or self.ws.numel() < nbytes + 256:
            self.ws = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.scene.centre.device)
        base = self.ws.data_ptr()
        self._ws_ptr = (base + 255) & ~255
        self._ws_bytes = self.ws.numel() - (self._ws_ptr - base)

    # -- the path ------------------------------------------------------------
    def preprocess(self, grid=None, sh=None, stream=None):
        self.grid = self.scene.grid if grid is None else grid
        self.sh = self.scene.sh if sh is None else sh
        self._alloc()
        self.sstruct = self.scene.struct(self.grid, self.sh)
        L = N.lib()
        if self.batched:
            rc = L.svr_preprocess_views(N.ref(self.frame), N.ref(self.sstruct), self.cstructs, len(self.cams),
                                        N.ref(self.pstruct), ctypes.c_void_p(self._ws_ptr), self._ws_bytes,
                                        self.pair_capacity, _stream(stream))
        else:
            rc = L.svr_preprocess(N.ref(self.frame), N.ref(self.sstruct), self.cstructs, N.ref(self.pstruct),
                                  ctypes.c_void_p(self._ws_ptr), self._ws_bytes, self.pair_capacity,
                                  _stream(stream))
        N.check(rc, "svr_preprocess")

    def bin_sort(self, sync: bool = True, stream=None) -> Optional[int]:
        """Emit and sort the pairs.  sync=True reads the pair count back (and
        grows the workspace and redoes the view if it did not fit)."""
        if not sync:
            N.check(N.lib().svr_bin_sort(N.ref(self.frame), None, _stream(stream)), "svr_bin_sort")
            self.n_pairs = None
            return None
        n = ctypes.c_int64(0)
        rc = N.lib().svr_bin_sort(N.ref(self.frame), N.ref(n), _stream(stream))
        if rc == N.SVR_ERR_CAPACITY:
            self.pair_capacity = int(n.value * 1.25) + 1024
            self.preprocess(self.grid, self.sh, stream)
            rc = N.lib().svr_bin_sort(N.ref(self.frame), N.ref(n), _stream(stream))
        N.check(rc, "svr_bin_sort")
        self.n_pairs = int(n.value)
        return self.n_pairs

    def new_outputs(self, counts: bool = False):
        dev = self.scene.centre.device
        P = self.n_pixels
        out = dict(rgb=torch.empty(3 * P, device=dev), depth=torch.empty(P, device=dev),
                   alpha=torch.empty(P, device=dev), T_final=torch.empty(P, device=dev),
                   last=torch.empty(P, dtype=torch.int32, device=dev))
        if counts:
            out["counts"] = torch.empty(P, 2, dtype=torch.int32, device=dev)
        if not self.batched:
            H, W = self.cam.height, self.cam.width
            out = {k: (v.view(3, H, W) if k == "rgb" else v.view(H, W, 2) if k == "counts" else v.view(H, W))
                   for k, v in out.items()}
        return out

    def forward(self, out=None, stream=None):
        if out is None:
            out = self.new_outputs()
        N.check(N.lib().svr_render_fwd(N.ref(self.frame), _ptr(out["rgb"]), _ptr(out["depth"]),
                                       _ptr(out["alpha"]), _ptr(out["T_final"]), _ptr(out["last"]),
                                       _stream(stream)), "svr_render_fwd")
        return out

    def forward_ex(self, out=None, normal: bool = False, max_weight: Optional[torch.Tensor] = None, stream=None):
        """svr_render_fwd_ex: the forward plus, on request, the normal image
        (out["normal"], planar like rgb) and the per-voxel maximum blending
        weights (raised in place in max_weight, float32 [N])."""
        if out is None:
            out = self.new_outputs()
        if normal and "normal" not in out:
            out["normal"] = torch.empty_like(out["rgb"])
        ex = N.SvrRenderExtras()
        ex.normal = out["normal"].data_ptr() if normal else None
        ex.max_weight = max_weight.data_ptr() if max_weight is not None else None
        N.check(N.lib().svr_render_fwd_ex(N.ref(self.frame), _ptr(out["rgb"]), _ptr(out["depth"]),
                                          _ptr(out["alpha"]), _ptr(out["T_final"]), _ptr(out["last"]), N.ref(ex),
                                          _stream(stream)), "svr_render_fwd_ex")
        return out

    def backward_ex(self, g_rgb, g_depth, g_alpha, out, g_normal=None, priority: Optional[torch.Tensor] = None,
                    d_grid=None, d_sh=None, max_weight: Optional[torch.Tensor] = None, stream=None):
        """svr_render_bwd_ex: the backward plus, on request, the normal
        image's upstream gradient and the per-voxel subdivision priority
        (accumulated in place in priority, float32 [N])."""
        dev = self.scene.centre.device
        if d_grid is None:
            d_grid = torch.zeros(self.grid.shape[0], device=dev)
        if d_sh is None:
            d_sh = torch.empty(self.scene.n_vox, 48, device=dev)
        gr, gd, ga, gn = (None if t is None else t.contiguous() for t in (g_rgb, g_depth, g_alpha, g_normal))
        ex = N.SvrRenderExtras()
        ex.d_normal = gn.data_ptr() if gn is not None else None
        ex.priority = priority.data_ptr() if priority is not None else None
        ex.max_weight = max_weight.data_ptr() if max_weight is not None else None
        N.check(N.lib().svr_render_bwd_ex(N.ref(self.frame), _ptr(gr), _ptr(gd), _ptr(ga), _ptr(out["T_final"]),
                                          _ptr(out["last"]), _ptr(d_grid), _ptr(d_sh), N.ref(ex), _stream(stream)),
                "svr_render_bwd_ex")
        del gr, gd, ga, gn
        return d_grid, d_sh

    def forward_stats(self, stream=None):
        """Forward render plus per-pixel (candidates examined, hits) counts."""
        out = self.new_outputs(counts=True)
        N.check(N.lib().svr_render_stats(N.ref(self.frame), _ptr(out["rgb"]), _ptr(out["depth"]),
                                         _ptr(out["alpha"]), _ptr(out["T_final"]), _ptr(out["last"]),
                                         _ptr(out["counts"]), _stream(stream)), "svr_render_stats")
        return out

    def render(self, grid=None, sh=None, sync: bool = True, stream=None):
        self.preprocess(grid, sh, stream)
        self.bin_sort(sync=sync, stream=stream)
        return self.forward(stream=stream)

    def backward(self, g_rgb, g_depth, g_alpha, out, d_grid=None, d_sh=None, stream=None):
        dev = self.scene.centre.device
        if d_grid is None:
            d_grid = torch.zeros(self.grid.shape[0], device=dev)
        if d_sh is None:
            d_sh = torch.empty(self.scene.n_vox, 48, device=dev)
        # contiguous copies (of expanded or strided gradients) are held by
        # these names until the call has been enqueued on the stream, so the
        # caching allocator cannot hand one copy's block to the next
        gr, gd, ga = (None if t is None else t.contiguous() for t in (g_rgb, g_depth, g_alpha))
        N.check(N.lib().svr_render_bwd(N.ref(self.frame), _ptr(gr), _ptr(gd), _ptr(ga), _ptr(out["T_final"]),
                                       _ptr(out["last"]), _ptr(d_grid), _ptr(d_sh), _stream(stream)),
                "svr_render_bwd")
        del gr, gd, ga
        return d_grid, d_sh

    def render_batched(self, out, grads=None, d_grid=None, d_sh=None, stream=None):
        """The whole step through svr_render_batched (no host synchronisation;
        graph-capturable).  grads: (g_rgb, g_depth, g_alpha) flat buffers or None."""
        if not self.batched:
            raise ValueError("render_batched needs a list of cameras")
        if self.ws is None:
            self._alloc()
        self.sstruct = self.scene.struct(self.grid, self.sh)
        g = grads if grads is not None else (None, None, None)
        N.check(N.lib().svr_render_batched(
            N.ref(self.frame), N.ref(self.sstruct), self.cstructs, len(self.cams), N.ref(self.pstruct),
            ctypes.c_void_p(self._ws_ptr), self._ws_bytes, self.pair_capacity, _ptr(out["rgb"]),
            _ptr(out["depth"]), _ptr(out["alpha"]), _ptr(out["T_final"]), _ptr(out["last"]), _ptr(g[0]),
            _ptr(g[1]), _ptr(g[2]), _ptr(d_grid), _ptr(d_sh), _stream(stream)), "svr_render_batched")
        return out

    def views(self, out):
        """Per-view images (views into the flat batch buffers)."""
        res = []
        for v, c in enumerate(self.cams):
            b, e = int(self.pixel_base[v]), int(self.pixel_base[v + 1])
            H, W = c.height, c.width
            d = {"rgb": out["rgb"].reshape(-1)[3 * b:3 * e].view(3, H, W)}
            for k in ("depth", "alpha", "T_final", "last"):
                d[k] = out[k].reshape(-1)[b:e].view(H, W)
            if "counts" in out:
                d["counts"] = out["counts"].reshape(-1, 2)[b:e].view(H, W, 2)
            if "normal" in out:
                d["normal"] = out["normal"].reshape(-1)[3 * b:3 * e].view(3, H, W)
            res.append(d)
        return res

    def status(self, stream=None):
        flags = ctypes.c_uint32(0)
        n = ctypes.c_int64(0)
        N.check(N.lib().svr_frame_status(N.ref(self.frame), N.ref(flags), N.ref(n), _stream(stream)),
                "svr_frame_status")
        return int(flags.value), int(n.value)

    def buffers(self) -> N.SvrBuffers:
        b = N.SvrBuffers()
        N.check(N.lib().svr_frame_buffers(N.ref(self.frame), N.ref(b)), "svr_frame_buffers")
        return b

    # -- inspection helpers (copies of internal buffers) ---------------------
    def _dev_array(self, ptr, n, dtype):
        if n == 0:
            return torch.empty(0, dtype=dtype, device=self.scene.centre.device)
        nbytes = n * torch.empty(0, dtype=dtype).element_size()
        out = torch.empty(n, dtype=dtype, device=self.scene.centre.device)
        _device_copy(out.data_ptr(), ptr, nbytes)
        return out

    def inspect(self):
        """Host copies of the integer buffers (synchronises)."""
        torch.cuda.synchronize()
        b = self.buffers()
        nv = self.scene.n_vox * len(self.cams)
        ntiles = int(self.frame.total_tiles)
        flags, P = self.status()
        Pc = min(P, self.pair_capacity) if not flags & N.SVR_FLAG_CAPACITY else 0
        get = lambda p, n, dt: self._dev_array(p, n, dt).cpu().numpy()
        return dict(
            flags=flags, n_pairs=P,
            tile_mask=get(b.tile_mask, ntiles, torch.uint8),
            octpath=get(b.octpath, self.scene.n_vox, torch.int64).view(np.uint64),
            rect=get(b.rect, 4 * nv, torch.int16).reshape(nv, 4),
            count=get(b.count, nv, torch.int32).view(np.uint32),
            keys=get(b.keys, Pc, torch.int64).view(np.uint64),
            values=get(b.values, Pc, torch.int32).view(np.uint32),
            ranges=get(b.ranges, 2 * ntiles, torch.int32).view(np.uint32).reshape(ntiles, 2),
        )


def l2_loss(pred: torch.Tensor, target: torch.Tensor, grad: Optional[torch.Tensor] = None,
            loss: Optional[torch.Tensor] = None, stream=None):
    """MSE of pred against target through svr_l2_loss: (loss [1], grad).
    grad (same shape as pred) receives 2 (pred - target) / n."""
    if pred.shape != target.shape or not pred.is_contiguous() or not target.is_contiguous():
        raise ValueError("pred and target must be contiguous tensors of one shape")
    if grad is None:
        grad = torch.empty_like(pred)
    if loss is None:
        loss = torch.empty(1, device=pred.device)
    N.check(N.lib().svr_l2_loss(_ptr(pred), _ptr(target), pred.numel(), _ptr(grad), _ptr(loss),
                                _stream(stream)), "svr_l2_loss")
    return loss, grad


def supersampled_camera(cam, h_ss: float):
    """The camera of an image h_ss times larger over the same image plane:
    round(h_ss W) x round(h_ss H) pixels, intrinsics scaled by the exact
    per-axis size ratio (Sec. 3.1.2 "Anti-aliasing")."""
    Ws, Hs = int(round(h_ss * cam.width)), int(round(h_ss * cam.height))
    sx, sy = Ws / cam.width, Hs / cam.height
    return dataclasses.replace(cam, fx=np.float32(float(cam.fx) * sx), fy=np.float32(float(cam.fy) * sy),
                               cx=np.float32(float(cam.cx) * sx), cy=np.float32(float(cam.cy) * sy),
                               width=Ws, height=Hs)


def downsample(src: torch.Tensor, height: int, width: int, dst: Optional[torch.Tensor] = None, stream=None):
    """svr_downsample of src [..., H_ss, W_ss] (contiguous) to [..., height, width]."""
    if not src.is_contiguous():
        raise ValueError("src must be contiguous")
    Hs, Ws = src.shape[-2], src.shape[-1]
    planes = src.numel() // (Hs * Ws)
    if dst is None:
        dst = torch.empty(*src.shape[:-2], height, width, device=src.device, dtype=src.dtype)
    N.check(N.lib().svr_downsample(_ptr(src), planes, Hs, Ws, _ptr(dst), height, width, _stream(stream)),
            "svr_downsample")
    return dst


def downsample_bwd(grad: torch.Tensor, height_ss: int, width_ss: int, out: Optional[torch.Tensor] = None,
                   stream=None):
    """svr_downsample_bwd: the gradient of downsample for upstream grad."""
    grad = grad.contiguous()
    H, W = grad.shape[-2], grad.shape[-1]
    planes = grad.numel() // (H * W)
    if out is None:
        out = torch.empty(*grad.shape[:-2], height_ss, width_ss, device=grad.device, dtype=grad.dtype)
    N.check(N.lib().svr_downsample_bwd(_ptr(grad), planes, H, W, _ptr(out), height_ss, width_ss, _stream(stream)),
            "svr_downsample_bwd")
    return out


def _device_copy(dst: int, src: int, nbytes: int):
    """Device-to-device copy through torch (no allocation by the library)."""
    d = torch.cuda.current_device()
    _wrap_device_ptr(dst, nbytes, d).copy_(_wrap_device_ptr(src, nbytes, d))


def _wrap_device_ptr(ptr: int, nbytes: int, device: int) -> torch.Tensor:
    """A uint8 tensor view of existing device memory (not owned)."""
    class _Holder:
        pass
    h = _Holder()
    h.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                  "version": 3, "strides": None}
    return torch.as_tensor(h, device=f"cuda:{device}")


# --------------------------------------------------------------------- autograd

class SVRasterFn(torch.autograd.Function):
    """rgb, depth, alpha = f(grid, sh) for a fixed voxel layout and camera.

    Forward: svr_preprocess + svr_bin_sort + svr_render_fwd.  Backward:
    svr_render_bwd, which recomputes each pixel's walk back to front from the
    saved T_final and last index."""

    @staticmethod
    def forward(ctx, grid, sh, scene: DeviceScene, cam, K: int, t_stop: float, bg, pair_capacity):
        frame = Frame(scene, cam, K=K, t_stop=t_stop, bg=bg, pair_capacity=pair_capacity)
        out = frame.render(grid.detach().contiguous(), sh.detach().contiguous())
        ctx.frame = frame
        ctx.out = out
        return out["rgb"], out["depth"], out["alpha"]

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_alpha):
        frame = ctx.frame
        d_grid, d_sh = frame.backward(g_rgb, g_depth, g_alpha, ctx.out)
        return d_grid, d_sh, None, None, None, None, None, None


def rasterize(grid, sh, scene: DeviceScene, cam, K: int = 1, t_stop: float = 1e-4,
              bg=(0.0, 0.0, 0.0), pair_capacity: Optional[int] = None):
    """Differentiable render of (grid densities, SH) -> (rgb [3,H,W], depth, alpha)."""
    return SVRasterFn.apply(grid, sh, scene, cam, K, t_stop, tuple(bg), pair_capacity)
