"""FP64 CPU oracle of the SVRaster hot path (arXiv 2412.04459).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA library and never imports it; the two meet only through the seeded
inputs of the ``synth`` package.

* ``oracle.render`` / ``oracle.render_grad``: brute-force renderer and its
  analytic gradient (plain C in svr_oracle.c, FP64, OpenMP over pixels),
  with the optional normal modality (Eq. vox_normal) and the pruning and
  subdivision statistics (Sec. 3.2.2).
* ``oracle.morton``: Morton codes and the direction-dependent order (Sec. B).
* ``oracle.binning``: pixel rays, tile sign masks, tile rectangles, the
  sorting keys/values, their sort order and the per-tile ranges (Sec. 3.1.2,
  Sec. B.1).

Parity unpinned (choices shared by statement, not fixed by the paper): the SH
sign convention (no Condon-Shortley phase), the sort tie-break (key, then
value), the camera convention (OpenCV, pixel centres at +0.5), the reading of
the early-termination rule (stop after the voxel that leaves T < t_stop) and
which ray-sign patterns a voxel covers in a tile (those of the tile's pixels).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_LIB = None

# Relative band |T / t_stop - 1| around the stop threshold inside which a
# pixel's termination decision is rounding-sensitive for an FP32 renderer
# (its transmittance after ~30 composited voxels carries a relative error of
# a few 1e-6): such pixels are reported as near_stop and left out of
# elementwise image and gradient comparisons, and counted.
NEAR_STOP_REL = 1e-5

_c_double_p = ctypes.POINTER(ctypes.c_double)


class OcCamera(ctypes.Structure):
    _fields_ = [("fx", ctypes.c_double), ("fy", ctypes.c_double), ("cx", ctypes.c_double),
                ("cy", ctypes.c_double), ("R", ctypes.c_double * 9), ("t", ctypes.c_double * 3),
                ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class OcParams(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("t_stop", ctypes.c_double), ("bg", ctypes.c_double * 3)]


def lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        P = ctypes.c_void_p
        L.oc_explin.restype = ctypes.c_double
        L.oc_explin.argtypes = [ctypes.c_double]
        L.oc_explin_grad.restype = ctypes.c_double
        L.oc_explin_grad.argtypes = [ctypes.c_double]
        L.oc_sh_basis.restype = None
        L.oc_sh_basis.argtypes = [P, P]
        L.oc_pixel_ray.restype = None
        L.oc_pixel_ray.argtypes = [P, ctypes.c_double, ctypes.c_double, P, P]
        L.oc_ray_aabb.restype = ctypes.c_int
        L.oc_ray_aabb.argtypes = [P, ctypes.c_double, P, P, P, P]
        L.oc_render.restype = ctypes.c_int
        L.oc_render.argtypes = [ctypes.c_double, ctypes.c_int64, P, P, P, P, P, P, P,
                                ctypes.c_int64, P, P, P, P, P, P, P, P, ctypes.c_int]
        L.oc_render_grad.restype = ctypes.c_int
        L.oc_render_grad.argtypes = [ctypes.c_double, ctypes.c_int64, P, P, P, P, P, P, P,
                                     ctypes.c_int64, P, P, P, P, P, P, P, P, P, P, ctypes.c_int]
        L.oc_render_ex.restype = ctypes.c_int
        L.oc_render_ex.argtypes = [ctypes.c_double, ctypes.c_int64, P, P, P, P, P, P, P,
                                   ctypes.c_int64, P, P, P, P, P, P, P, P, P, P, P, ctypes.c_int]
        L.oc_render_grad_ex.restype = ctypes.c_int
        L.oc_render_grad_ex.argtypes = [ctypes.c_double, ctypes.c_int64, P, P, P, P, P, P, P,
                                        ctypes.c_int64, P, P, P, P, P, P, P, P, P, P, P, P, P, P, ctypes.c_int]
        L.oc_trilinear.restype = ctypes.c_double
        L.oc_trilinear.argtypes = [P, P]
        L.oc_interp_grad_centre.restype = None
        L.oc_interp_grad_centre.argtypes = [P, P]
        L.oc_ray_hits.restype = ctypes.c_int64
        L.oc_ray_hits.argtypes = [ctypes.c_double, ctypes.c_int64, P, P, P, P, ctypes.c_int64,
                                  P, P, P]
        _LIB = L
    return _LIB


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def camera_struct(cam) -> OcCamera:
    """FP64 widening of the float32 camera the rasterizer receives."""
    c = OcCamera()
    c.fx, c.fy, c.cx, c.cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    w2c = np.asarray(cam.w2c, np.float32).astype(np.float64)
    for i in range(9):
        c.R[i] = w2c[i // 3, i % 3]
    for i in range(3):
        c.t[i] = w2c[i, 3]
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def params_struct(K: int, t_stop: float, bg=(0.0, 0.0, 0.0)) -> OcParams:
    p = OcParams()
    p.K = int(K)
    p.t_stop = float(np.float32(t_stop))
    for i in range(3):
        p.bg[i] = float(np.float32(bg[i]))
    return p


def _threads(n):
    return int(n) if n else (os.cpu_count() or 1)


def _scene_arrays(scene, grid=None, sh=None):
    """FP64 widening of the float32 scene arrays (or FP64 overrides)."""
    centre = np.ascontiguousarray(np.asarray(scene.centre, np.float32).astype(np.float64))
    level = np.ascontiguousarray(scene.level, np.uint8)
    corner = np.ascontiguousarray(scene.corner_idx, np.int32)
    if grid is None:
        g = np.asarray(scene.grid, np.float32).astype(np.float64)
    else:
        g = np.ascontiguousarray(grid, np.float64)
    if sh is None:
        s = np.asarray(scene.sh, np.float32).astype(np.float64)
    else:
        s = np.ascontiguousarray(sh, np.float64)
    return centre, level, corner, np.ascontiguousarray(g), np.ascontiguousarray(s)


def _pixels(cam, pixels):
    if pixels is None:
        return cam.width * cam.height, None
    px = np.ascontiguousarray(pixels, np.int32).reshape(-1, 2)
    return len(px), px


def render(scene, cam, K=1, t_stop=1e-4, bg=(0.0, 0.0, 0.0), pixels=None, threads=None,
           grid=None, sh=None, near_stop_rel=None, normals=False, max_weight=None, distortion=False):
    """Brute-force FP64 render.  pixels: int [n, 2] of (x, y), or None for the
    whole image (outputs then reshaped to [H, W]).  grid / sh: optional FP64
    overrides of the scene's parameters (finite differences).

    Besides the images, per pixel: n_comp (voxels composited), term_vox (the
    voxel that stopped the walk, -1 if none), stop_margin (smallest
    |T / t_stop - 1| after a composited voxel: how close the walk came to a
    different termination decision) and near_stop = stop_margin <
    near_stop_rel (default NEAR_STOP_REL), the pixels whose termination an
    FP32 renderer may legitimately decide the other way.

    normals=True adds "normal" ([3, H, W] or [n, 3]): the composited voxel
    normals of Eq. (vox_normal).  max_weight: an FP64 array [N] that is raised
    to each voxel's largest blending weight T_i alpha_i over these pixels
    (pruning statistic, Sec. 3.2.2).  distortion=True adds "dist": each
    ray's distortion loss (Sec. 3.2.3; Mip-NeRF 360's loss over the composited
    voxels' weights, interval midpoints and lengths in ray distance)."""
    centre, level, corner, g, s = _scene_arrays(scene, grid, sh)
    n, px = _pixels(cam, pixels)
    out = dict(rgb=np.zeros((n, 3)), depth=np.zeros(n), alpha=np.zeros(n), t_final=np.zeros(n),
               n_comp=np.zeros(n, np.int32), term_vox=np.zeros(n, np.int64),
               stop_margin=np.zeros(n))
    if normals:
        out["normal"] = np.zeros((n, 3))
    if distortion:
        out["dist"] = np.zeros(n)
    if max_weight is not None:
        assert max_weight.dtype == np.float64 and max_weight.shape == (scene.n_vox,)
        assert max_weight.flags.c_contiguous
    c = camera_struct(cam)
    p = params_struct(K, t_stop, bg)
    rc = lib().oc_render_ex(float(np.float32(scene.world_size)), scene.n_vox, _ptr(centre), _ptr(level),
                            _ptr(corner), _ptr(g), _ptr(s), ctypes.byref(c), ctypes.byref(p), n,
                            _ptr(px), _ptr(out["rgb"]), _ptr(out["depth"]), _ptr(out["alpha"]),
                            _ptr(out["t_final"]), _ptr(out["n_comp"]), _ptr(out["term_vox"]),
                            _ptr(out["stop_margin"]), _ptr(out.get("normal")), _ptr(max_weight),
                            _ptr(out.get("dist")), _threads(threads))
    if rc != 0:
        raise RuntimeError(f"oc_render failed ({rc})")
    band = NEAR_STOP_REL if near_stop_rel is None else float(near_stop_rel)
    out["near_stop"] = (out["stop_margin"] < band).astype(np.uint8)
    if pixels is None:
        H, W = cam.height, cam.width
        out["rgb"] = out["rgb"].reshape(H, W, 3).transpose(2, 0, 1).copy()
        if normals:
            out["normal"] = out["normal"].reshape(H, W, 3).transpose(2, 0, 1).copy()
        for k in ("depth", "alpha", "t_final", "n_comp", "term_vox", "stop_margin", "near_stop", "dist"):
            if k not in out:
                continue
            out[k] = out[k].reshape(H, W)
    return out


def render_grad(scene, cam, g_rgb, g_depth, g_alpha, K=1, t_stop=1e-4, bg=(0.0, 0.0, 0.0),
                pixels=None, threads=None, grid=None, sh=None, magnitudes=None, g_normal=None,
                priority=None, g_dist=None):
    """Analytic FP64 gradient of sum(g_rgb*C + g_depth*D + g_alpha*A).
    Full image: g_rgb [3, H, W], g_depth/g_alpha [H, W]; pixel list: g_rgb
    [n, 3], g_depth/g_alpha [n].  Returns (d_grid [Pts], d_sh [N, 48]).
    magnitudes: a dict that, if given, receives "grid" and "sh", the sums of
    the absolute values of the terms each gradient element adds up (per
    pixel, voxel hit and sample), and "grid_seg" and "sh_seg", the same sums
    with every term weighted by the condition number of its hit's segment
    length b - a with respect to relative perturbations of the entry and exit
    plane coordinates, the ray origin and the direction components:
    ((|P_i| + |o_i|) / |d_i| + |a| + (|Q_j| + |o_j|) / |d_j| + |b|) / (b - a),
    i and j the axes of the entry plane P and the exit plane Q (large for a
    ray that grazes the voxel).

    g_normal ([3, H, W] or [n, 3]) adds g_normal . N to the objective (the
    normal image of Eq. vox_normal); g_dist ([H, W] or [n]) adds g_dist times
    each ray's distortion loss.  priority: an FP64 array [N] to which
    each voxel's subdivision priority sum |alpha_i dL/dalpha_i| over these
    pixels is added (Eq. priority, Sec. 3.2.2); with magnitudes also
    "priority_seg", its terms weighted by their segment condition numbers."""
    centre, level, corner, g, s = _scene_arrays(scene, grid, sh)
    n, px = _pixels(cam, pixels)
    if pixels is None:
        g_rgb = np.asarray(g_rgb, np.float64).reshape(3, -1).T
    gn = None
    if g_normal is not None:
        gn = np.asarray(g_normal, np.float64)
        if pixels is None:
            gn = gn.reshape(3, -1).T
        gn = np.ascontiguousarray(gn, np.float64).reshape(n, 3)
    gdist = None if g_dist is None else np.ascontiguousarray(g_dist, np.float64).reshape(n)
    if priority is not None:
        assert priority.dtype == np.float64 and priority.shape == (scene.n_vox,)
        assert priority.flags.c_contiguous
    gr = np.ascontiguousarray(g_rgb, np.float64).reshape(n, 3)
    gd = np.ascontiguousarray(g_depth, np.float64).reshape(n)
    ga = np.ascontiguousarray(g_alpha, np.float64).reshape(n)
    d_grid = np.zeros(len(g))
    d_sh = np.zeros((scene.n_vox, 48))
    want = magnitudes is not None
    a_grid, a_sh = (np.zeros(len(g)), np.zeros((scene.n_vox, 48))) if want else (None, None)
    k_grid, k_sh = (np.zeros(len(g)), np.zeros((scene.n_vox, 48))) if want else (None, None)
    k_pr = np.zeros(scene.n_vox) if (want and priority is not None) else None
    c = camera_struct(cam)
    p = params_struct(K, t_stop, bg)
    rc = lib().oc_render_grad_ex(float(np.float32(scene.world_size)), scene.n_vox, _ptr(centre),
                                 _ptr(level), _ptr(corner), _ptr(g), _ptr(s), ctypes.byref(c),
                                 ctypes.byref(p), n, _ptr(px), _ptr(gr), _ptr(gd), _ptr(ga), _ptr(gn), _ptr(gdist),
                                 _ptr(d_grid), _ptr(d_sh), _ptr(a_grid), _ptr(a_sh), _ptr(k_grid), _ptr(k_sh),
                                 _ptr(priority), _ptr(k_pr), _threads(threads))
    if rc != 0:
        raise RuntimeError(f"oc_render_grad failed ({rc})")
    if magnitudes is not None:
        magnitudes.update(grid=a_grid, sh=a_sh, grid_seg=k_grid, sh_seg=k_sh)
        if k_pr is not None:
            magnitudes["priority_seg"] = k_pr
    return d_grid, d_sh


def trilinear(V, q) -> float:
    """Trilinear interpolation of Eq. (interp) of 8 corner values at q."""
    return lib().oc_trilinear(_ptr(np.ascontiguousarray(V, np.float64)), _ptr(np.ascontiguousarray(q, np.float64)))


def interp_grad_centre(V) -> np.ndarray:
    """Gradient of the trilinear field at the voxel centre, Eq. (interp_grad)."""
    g = np.zeros(3)
    lib().oc_interp_grad_centre(_ptr(np.ascontiguousarray(V, np.float64)), _ptr(g))
    return g


def explin(x: float) -> float:
    return lib().oc_explin(float(x))


def explin_grad(x: float) -> float:
    return lib().oc_explin_grad(float(x))


def sh_basis(d) -> np.ndarray:
    d = np.ascontiguousarray(d, np.float64)
    Y = np.zeros(16)
    lib().oc_sh_basis(_ptr(d), _ptr(Y))
    return Y


def pixel_ray(cam, x, y):
    ro = np.zeros(3)
    rd = np.zeros(3)
    c = camera_struct(cam)
    lib().oc_pixel_ray(ctypes.byref(c), float(x), float(y), _ptr(ro), _ptr(rd))
    return ro, rd


def ray_aabb(centre, size, ro, rd):
    c = np.ascontiguousarray(centre, np.float64)
    o = np.ascontiguousarray(ro, np.float64)
    d = np.ascontiguousarray(rd, np.float64)
    a = ctypes.c_double()
    b = ctypes.c_double()
    valid = lib().oc_ray_aabb(_ptr(c), float(size), _ptr(o), _ptr(d), ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value, bool(valid)


def ray_hits(scene, ro, rd, cap=1 << 16):
    """Valid hits of one ray with every voxel, sorted by (a, b, voxel)."""
    centre = np.ascontiguousarray(scene.centre, np.float32).astype(np.float64)
    level = np.ascontiguousarray(scene.level, np.uint8)
    o = np.ascontiguousarray(ro, np.float64)
    d = np.ascontiguousarray(rd, np.float64)
    a = np.zeros(cap)
    b = np.zeros(cap)
    v = np.zeros(cap, np.int64)
    n = lib().oc_ray_hits(float(np.float32(scene.world_size)), scene.n_vox, _ptr(centre),
                          _ptr(level), _ptr(o), _ptr(d), cap, _ptr(a), _ptr(b), _ptr(v))
    n = min(int(n), cap)
    return a[:n], b[:n], v[:n]
