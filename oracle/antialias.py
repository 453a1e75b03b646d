"""Supersampling anti-aliasing (oracle side, FP64 numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 3.1.2 ("Anti-aliasing"): render at h_ss times the target resolution and
downsample to the target with an anti-aliasing filter (h_ss = 1.5 in the
implementation details, 1.1 in the ablation of the supplementary; the
paper names no filter).  Reading taken: the supersampled image has
round(h_ss W) x round(h_ss H) pixels over the same image plane (intrinsics
scaled by the per-axis ratio s = W_ss / W, so the target pixel x covers the
supersampled interval [s x, s (x + 1))), and the filter is the area
(box) average over that footprint: target pixel x gets the supersampled
pixels X with weight |[X, X + 1) n [s x, s (x + 1))| / s, separably in x and
y.  The backward of the downsampling is the transposed operator.
"""
from __future__ import annotations

import numpy as np


def supersampled_size(width: int, height: int, h_ss: float):
    return int(round(h_ss * width)), int(round(h_ss * height))


def supersampled_camera(cam, h_ss: float):
    """The camera of the supersampled image: same pose, intrinsics scaled by
    W_ss / W in x and H_ss / H in y (pixel edges scale with the image)."""
    import dataclasses
    Ws, Hs = supersampled_size(cam.width, cam.height, h_ss)
    sx, sy = Ws / cam.width, Hs / cam.height
    return dataclasses.replace(cam, fx=np.float32(float(cam.fx) * sx), fy=np.float32(float(cam.fy) * sy),
                               cx=np.float32(float(cam.cx) * sx), cy=np.float32(float(cam.cy) * sy),
                               width=Ws, height=Hs)


def area_weights(n_in: int, n_out: int) -> np.ndarray:
    """[n_out, n_in] 1-D area filter: row x holds, for each input pixel X, the
    length of [X, X + 1) n [s x, s (x + 1)) divided by s = n_in / n_out."""
    s = n_in / n_out
    M = np.zeros((n_out, n_in))
    for x in range(n_out):
        lo, hi = s * x, s * (x + 1)
        for X in range(int(np.floor(lo)), min(n_in, int(np.ceil(hi)))):
            overlap = min(hi, X + 1) - max(lo, X)
            if overlap > 0:
                M[x, X] = overlap / s
    return M


def downsample(img: np.ndarray, height: int, width: int) -> np.ndarray:
    """[..., H_ss, W_ss] -> [..., height, width] by the separable area filter."""
    img = np.asarray(img, np.float64)
    My = area_weights(img.shape[-2], height)
    Mx = area_weights(img.shape[-1], width)
    return My @ img @ Mx.T


def downsample_adjoint(grad: np.ndarray, height_ss: int, width_ss: int) -> np.ndarray:
    """The transposed operator: [..., H, W] -> [..., H_ss, W_ss]."""
    grad = np.asarray(grad, np.float64)
    My = area_weights(height_ss, grad.shape[-2])
    Mx = area_weights(width_ss, grad.shape[-1])
    return My.T @ grad @ Mx
