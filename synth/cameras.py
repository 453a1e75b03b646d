"""Seeded pinhole cameras (OpenCV convention: x right, y down, z forward).

A camera is the intrinsics (fx, fy, cx, cy), the world-to-camera extrinsics
[R | t] (camera point = R @ world point + t) and the image size.  Every value
is stored in float32 because that is what the rasterizer receives; whoever
needs float64 widens these float32 values exactly.

This module only builds inputs.  It holds none of the rasterizer's arithmetic.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Camera:
    fx: np.float32
    fy: np.float32
    cx: np.float32
    cy: np.float32
    w2c: np.ndarray  # float32 [3, 4], row-major [R | t]
    width: int
    height: int

    @property
    def R(self) -> np.ndarray:
        return self.w2c[:, :3]

    @property
    def t(self) -> np.ndarray:
        return self.w2c[:, 3]


def look_at(eye, target, up, fov_x_deg: float, width: int, height: int) -> Camera:
    """Camera at `eye` looking at `target`; `up` is the world up vector.

    The camera y axis points down the image, so it is the negative of `up`
    made orthogonal to the viewing direction.  The focal length follows the
    horizontal field of view: fx = (W / 2) / tan(fov_x / 2), square pixels,
    principal point at the image centre.
    """
    eye = np.asarray(eye, np.float64)
    target = np.asarray(target, np.float64)
    up = np.asarray(up, np.float64)
    z = target - eye
    z /= np.linalg.norm(z)
    x = np.cross(z, up)
    x /= np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    t = -R @ eye
    w2c = np.concatenate([R, t[:, None]], axis=1).astype(np.float32)
    f = 0.5 * width / math.tan(math.radians(fov_x_deg) * 0.5)
    return Camera(np.float32(f), np.float32(f), np.float32(0.5 * width),
                  np.float32(0.5 * height), w2c, int(width), int(height))


def orbit_camera(seed: int, width: int, height: int, distance: float = 2.5,
                 fov_x_deg: float = 50.0, target=(0.5, 0.5, 0.5)) -> Camera:
    """Camera on a sphere of radius `distance` around `target`, looking at it.

    The direction is uniform on the sphere (a normalised standard normal
    draw from numpy's default_rng(seed)).
    """
    rng = np.random.default_rng(seed)
    d = rng.normal(size=3)
    d /= np.linalg.norm(d)
    target = np.asarray(target, np.float64)
    up = np.array([0.0, 1.0, 0.0])
    if abs(float(d @ up)) > 0.99:
        up = np.array([0.0, 0.0, 1.0])
    return look_at(target + distance * d, target, up, fov_x_deg, width, height)


def dense_view_camera(width: int = 128, height: int = 128) -> Camera:
    """The 128x128, 50 degree camera of the dense level-5 workload.

    It sits at distance 2.5 from the cube centre along normalize(0.05, 0.03, -1),
    so the optical axis is close to the world z axis and the image holds tiles
    whose pixel rays disagree in the sign of their x and y components.
    """
    c = np.array([0.5, 0.5, 0.5])
    d = np.array([0.05, 0.03, -1.0])
    d /= np.linalg.norm(d)
    return look_at(c + 2.5 * d, c, (0.0, 1.0, 0.0), 50.0, width, height)
