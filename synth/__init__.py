"""Seeded synthetic inputs for the sparse-voxel rasterizer: scenes, cameras and
upstream gradients.  Shared by the FP64 oracle and the CUDA path as data; it
holds none of the rasterizer's arithmetic."""
from .cameras import Camera, dense_view_camera, look_at, orbit_camera  # noqa: F401
from .scenes import (Scene, calibrate_shell, constant_grid, dense_scene,  # noqa: F401
                     normal_grid, random_octree_scene, shell_scene, subscene,
                     upstream_grads, SHELL_ONE, SHELL_THREE)
