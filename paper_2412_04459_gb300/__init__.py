"""GB300-native (sm_103a) hot path of SVRaster (arXiv 2412.04459): sparse-voxel
rasterization forward and backward behind the C ABI of include/svr.h.

The package holds the CUDA sources (csrc/), their in-tree build (build.py ->
libsvr.so), the ctypes binding (_native.py), the PyTorch front end
(raster.py: DeviceScene, Frame, rasterize, l2_loss) and the batched
multi-view runner with its autotuner (autotune.py).  Importing it does not
build or load the library; the first call that needs it loads libsvr.so and
fails loudly if it is missing.
"""
from .raster import (DeviceScene, Frame, SVRasterFn, camera_struct, l2_loss,  # noqa: F401
                     params_struct, rasterize, workspace_size)

__all__ = ["DeviceScene", "Frame", "SVRasterFn", "rasterize", "l2_loss", "camera_struct", "params_struct",
           "workspace_size"]
