"""svr_render_fwd_static: the forward render for callers that may not allocate
device memory themselves (the scratch lives in a fixed array inside the
library).  Its images must equal those of the regular path
(svr_preprocess + svr_bin_sort + svr_render_fwd with a caller workspace) on
two calls in a row, so nothing a call leaves in the shared array leaks into
the next.  Kept in its own file, collected last."""
import ctypes

import numpy as np
import pytest

import synth
from tests.gpu_common import IMG_TOL, require_gpu

pytestmark = pytest.mark.gpu


def _static_call(scene_dev, cam, K, t_stop, bg, tile=16):
    """(return code, outputs as numpy, pair count) of one call."""
    import torch
    from paper_2412_04459_gb300 import _native as N
    from paper_2412_04459_gb300.raster import camera_struct, params_struct
    H, W = cam.height, cam.width
    out = dict(rgb=torch.empty(3, H, W, device="cuda"), depth=torch.empty(H, W, device="cuda"),
               alpha=torch.empty(H, W, device="cuda"), T_final=torch.empty(H, W, device="cuda"),
               last=torch.empty(H, W, dtype=torch.int32, device="cuda"))
    sc = scene_dev.struct()
    c = camera_struct(cam)
    p = params_struct(K, t_stop, tile, bg)
    n = ctypes.c_int64(-1)
    ptr = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = N.lib().svr_render_fwd_static(N.ref(sc), N.ref(c), N.ref(p), ptr(out["rgb"]), ptr(out["depth"]),
                                        ptr(out["alpha"]), ptr(out["T_final"]), ptr(out["last"]), N.ref(n),
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, {k: v.cpu().numpy() for k, v in out.items()}, n.value


def _static_render(scene_dev, cam, K, t_stop, bg):
    from paper_2412_04459_gb300 import _native as N
    rc, out, n = _static_call(scene_dev, cam, K, t_stop, bg)
    N.check(rc, "svr_render_fwd_static")
    return out, n


def _regular_render(scene_dev, cam, K, t_stop, bg):
    from paper_2412_04459_gb300 import Frame
    fr = Frame(scene_dev, cam, K=K, t_stop=t_stop, bg=bg)
    out = fr.render()
    return {k: v.cpu().numpy() for k, v in out.items()}, fr.n_pairs


def test_static_workspace_matches_caller_workspace_twice():
    require_gpu()
    from paper_2412_04459_gb300 import DeviceScene
    cases = [
        (synth.dense_scene(4, seed=3), synth.dense_view_camera(96, 80), 3, 1e-4, (0.0, 0.0, 0.0)),
        (synth.random_octree_scene(8, max_level=5, p_split=0.5, grid_fn=synth.normal_grid(2.0, 1.0)),
         synth.orbit_camera(12, 72, 56, distance=1.7), 1, 1e-3, (0.2, 0.1, 0.3)),
    ]
    for scene, cam, K, t_stop, bg in cases:
        dev = DeviceScene.from_host(scene)
        got, n_static = _static_render(dev, cam, K, t_stop, bg)
        ref, n_regular = _regular_render(dev, cam, K, t_stop, bg)
        assert n_static == n_regular > 0
        for k in ("rgb", "depth", "alpha", "T_final"):
            assert np.abs(got[k] - ref[k]).max() <= IMG_TOL, k
        assert np.array_equal(got["last"], ref["last"])


def test_static_workspace_rejects_oversized_scenes():
    require_gpu()
    from paper_2412_04459_gb300 import DeviceScene, _native as N
    scene = synth.dense_scene(6, seed=0)              # 262144 voxels > 65536
    dev = DeviceScene.from_host(scene)
    with pytest.raises(N.SvrError) as e:
        _static_render(dev, synth.dense_view_camera(), 1, 1e-4, (0.0, 0.0, 0.0))
    assert e.value.code == N.SVR_ERR_LIMIT
    assert "65536" in str(e.value)


def test_static_workspace_reports_pair_overflow():
    """32,768 voxels (within the voxel limit) filling a 1280x840 view make
    more pairs than fit in the array: the call returns SVR_ERR_CAPACITY,
    skips the render, and reports the true pair count, which equals the
    regular path's."""
    require_gpu()
    from paper_2412_04459_gb300 import DeviceScene, _native as N
    scene = synth.dense_scene(5, seed=1)
    cam = synth.orbit_camera(3, 1280, 840, distance=1.2)
    dev = DeviceScene.from_host(scene)
    rc, _, n_static = _static_call(dev, cam, 1, 1e-4, (0.0, 0.0, 0.0))
    assert rc == N.SVR_ERR_CAPACITY
    _, n_regular = _regular_render(dev, cam, 1, 1e-4, (0.0, 0.0, 0.0))
    assert n_static == n_regular > 0
    # the array still serves a call that fits, right after the overflow
    small = synth.dense_view_camera(96, 80)
    got, _ = _static_render(dev, small, 1, 1e-4, (0.0, 0.0, 0.0))
    ref, _ = _regular_render(dev, small, 1, 1e-4, (0.0, 0.0, 0.0))
    assert np.abs(got["rgb"] - ref["rgb"]).max() <= IMG_TOL


def test_static_workspace_rejects_too_many_tiles():
    """An image of more than 2^16 tiles is reported as the tile limit."""
    require_gpu()
    from paper_2412_04459_gb300 import DeviceScene, _native as N
    dev = DeviceScene.from_host(synth.dense_scene(2, seed=0))
    cam = synth.orbit_camera(0, 4200, 4200)          # 263 x 263 tiles of 16 pixels
    with pytest.raises(N.SvrError) as e:
        _static_render(dev, cam, 1, 1e-4, (0.0, 0.0, 0.0))
    assert e.value.code == N.SVR_ERR_LIMIT
    assert "tiles" in str(e.value)
