"""Supersampling anti-aliasing (Sec. 3.1.2) on the GPU against the oracle:
the area-filter kernels (svr_downsample and its backward) against the FP64
operator, and whole supersampled renders, batched over views of mixed size,
forward and backward, against the oracle's render of the same supersampled
cameras followed by its own downsampling."""
import numpy as np
import pytest

import oracle
import synth
from oracle import antialias
from tests.gpu_common import (IMG_TOL, compare_grads, near_stop_allowance, oracle_grads, require_gpu)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


@pytest.mark.parametrize("H,W,Hs,Ws", [(84, 128, 92, 141), (40, 64, 60, 96), (33, 17, 66, 34), (9, 11, 36, 44),
                                       (21, 30, 21, 30), (840, 1280, 924, 1408)])
def test_kernels_against_the_operator(H, W, Hs, Ws):
    import torch
    from paper_2412_04459_gb300.raster import downsample, downsample_bwd
    rng = np.random.default_rng(H + W)
    src = rng.normal(size=(3, Hs, Ws)).astype(np.float32)
    got = downsample(torch.as_tensor(src, device="cuda"), H, W).cpu().numpy()
    want = antialias.downsample(src.astype(np.float64), H, W)
    assert np.abs(got - want).max() <= 2e-6 * max(1.0, np.abs(want).max())
    g = rng.normal(size=(3, H, W)).astype(np.float32)
    got_b = downsample_bwd(torch.as_tensor(g, device="cuda"), Hs, Ws).cpu().numpy()
    want_b = antialias.downsample_adjoint(g.astype(np.float64), Hs, Ws)
    assert np.abs(got_b - want_b).max() <= 2e-6 * max(1.0, np.abs(want_b).max())


def test_ratio_limits():
    import torch
    from paper_2412_04459_gb300 import _native as N
    from paper_2412_04459_gb300.raster import downsample
    with pytest.raises(N.SvrError) as e:
        downsample(torch.zeros(1, 10, 10, device="cuda"), 11, 10)       # upsampling
    assert e.value.code == N.SVR_ERR_INVALID
    with pytest.raises(N.SvrError):
        downsample(torch.zeros(1, 50, 50, device="cuda"), 10, 10)       # ratio 5 > 4


@pytest.mark.parametrize("h_ss", [1.1, 1.5])
def test_supersampled_batch_against_oracle(h_ss):
    """Three views of mixed size rendered as one batch at h_ss times their
    size, each downsampled; images at 1e-4 and gradients (through the
    downsampling's transpose and the render backward) at the gradient bars
    against the oracle's supersampled renders and its own filter."""
    import torch
    from paper_2412_04459_gb300 import DeviceScene, Frame
    from paper_2412_04459_gb300.raster import downsample, downsample_bwd, supersampled_camera
    sc = synth.random_octree_scene(81, max_level=4, p_split=0.5, max_cells=400, grid_fn=synth.normal_grid(1.5, 1.5))
    cams = [synth.orbit_camera(90 + i, *wh, distance=1.8) for i, wh in enumerate([(48, 40), (64, 36), (30, 50)])]
    ss_cams = [supersampled_camera(c, h_ss) for c in cams]
    for c, s in zip(cams, ss_cams):                       # the product and the oracle agree on the cameras
        o = antialias.supersampled_camera(c, h_ss)
        assert (s.width, s.height, float(s.fx), float(s.cx)) == (o.width, o.height, float(o.fx), float(o.cx))
    dev = DeviceScene.from_host(sc)
    fr = Frame(dev, ss_cams, K=2)
    out = fr.render()
    views = fr.views(out)
    rng = np.random.default_rng(4)
    d_grid = torch.zeros(sc.n_pts, device="cuda")
    ups = [[], [], []]
    og, osh = np.zeros(sc.n_pts), np.zeros((sc.n_vox, 48))
    mg, ms = [np.zeros(sc.n_pts), np.zeros(sc.n_pts)], [np.zeros((sc.n_vox, 48)), np.zeros((sc.n_vox, 48))]
    for v, (c, s) in enumerate(zip(cams, ss_cams)):
        lo = {k: downsample(views[v][k].contiguous(), c.height, c.width) for k in ("rgb", "depth", "alpha")}
        ref = oracle.render(sc, s, K=2)
        keep_ss = (ref["near_stop"] == 0).astype(np.float64)
        # target pixels whose footprint holds a rounding-sensitive pixel are left out
        keep = antialias.downsample(keep_ss, c.height, c.width) > 1 - 1e-9
        assert (~keep).sum() <= near_stop_allowance(keep.size)
        for k, planes in (("rgb", ref["rgb"]), ("depth", ref["depth"]), ("alpha", ref["alpha"])):
            want = antialias.downsample(planes, c.height, c.width)
            err = np.abs(lo[k].cpu().numpy() - want)[..., keep].max()
            assert err <= IMG_TOL, (v, k, err)
        # backward: upstream on the target image, zero where left out
        g = [rng.normal(size=(3, c.height, c.width)) * keep, rng.normal(size=(c.height, c.width)) * keep,
             rng.normal(size=(c.height, c.width)) * keep]
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")
        g_ss = [downsample_bwd(t(x), s.height, s.width) for x in g]
        for i in range(3):
            ups[i].append(g_ss[i].reshape(-1))
        g64 = [antialias.downsample_adjoint(x.astype(np.float32).astype(np.float64), s.height, s.width) for x in g]
        a, b, m = oracle_grads(sc, s, g64[0], g64[1], g64[2], K=2)
        og += a
        osh += b
        mg[0] += m["grid"]
        mg[1] += m["grid_seg"]
        ms[0] += m["sh"]
        ms[1] += m["sh_seg"]
    dg, dsh = fr.backward(torch.cat(ups[0]), torch.cat(ups[1]), torch.cat(ups[2]), out, d_grid)
    compare_grads(dg.cpu().numpy(), og, name="grid", mag=mg)
    compare_grads(dsh.cpu().numpy(), osh, name="sh", mag=ms)
