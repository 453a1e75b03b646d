"""The batched multi-view path against the FP64 oracle directly.

svr_render_batched is captured in a CUDA graph (BatchedRenderer) and
replayed; every view's images are compared with the oracle's brute-force
render of that view at 1e-4, and the gradients summed over the views with
the sum of the oracle's per-view gradients at 1e-3 (per tensor and
elementwise).  Views of mixed resolution, tiles of 8, 16 and 32 pixels, and
a reduced copy of the large batched workload: an octree up to level 11 with
touching leaves at most 4 levels apart, seen by 2560x1440 views, compared on
sampled pixels that include whole tile rows."""
import numpy as np
import pytest

import oracle
import synth
from tests.conftest import cached
from tests.gpu_common import compare_grads, compare_images, oracle_grads, require_gpu

pytestmark = pytest.mark.gpu

SIZES = [(64, 48), (40, 40), (72, 56), (33, 65)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _view(r, out, v, cam):
    """View v of the batch outputs (tensors), shaped like a single view's."""
    a, b = int(r.pixel_base[v]), int(r.pixel_base[v + 1])
    H, W = cam.height, cam.width
    o = {"rgb": out["rgb"][3 * a:3 * b].reshape(3, H, W)}
    for k in ("depth", "alpha", "T_final", "last"):
        o[k] = out[k][a:b].reshape(H, W)
    return o


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_graph_replayed_batch_against_oracle(tile):
    import torch
    from paper_2412_04459_gb300 import DeviceScene
    from paper_2412_04459_gb300.autotune import BatchedRenderer
    sc = cached("batched_oracle_scene", lambda: synth.random_octree_scene(
        27, max_level=5, p_split=0.5, max_cells=1500, grid_fn=synth.normal_grid(2.0, 1.5)))
    cams = [synth.orbit_camera(80 + i, *SIZES[i % len(SIZES)], distance=1.8) for i in range(4)]
    K, bg = 3, (0.1, 0.0, 0.2)
    refs = [cached(("batched_oracle_ref", i), lambda c=c: oracle.render(sc, c, K=K, bg=bg))
            for i, c in enumerate(cams)]
    dev = DeviceScene.from_host(sc)
    r = BatchedRenderer(dev, cams, K=K, tile=tile, bg=bg)
    # upstream gradients, zero on the rounding-sensitive pixels (whose
    # termination may flip) so that both sides differentiate the same walk
    ups = []
    for v, c in enumerate(cams):
        g = synth.upstream_grads(40 + v, c.height, c.width)
        keep = refs[v]["near_stop"] == 0
        ups.append((g[0] * keep[None], g[1] * keep, g[2] * keep))
    for i in range(3):
        r.grads[i].copy_(torch.as_tensor(np.concatenate([u[i].reshape(-1) for u in ups]), device="cuda"))
    r.capture()
    for _ in range(2):                     # replayed twice: the second replay starts from the first's state
        r.step()
    torch.cuda.synchronize()
    flags, pairs = r.status()
    assert flags == 0 and pairs > 0
    og, osh = np.zeros(sc.n_pts), np.zeros((sc.n_vox, 48))
    mg = [np.zeros(sc.n_pts), np.zeros(sc.n_pts)]
    ms = [np.zeros((sc.n_vox, 48)), np.zeros((sc.n_vox, 48))]
    for v, c in enumerate(cams):
        compare_images(_view(r, r.out, v, c), refs[v])
        g, s, m = oracle_grads(sc, c, ups[v][0].astype(np.float64), ups[v][1], ups[v][2], K=K, bg=bg)
        og += g
        osh += s
        mg[0] += m["grid"]
        mg[1] += m["grid_seg"]
        ms[0] += m["sh"]
        ms[1] += m["sh_seg"]
    compare_grads(r.d_grid.cpu().numpy(), og, name="grid", mag=mg)
    compare_grads(r.d_sh.cpu().numpy(), osh, name="sh", mag=ms)


def _tile_row_and_random(cam, tile, n_tiles, n_random, rng):
    """The first n_tiles tiles (all of them: None) of a tile row through the
    middle of the image, plus n_random random pixels."""
    ty = (cam.height // tile) // 2
    xs = np.arange(cam.width if n_tiles is None else min(cam.width, n_tiles * tile))
    ys = np.arange(tile * ty, min(tile * ty + tile, cam.height))
    yy, xx = np.meshgrid(ys, xs, indexing="ij")
    px = [np.stack([xx.ravel(), yy.ravel()], 1)]
    px.append(np.stack([rng.integers(0, cam.width, n_random), rng.integers(0, cam.height, n_random)], 1))
    return np.unique(np.concatenate(px), axis=0)


def _batch_against_oracle(sc, cams, tile, img_px, grad_px, grad_vals):
    """One graph-replayed batched forward + backward of `cams` with upstream
    gradients grad_vals at grad_px (zeroed where the oracle is near the stop
    threshold); images at img_px and the summed gradients against the
    oracle."""
    import torch
    from paper_2412_04459_gb300 import DeviceScene
    from paper_2412_04459_gb300.autotune import BatchedRenderer
    dev = DeviceScene.from_host(sc)
    r = BatchedRenderer(dev, cams, K=3, t_stop=1e-4, tile=tile)
    refs_g = [oracle.render(sc, c, K=3, t_stop=1e-4, pixels=grad_px[v]) for v, c in enumerate(cams)]
    for v, c in enumerate(cams):
        keep = refs_g[v]["near_stop"] == 0
        grad_vals[v][~keep] = 0.0
        a = int(r.pixel_base[v])
        lin = grad_px[v][:, 1] * c.width + grad_px[v][:, 0]
        HW = c.width * c.height
        for ch in range(3):
            r.grads[0][3 * a + ch * HW + lin] = torch.as_tensor(grad_vals[v][:, ch], dtype=torch.float32,
                                                                device="cuda")
        r.grads[1][a + lin] = torch.as_tensor(grad_vals[v][:, 3], dtype=torch.float32, device="cuda")
        r.grads[2][a + lin] = torch.as_tensor(grad_vals[v][:, 4], dtype=torch.float32, device="cuda")
    r.capture()
    r.step()
    torch.cuda.synchronize()
    flags, pairs = r.status()
    assert flags == 0 and pairs > 10 ** 6
    og, osh = np.zeros(sc.n_pts), np.zeros((sc.n_vox, 48))
    mg = [np.zeros(sc.n_pts), np.zeros(sc.n_pts)]
    ms = [np.zeros((sc.n_vox, 48)), np.zeros((sc.n_vox, 48))]
    for v, c in enumerate(cams):
        ref = oracle.render(sc, c, K=3, t_stop=1e-4, pixels=img_px[v])
        compare_images(_view(r, r.out, v, c), ref, pixels=img_px[v])
        g, s, m = oracle_grads(sc, c, grad_vals[v][:, :3], grad_vals[v][:, 3], grad_vals[v][:, 4], K=3,
                               t_stop=1e-4, pixels=grad_px[v])
        og += g
        osh += s
        mg[0] += m["grid"]
        mg[1] += m["grid_seg"]
        ms[0] += m["sh"]
        ms[1] += m["sh_seg"]
    compare_grads(r.d_grid.cpu().numpy(), og, name="grid", mag=mg)
    compare_grads(r.d_sh.cpu().numpy(), osh, name="sh", mag=ms)
    return pairs


def _grad_pixels(cams, n, rng):
    px, vals = [], []
    for c in cams:
        gp = np.unique(np.stack([rng.integers(0, c.width, n), rng.integers(0, c.height, n)], 1), axis=0)
        px.append(gp)
        vals.append(rng.normal(size=(len(gp), 5)))
    return px, vals


def test_reduced_large_workload_against_oracle():
    """The large batched workload's structure at reduced size: three noisy
    shells, leaves of levels 4..11 with touching leaves at most 4 levels
    apart (146,504 voxels), three 2560x1440 orbit views, K = 3, t_stop =
    1e-4, forward + backward in one graph-replayed batch.  Images on a whole
    tile row of the first view, 16 tiles of a row of the others, and random
    pixels; gradients from the upstream gradients of random pixels."""
    sc = cached("three_shell_reduced", lambda: synth.shell_scene(0, 146_504, p_split=0.25,
                                                                spec=synth.scenes.SHELL_THREE))
    assert sc.max_level == 11 and sc.n_vox > 100_000
    cams = [synth.orbit_camera(200 + v, 2560, 1440) for v in range(3)]
    rng = np.random.default_rng(12)
    img_px = [_tile_row_and_random(c, 16, None if v == 0 else 16, 1500, rng) for v, c in enumerate(cams)]
    grad_px, grad_vals = _grad_pixels(cams, 1500, rng)
    _batch_against_oracle(sc, cams, 16, img_px, grad_px, grad_vals)


def test_large_workload_full_size_sampled():
    """The large batched workload at full size, in the launch configuration
    bench.py times (tile 16, one partition): the ~8M-voxel three-shell octree
    (levels 4..11, touching leaves at most 4 levels apart), the bench's eight
    2560x1440 orbit views, K = 3, t_stop = 1e-4, one graph-replayed batched
    forward + backward.  Images on 4 tiles of a tile row of every view plus
    random pixels; gradients from the upstream gradients of random pixels of
    every view (the oracle tests every voxel against every sampled ray)."""
    sc = cached("three_shell_8m", lambda: synth.shell_scene(0, 8_000_000, spec=synth.scenes.SHELL_THREE))
    assert sc.max_level == 11 and sc.n_vox > 8_000_000
    cams = [synth.orbit_camera(200 + v, 2560, 1440) for v in range(8)]
    rng = np.random.default_rng(13)
    img_px = [_tile_row_and_random(c, 16, 4, 192, rng) for c in cams]
    grad_px, grad_vals = _grad_pixels(cams, 192, rng)
    pairs = _batch_against_oracle(sc, cams, 16, img_px, grad_px, grad_vals)
    assert pairs > 5 * 10 ** 7
