"""Backward parity: the CUDA back-to-front backward (through the C ABI) vs the
oracle's FP64 analytic gradient, which the CPU tests pin to finite
differences; and the autograd front end."""
import numpy as np
import pytest

import oracle
import synth
from tests.conftest import cached
from tests.gpu_common import compare_grads, oracle_grads, require_gpu, run_gpu, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _grads(scene, cam, K, t_stop, bg, seed, ref_stop=None):
    import torch
    fr, out, _ = run_gpu(scene, cam, K=K, t_stop=t_stop, bg=bg, inspect=False)
    g_rgb, g_depth, g_alpha = synth.upstream_grads(seed, cam.height, cam.width)
    if ref_stop is not None:
        # pixels whose transmittance grazes the threshold have a jump there
        keep = ref_stop == 0
        g_rgb = g_rgb * keep[None]
        g_depth = g_depth * keep
        g_alpha = g_alpha * keep
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    d_grid, d_sh = fr.backward(t(g_rgb), t(g_depth), t(g_alpha), out)
    og, osh, mag = oracle_grads(scene, cam, g_rgb.astype(np.float64), g_depth, g_alpha, K=K,
                                t_stop=t_stop, bg=bg)
    return d_grid.cpu().numpy(), d_sh.cpu().numpy(), og, osh, mag


@pytest.mark.parametrize("K", [1, 2, 3])
@pytest.mark.parametrize("seed", [0, 1])
def test_tiny_gradients(K, seed):
    sc = synth.random_octree_scene(seed + 20, max_level=4, p_split=0.5, max_cells=64,
                                   grid_fn=synth.normal_grid(1.0, 1.5))
    cam = synth.orbit_camera(seed + 3, 48, 40, distance=1.7)
    bg = (0.1, 0.2, 0.3) if seed else (0.0, 0.0, 0.0)
    ref = oracle.render(sc, cam, K=K, t_stop=1e-4, bg=bg)
    dg, ds, og, osh, mag = _grads(sc, cam, K, 1e-4, bg, seed, ref["near_stop"])
    compare_grads(dg, og, name="grid", mag=(mag["grid"], mag["grid_seg"]))
    compare_grads(ds, osh, name="sh", mag=(mag["sh"], mag["sh_seg"]))


@pytest.mark.parametrize("K", [1, 3])
def test_dense_level5_gradients(K):
    sc = cached("dense5", lambda: synth.dense_scene(5, seed=0))
    cam = synth.dense_view_camera()
    ref = cached(("dense5_ref", K), lambda: oracle.render(sc, cam, K=K, t_stop=1e-4))
    dg, ds, og, osh, mag = _grads(sc, cam, K, 1e-4, (0.0, 0.0, 0.0), 5, ref["near_stop"])
    compare_grads(dg, og, name="grid", mag=(mag["grid"], mag["grid_seg"]))
    compare_grads(ds, osh, name="sh", mag=(mag["sh"], mag["sh_seg"]))


def test_terminated_pixels_gradients():
    """Opaque scene: most pixels stop early; the backward starts at `last`."""
    sc = synth.random_octree_scene(31, max_level=4, p_split=0.4,
                                   grid_fn=synth.normal_grid(12.0, 2.0))
    cam = synth.orbit_camera(6, 40, 40, distance=1.6)
    ref = oracle.render(sc, cam, K=3, t_stop=1e-3)
    assert (ref["term_vox"] >= 0).mean() > 0.2
    dg, ds, og, osh, mag = _grads(sc, cam, 3, 1e-3, (0.0, 0.0, 0.0), 2, ref["near_stop"])
    compare_grads(dg, og, name="grid", mag=(mag["grid"], mag["grid_seg"]))
    compare_grads(ds, osh, name="sh", mag=(mag["sh"], mag["sh_seg"]))


def test_underflowing_transmittance_takes_front_to_back_phase():
    """Densities so high that T_final underflows to 0 (t_stop = 0): the
    back-to-front division is impossible and the kernel's front-to-back
    phase must give the same gradients."""
    def grid_fn(pos, rng):
        dense = rng.random(len(pos)) < 0.3
        return np.where(dense, 400.0, rng.normal(0.5, 1.0, size=len(pos)))
    sc = synth.random_octree_scene(41, max_level=3, p_split=0.4, max_cells=60, grid_fn=grid_fn)
    cam = synth.orbit_camera(8, 32, 32, distance=1.6)
    fr, out, _ = run_gpu(sc, cam, K=2, t_stop=0.0, inspect=False)
    T = to_np(out)["T_final"]
    assert (T < 1e-30).mean() > 0.05
    dg, ds, og, osh, mag = _grads(sc, cam, 2, 0.0, (0.2, 0.2, 0.2), 4)
    assert np.isfinite(dg).all() and np.isfinite(ds).all()
    compare_grads(dg, og, name="grid", mag=(mag["grid"], mag["grid_seg"]))
    compare_grads(ds, osh, name="sh", mag=(mag["sh"], mag["sh_seg"]))


def test_l2_loss_kernel():
    """svr_l2_loss: sum (p - t)^2 / n and 2 (p - t) / n, against numpy in FP64,
    on a size with a ragged last block and on an empty input."""
    import torch
    from paper_2412_04459_gb300 import l2_loss
    rng = np.random.default_rng(0)
    for n in (3 * 37 * 53, 1, 1 << 20):
        p = rng.normal(size=n).astype(np.float32)
        t = rng.normal(size=n).astype(np.float32)
        loss, grad = l2_loss(torch.as_tensor(p, device="cuda"), torch.as_tensor(t, device="cuda"))
        d = p.astype(np.float64) - t.astype(np.float64)
        assert abs(float(loss.item()) - float((d * d).mean())) <= 1e-5 * float((d * d).mean())
        assert np.allclose(grad.cpu().numpy(), 2 * d / n, rtol=1e-6, atol=1e-12)
    loss, _ = l2_loss(torch.empty(0, device="cuda"), torch.empty(0, device="cuda"))
    assert float(loss.item()) == 0.0


def test_autograd_matches_frame_backward_and_l2_loss():
    """rasterize() under autograd: an L2 loss against a target rendered from
    perturbed densities.  The gradients equal the oracle's for the upstream
    gradient this loss hands the backward (2 (C - C*) / n of the rendered
    images), and, through the oracle's own images, for the whole loss."""
    import torch
    from paper_2412_04459_gb300 import DeviceScene, rasterize
    sc = synth.random_octree_scene(51, max_level=4, p_split=0.5, max_cells=64,
                                   grid_fn=synth.normal_grid(1.5, 1.0))
    cam = synth.orbit_camera(10, 40, 32, distance=1.7)
    dev = DeviceScene.from_host(sc)
    rng = np.random.default_rng(1)
    target_grid = torch.as_tensor(sc.grid + 0.1 * rng.normal(size=sc.n_pts).astype(np.float32), device="cuda")
    with torch.no_grad():
        target, _, _ = rasterize(target_grid, dev.sh, dev, cam, K=3)
    grid = dev.grid.clone().requires_grad_(True)
    sh = dev.sh.clone().requires_grad_(True)
    rgb, depth, alpha = rasterize(grid, sh, dev, cam, K=3)
    loss = ((rgb - target) ** 2).mean()
    loss.backward()
    zeros = np.zeros((cam.height, cam.width))
    # the backward for the upstream gradient the loss produced
    g_up = (2.0 * (rgb.detach() - target) / rgb.numel()).cpu().numpy().astype(np.float64)
    og, osh, mag = oracle_grads(sc, cam, g_up, zeros, zeros, K=3)
    compare_grads(grid.grad.cpu().numpy(), og, name="grid", mag=(mag["grid"], mag["grid_seg"]))
    compare_grads(sh.grad.cpu().numpy(), osh, name="sh", mag=(mag["sh"], mag["sh_seg"]))
    # the whole loss through the oracle: dL/dC = 2 (C - C*) / (3 H W)
    ref = oracle.render(sc, cam, K=3)
    tgt = oracle.render(sc, cam, K=3, grid=target_grid.cpu().numpy().astype(np.float64))
    assert not ref["near_stop"].any() and not tgt["near_stop"].any()
    g_rgb = 2.0 * (ref["rgb"] - tgt["rgb"]) / ref["rgb"].size
    og, osh, mag = oracle_grads(sc, cam, g_rgb, zeros, zeros, K=3)
    compare_grads(grid.grad.cpu().numpy(), og, name="grid (oracle images)", mag=(mag["grid"], mag["grid_seg"]))
    compare_grads(sh.grad.cpu().numpy(), osh, name="sh (oracle images)", mag=(mag["sh"], mag["sh_seg"]))
    assert abs(loss.item() - float(((ref["rgb"] - tgt["rgb"]) ** 2).mean())) < 1e-6


def test_autograd_with_expanded_upstream_gradients():
    """rgb.sum() + depth.sum() + alpha.sum() hands the backward expanded
    (stride-0) gradients for all three images, which the front end copies to
    contiguous buffers; the result equals the backward of the same loss given
    contiguous ones-tensors."""
    import torch
    from paper_2412_04459_gb300 import DeviceScene, Frame, rasterize
    sc = synth.random_octree_scene(53, max_level=4, p_split=0.5, max_cells=64,
                                   grid_fn=synth.normal_grid(1.5, 1.0))
    cam = synth.orbit_camera(12, 48, 40, distance=1.7)
    dev = DeviceScene.from_host(sc)
    grid = dev.grid.clone().requires_grad_(True)
    sh = dev.sh.clone().requires_grad_(True)
    for _ in range(2):              # the second pass reuses the allocator's freed blocks
        grid.grad = None
        sh.grad = None
        rgb, depth, alpha = rasterize(grid, sh, dev, cam, K=2)
        (rgb.sum() + depth.sum() + alpha.sum()).backward()
    fr = Frame(dev, cam, K=2)
    out = fr.render()
    ones = lambda *s: torch.ones(*s, device="cuda")
    dg, ds = fr.backward(ones(3, cam.height, cam.width), ones(cam.height, cam.width),
                         ones(cam.height, cam.width), out)
    assert torch.allclose(grid.grad, dg, rtol=1e-5, atol=1e-6 * float(dg.abs().max()))
    assert torch.allclose(sh.grad, ds, rtol=1e-5, atol=1e-6 * float(ds.abs().max()))
    g = np.ones((3, cam.height, cam.width))
    og, osh, mag = oracle_grads(sc, cam, g, g[0], g[0], K=2)
    compare_grads(dg.cpu().numpy(), og, name="grid", mag=(mag["grid"], mag["grid_seg"]))
    compare_grads(ds.cpu().numpy(), osh, name="sh", mag=(mag["sh"], mag["sh_seg"]))
