"""Parity at the benchmark's full size: the ~1M-voxel shell scene, the
1280x840 camera of bench.py's rank 0, K = 3, in the launch configuration the
bench times.  Integer outputs are compared in full; images and gradients on
sampled pixels the oracle computes one by one (a full tile row through the
middle of the image plus random pixels)."""
import numpy as np
import pytest

import oracle
import synth
from tests.conftest import cached
from tests.gpu_common import (compare_grads, compare_images, compare_integers, oracle_grads, require_gpu,
                              run_gpu, to_np)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def shell():
    require_gpu()
    scene = cached("shell1m", lambda: synth.shell_scene(seed=0))
    cam = synth.orbit_camera(100, 1280, 840)
    fr, out, ins = run_gpu(scene, cam, K=3, t_stop=1e-4)
    return scene, cam, fr, out, ins


def _pixels(cam, n_random=2048, seed=0):
    rng = np.random.default_rng(seed)
    ty = cam.height // 32                       # tile row in the middle of the image
    ys, xs = np.meshgrid(np.arange(16 * ty, 16 * ty + 16), np.arange(cam.width), indexing="ij")
    row = np.stack([xs.ravel(), ys.ravel()], 1)
    rnd = np.stack([rng.integers(0, cam.width, n_random), rng.integers(0, cam.height, n_random)], 1)
    return row, rnd


def test_integers_full_size(shell):
    scene, cam, fr, out, ins = shell
    n_diff, n_either = compare_integers(scene, cam, ins)
    _, amb = oracle.binning.voxel_rects(scene, cam)
    assert n_diff <= amb.sum()
    assert ins["n_pairs"] > 10 ** 6


def test_images_full_size_sampled(shell):
    scene, cam, fr, out, ins = shell
    row, rnd = _pixels(cam)
    px = np.concatenate([row, rnd])
    ref = oracle.render(scene, cam, K=3, t_stop=1e-4, pixels=px)
    compare_images(out, ref, pixels=px)
    # the forward's own work count agrees with the oracle's composited hits
    st = to_np(fr.forward_stats())
    hits = st["counts"][px[:, 1], px[:, 0], 1]
    assert abs(int(hits.sum()) - int(ref["n_comp"].sum())) <= 1e-3 * ref["n_comp"].sum() + 2
    assert np.array_equal(st["rgb"], to_np(out)["rgb"])


def test_gradients_full_size_sampled(shell):
    import torch
    scene, cam, fr, out, ins = shell
    _, rnd = _pixels(cam, n_random=3000, seed=1)
    rnd = np.unique(rnd, axis=0)
    rng = np.random.default_rng(2)
    H, W = cam.height, cam.width
    g_rgb = np.zeros((3, H, W), np.float32)
    g_d = np.zeros((H, W), np.float32)
    g_a = np.zeros((H, W), np.float32)
    vals = rng.normal(size=(len(rnd), 5)).astype(np.float32)
    g_rgb[:, rnd[:, 1], rnd[:, 0]] = vals[:, :3].T
    g_d[rnd[:, 1], rnd[:, 0]] = vals[:, 3]
    g_a[rnd[:, 1], rnd[:, 0]] = vals[:, 4]
    t = lambda a: torch.as_tensor(a, device="cuda")
    d_grid, d_sh = fr.backward(t(g_rgb), t(g_d), t(g_a), out)
    og, osh, mag = oracle_grads(scene, cam, vals[:, :3].astype(np.float64), vals[:, 3], vals[:, 4],
                                K=3, t_stop=1e-4, pixels=rnd)
    compare_grads(d_grid.cpu().numpy(), og, name="grid", mag=(mag["grid"], mag["grid_seg"]))
    compare_grads(d_sh.cpu().numpy(), osh, name="sh", mag=(mag["sh"], mag["sh_seg"]))
