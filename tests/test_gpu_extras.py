"""The extra outputs of svr_render_fwd_ex / svr_render_bwd_ex against the FP64
oracle: the normal image (Eq. vox_normal) and its gradient (Eq.
interp_grad_grad through the normalisation), the per-voxel maximum blending
weight (pruning) and subdivision priority (Eq. priority) of Sec. 3.2.2.

Images and weights are held to 1e-4 absolute like the colour image, the
normal gradient to the gradient bars, the priority (a sum of non-negative
terms) to 1e-3 relative per tensor and elementwise.  Cases cover tiny random
octrees, the dense level-5 grid, and tile lists split into segments (where
the maximum weights need the forward's second walk from the true
transmittance)."""
import numpy as np
import pytest

import oracle
import synth
from tests.conftest import cached
from tests.gpu_common import (IMG_TOL, SEG_REL, compare_grads, compare_images, near_stop_allowance,
                              oracle_grads, require_gpu)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _back_heavy(front, back_mean, back_std=2.0, z_cut=0.5):
    def grid_fn(pos, rng):
        out = np.full(len(pos), front, dtype=np.float64)
        far = pos[:, 2] >= z_cut
        out[far] = rng.normal(back_mean, back_std, size=int(far.sum()))
        return out
    return grid_fn


CASES = {
    "tiny": (lambda: synth.random_octree_scene(71, max_level=4, p_split=0.5, max_cells=64,
                                               grid_fn=synth.normal_grid(1.0, 1.5)),
             lambda: synth.orbit_camera(13, 48, 40, distance=1.7), 3, 1e-4),
    "dense5": (lambda: cached("dense5", lambda: synth.dense_scene(5, seed=0)),
               lambda: synth.dense_view_camera(), 1, 1e-4),
    "split": (lambda: cached("dense5_backheavy", lambda: synth.dense_scene(5, seed=3,
                                                                           grid_fn=_back_heavy(-4.0, 40.0, 5.0))),
              lambda: synth.dense_view_camera(), 2, 1e-3),
}


def _frame(name):
    from paper_2412_04459_gb300 import DeviceScene, Frame
    make_scene, make_cam, K, t_stop = CASES[name]
    sc, cam = make_scene(), make_cam()
    dev = DeviceScene.from_host(sc)
    fr = Frame(dev, cam, K=K, t_stop=t_stop)
    fr.preprocess()
    fr.bin_sort()
    return sc, cam, dev, fr, K, t_stop


@pytest.mark.parametrize("name", list(CASES))
def test_normal_image_and_max_weight(name):
    import torch
    sc, cam, dev, fr, K, t_stop = _frame(name)
    mw = torch.zeros(sc.n_vox, device="cuda")
    out = fr.forward_ex(normal=True, max_weight=mw)
    mw_ref = np.zeros(sc.n_vox)
    ref = oracle.render(sc, cam, K=K, t_stop=t_stop, normals=True, max_weight=mw_ref)
    compare_images(out, ref)
    keep = ref["near_stop"] == 0
    err_n = np.abs(out["normal"].cpu().numpy() - ref["normal"])[:, keep].max()
    assert err_n <= IMG_TOL, err_n
    # the plain forward gives the same images up to rounding: the kernel
    # variants contract the same arithmetic differently, and with maximum
    # weights a split list is composited by one walk instead of merged
    # segments (another association of the same sums)
    plain = fr.forward()
    for k in ("rgb", "depth", "alpha", "T_final"):
        assert torch.allclose(plain[k], out[k], rtol=0, atol=1e-5), k
    err_w = np.abs(mw.cpu().numpy() - mw_ref)
    print(f"PARITY max_weight {name}: {err_w.max():.3e}, voxels with weight {(mw_ref > 0).sum()}")
    assert err_w.max() <= IMG_TOL, (err_w.max(), int(np.argmax(err_w)))
    assert (mw_ref > 0.05).sum() > 10
    if name == "split":
        ins = fr.inspect()
        lens = np.diff(ins["ranges"].astype(np.int64), axis=1)
        assert lens.max() > 1024                  # split lists: weights from the second walk


def test_max_weight_accumulates_over_views_and_calls():
    """Raised, never lowered, over views and over calls: two views of the tiny
    scene give the oracle's maximum over both, and a repeated call changes
    nothing."""
    import torch
    from paper_2412_04459_gb300 import DeviceScene, Frame
    sc = CASES["tiny"][0]()
    dev = DeviceScene.from_host(sc)
    cams = [synth.orbit_camera(13, 48, 40, distance=1.7), synth.orbit_camera(14, 40, 56, distance=1.5)]
    mw = torch.zeros(sc.n_vox, device="cuda")
    mw_ref = np.zeros(sc.n_vox)
    for cam in cams:
        fr = Frame(dev, cam, K=3)
        fr.preprocess()
        fr.bin_sort()
        fr.forward_ex(max_weight=mw)
        oracle.render(sc, cam, K=3, max_weight=mw_ref)
    before = mw.clone()
    fr.forward_ex(max_weight=mw)
    assert torch.equal(before, mw)
    assert np.abs(mw.cpu().numpy() - mw_ref).max() <= IMG_TOL


@pytest.mark.parametrize("name", list(CASES))
def test_normal_gradient_and_priority(name):
    import torch
    sc, cam, dev, fr, K, t_stop = _frame(name)
    out = fr.forward_ex(normal=True)
    ref = oracle.render(sc, cam, K=K, t_stop=t_stop)
    keep = ref["near_stop"] == 0
    assert (~keep).sum() <= near_stop_allowance(keep.size)
    H, W = cam.height, cam.width
    rng = np.random.default_rng(3)
    g_rgb, g_d, g_a = (x * keep for x in synth.upstream_grads(17, H, W))
    g_n = (rng.normal(size=(3, H, W)) * keep).astype(np.float32)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")
    pr = torch.zeros(sc.n_vox, device="cuda")
    d_grid, d_sh = fr.backward_ex(t(g_rgb), t(g_d), t(g_a), out, g_normal=t(g_n), priority=pr)
    pr_ref = np.zeros(sc.n_vox)
    og, osh, mag = oracle_grads(sc, cam, g_rgb.astype(np.float64), g_d, g_a, K=K, t_stop=t_stop,
                                g_normal=g_n.astype(np.float64), priority=pr_ref)
    compare_grads(d_grid.cpu().numpy(), og, name="grid", mag=(mag["grid"], mag["grid_seg"]))
    compare_grads(d_sh.cpu().numpy(), osh, name="sh", mag=(mag["sh"], mag["sh_seg"]))
    p = pr.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(p - pr_ref) / np.linalg.norm(pr_ref)
    # a sum of non-negative terms: the relative bar, plus the rounding its
    # grazing segments carry (as for the gradients)
    ratio = np.abs(p - pr_ref) / (1e-3 * (pr_ref + 1e-3 * pr_ref.max()) + SEG_REL * mag["priority_seg"])
    print(f"PARITY priority {name}: rel L2 {rel:.3e}, worst elementwise ratio {ratio.max():.3f}")
    assert rel <= 1e-3 and (ratio <= 1.0).all(), (rel, ratio.max(), int(np.argmax(ratio)))
    # the backward raises the maximum blending weights from its own walk
    mw = torch.zeros(sc.n_vox, device="cuda")
    fr.backward_ex(t(g_rgb), t(g_d), t(g_a), out, max_weight=mw)
    mw_ref = np.zeros(sc.n_vox)
    oracle.render(sc, cam, K=K, t_stop=t_stop, max_weight=mw_ref)
    assert np.abs(mw.cpu().numpy() - mw_ref).max() <= IMG_TOL
    # without the normal term the gradient is the plain backward's
    d0, s0 = fr.backward(t(g_rgb), t(g_d), t(g_a), out)
    d1, s1 = fr.backward_ex(t(g_rgb), t(g_d), t(g_a), out)
    assert torch.allclose(d0, d1, rtol=1e-5, atol=1e-7 * float(d0.abs().max()))
    assert torch.allclose(s0, s1, rtol=1e-5, atol=1e-7 * float(s0.abs().max()))


def test_normal_gradient_needs_a_forward_with_normals():
    """Split tile lists start the backward from the forward's segment sums;
    after a forward without the normal image, a backward with d_normal skips
    them and raises SVR_FLAG_NO_FORWARD."""
    import torch
    from paper_2412_04459_gb300 import _native as N
    sc, cam, dev, fr, K, t_stop = _frame("split")
    out = fr.forward()
    z = torch.zeros(cam.height, cam.width, device="cuda")
    fr.backward_ex(torch.zeros(3, cam.height, cam.width, device="cuda"), z, z, out,
                   g_normal=torch.ones(3, cam.height, cam.width, device="cuda"))
    flags, _ = fr.status()
    assert flags & N.SVR_FLAG_NO_FORWARD
