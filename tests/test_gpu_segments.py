"""Tile lists longer than 1024 entries are composited in segments by separate
warps and merged.  These cases put the stopping voxel, the underflow of the
transmittance and the work counts into later segments of split lists and
compare with the FP64 oracle, which walks every list in one piece."""
import numpy as np
import pytest

import oracle
import synth
from tests.conftest import cached
from tests.gpu_common import compare_grads, compare_images, oracle_grads, require_gpu, run_gpu, to_np

pytestmark = pytest.mark.gpu

SEG = 1024   # entries per segment of a split tile list


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _back_heavy(front, back_mean, back_std=2.0, z_cut=0.5):
    """Raw densities: `front` for grid points nearer the camera than z_cut
    (the dense-view camera looks along +z), N(back_mean, back_std) behind."""
    def grid_fn(pos, rng):
        out = np.full(len(pos), front, dtype=np.float64)
        far = pos[:, 2] >= z_cut
        out[far] = rng.normal(back_mean, back_std, size=int(far.sum()))
        return out
    return grid_fn


def _split_position(ins, last):
    """Position of each pixel's `last` entry within its tile's list."""
    ranges = ins["ranges"].astype(np.int64)
    keys = ins["keys"]
    tile = (keys[np.clip(last, 0, None)] >> np.uint64(48)).astype(np.int64)
    return last - ranges[tile, 0], ranges[tile, 1] - ranges[tile, 0]


@pytest.mark.parametrize("K", [1, 3])
def test_stop_inside_later_segments(K):
    """Transparent front half, opaque back half: pixels stop deep in their
    lists, after the first segment; images, the stopping voxel and the
    gradients equal the oracle's."""
    import torch
    sc = cached("dense5_backheavy", lambda: synth.dense_scene(5, seed=3, grid_fn=_back_heavy(-4.0, 40.0, 5.0)))
    cam = synth.dense_view_camera()
    fr, out, ins = run_gpu(sc, cam, K=K, t_stop=1e-3)
    ref = oracle.render(sc, cam, K=K, t_stop=1e-3)
    compare_images(out, ref)
    o = to_np(out)
    keep = ref["near_stop"] == 0
    stopped = (ref["term_vox"] >= 0) & keep
    pos, length = _split_position(ins, o["last"][stopped])
    assert (length > SEG).any() and (pos >= SEG).sum() > 50   # stops inside later segments
    vox = (ins["values"][o["last"][stopped]] & 0x1FFFFFFF).astype(np.int64)
    assert (vox == ref["term_vox"][stopped]).all()
    g_rgb, g_d, g_a = synth.upstream_grads(7, cam.height, cam.width)
    g_rgb, g_d, g_a = g_rgb * keep[None], g_d * keep, g_a * keep
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    dg, ds = fr.backward(t(g_rgb), t(g_d), t(g_a), out)
    og, osh, mag = oracle_grads(sc, cam, g_rgb.astype(np.float64), g_d, g_a, K=K, t_stop=1e-3)
    compare_grads(dg.cpu().numpy(), og, name="grid", mag=(mag["grid"], mag["grid_seg"]))
    compare_grads(ds.cpu().numpy(), osh, name="sh", mag=(mag["sh"], mag["sh_seg"]))


def test_underflow_inside_later_segments():
    """t_stop = 0 and very dense back voxels: T_final underflows in later
    segments, whose backward then runs front to back from the transmittance
    the forward left in front of them."""
    import torch
    sc = cached("dense5_underflow", lambda: synth.dense_scene(5, seed=4, grid_fn=_back_heavy(-2.0, 300.0, 50.0)))
    cam = synth.dense_view_camera()
    fr, out, ins = run_gpu(sc, cam, K=2, t_stop=0.0)
    o = to_np(out)
    under = o["T_final"] < 1e-30
    assert under.mean() > 0.1
    ref = oracle.render(sc, cam, K=2, t_stop=0.0)
    compare_images(out, ref)
    g_rgb, g_d, g_a = synth.upstream_grads(8, cam.height, cam.width)
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    dg, ds = fr.backward(t(g_rgb), t(g_d), t(g_a), out)
    assert np.isfinite(dg.cpu().numpy()).all() and np.isfinite(ds.cpu().numpy()).all()
    og, osh, mag = oracle_grads(sc, cam, g_rgb.astype(np.float64), g_d, g_a, K=2, t_stop=0.0)
    compare_grads(dg.cpu().numpy(), og, name="grid", mag=(mag["grid"], mag["grid_seg"]))
    compare_grads(ds.cpu().numpy(), osh, name="sh", mag=(mag["sh"], mag["sh_seg"]))


def test_work_counts_across_segments():
    """svr_render_stats counts each pixel's composited hits once, however its
    list was split, and gives the same images as svr_render_fwd."""
    sc = cached("dense5_backheavy", lambda: synth.dense_scene(5, seed=3, grid_fn=_back_heavy(-4.0, 40.0, 5.0)))
    cam = synth.dense_view_camera()
    fr, out, ins = run_gpu(sc, cam, K=2, t_stop=1e-3)
    ref = oracle.render(sc, cam, K=2, t_stop=1e-3)
    st = to_np(fr.forward_stats())
    keep = ref["near_stop"] == 0
    hits = st["counts"][..., 1]
    assert (hits[keep] == ref["n_comp"][keep]).mean() > 0.999
    assert np.array_equal(st["rgb"], to_np(out)["rgb"])
    assert np.array_equal(st["last"], to_np(out)["last"])


def test_repeated_forward_and_backward_are_stable():
    """The merge counters reset themselves: a second forward of the same sort
    gives identical outputs, and so does the backward after it."""
    import torch
    sc = cached("dense5", lambda: synth.dense_scene(5, seed=0))
    cam = synth.dense_view_camera()
    fr, out, _ = run_gpu(sc, cam, K=3, inspect=False)
    g = [torch.as_tensor(a, device="cuda") for a in synth.upstream_grads(3, cam.height, cam.width)]
    d1 = fr.backward(*g, out)
    out2 = fr.forward()
    for k in out:
        assert torch.equal(out[k], out2[k]), k
    d2 = fr.backward(*g, out2)
    assert torch.allclose(d1[0], d2[0], rtol=1e-5, atol=1e-7)
    assert torch.allclose(d1[1], d2[1], rtol=1e-5, atol=1e-7)


def test_backward_without_forward_is_flagged():
    """A backward after a new sort but before its forward has neither the
    forward's hit masks nor the split tiles' segment sums: it skips every tile
    and raises the flag; after the forward it runs."""
    import torch
    from paper_2412_04459_gb300 import _native as N
    sc = cached("dense5", lambda: synth.dense_scene(5, seed=0))
    cam = synth.dense_view_camera()
    fr, out, _ = run_gpu(sc, cam, K=1, inspect=False)
    fr.preprocess()
    fr.bin_sort()
    g = [torch.as_tensor(a, device="cuda") for a in synth.upstream_grads(3, cam.height, cam.width)]
    d0, _ = fr.backward(*g, out)
    flags, _ = fr.status()
    assert flags & N.SVR_FLAG_NO_FORWARD
    assert float(d0.abs().max()) == 0.0
    fr.forward(out)
    d1, _ = fr.backward(*g, out)
    torch.cuda.synchronize()
    assert float(d1.abs().max()) > 0.0


def test_very_long_lists_sort_and_render():
    """A dense level-6 grid (262,144 voxels) seen whole by a 32x32 camera:
    each of the 4 tiles lists 65K-70K pairs, past what the per-tile merge
    holds in shared memory, so the runs are merged through global memory and
    the walks span 64+ segments; sorted pairs bit-exact, images vs oracle."""
    from tests.gpu_common import compare_integers
    sc = cached("dense6_lowdensity", lambda: synth.dense_scene(6, seed=1, grid_fn=synth.normal_grid(-1.0, 1.0)))
    cam = synth.look_at((0.5, 0.5, -1.5), (0.5, 0.5, 0.5), (0, 1, 0), 40, 32, 32)
    fr, out, ins = run_gpu(sc, cam, K=2, t_stop=1e-4)
    lens = np.diff(ins["ranges"].astype(np.int64), axis=1).ravel()
    assert lens.min() > 8192
    compare_integers(sc, cam, ins)
    compare_images(out, oracle.render(sc, cam, K=2, t_stop=1e-4))
