"""CUDA path (through the C ABI) vs the FP64 oracle: integer outputs bit-exact,
images within 1e-4, gradients within 1e-3 relative."""
import numpy as np
import pytest

import oracle
import synth
from tests.conftest import cached
from tests.gpu_common import (compare_grads, compare_images, compare_integers, require_gpu,
                              run_gpu, to_np)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def dense5():
    return cached("dense5", lambda: synth.dense_scene(5, seed=0))


TINY = [
    # (scene seed, max level, max cells, camera seed, width, height, distance)
    (0, 3, 64, 0, 48, 40, 1.6),
    (1, 4, 64, 1, 50, 37, 1.8),     # ragged tiles in both directions
    (2, 5, 60, 2, 64, 64, 2.2),
    (3, 4, 64, 3, 33, 17, 1.4),
]


@pytest.mark.parametrize("case", TINY)
@pytest.mark.parametrize("K", [1, 2, 3])
def test_tiny_brute_force_parity(case, K):
    seed, ml, mc, cseed, W, H, dist = case
    sc = synth.random_octree_scene(seed, max_level=ml, p_split=0.5, max_cells=mc,
                                   grid_fn=synth.normal_grid(1.0, 1.5))
    cam = synth.orbit_camera(cseed, W, H, distance=dist)
    fr, out, ins = run_gpu(sc, cam, K=K, t_stop=1e-4)
    compare_integers(sc, cam, ins)
    ref = oracle.render(sc, cam, K=K, t_stop=1e-4)
    compare_images(out, ref)


@pytest.mark.parametrize("K", [1, 3])
def test_dense_level5_full_frame(K):
    """The dense level-5 workload (32^3 voxels, 128x128, mixed-sign tiles)."""
    sc = dense5()
    cam = synth.dense_view_camera()
    fr, out, ins = run_gpu(sc, cam, K=K, t_stop=1e-4)
    n_diff, n_either = compare_integers(sc, cam, ins)
    # rectangles may differ only where a projected corner lands within the
    # rounding margin of a tile edge (lattice corners on the optical axis do)
    _, amb = oracle.binning.voxel_rects(sc, cam)
    assert n_diff <= amb.sum() and n_either <= 2
    assert len(np.unique(ins["tile_mask"])) > 2          # several sign patterns present
    ref = cached(("dense5_ref", K), lambda: oracle.render(sc, cam, K=K, t_stop=1e-4))
    err, excluded = compare_images(out, ref)
    assert excluded <= 5


def test_last_index_names_the_stopping_voxel():
    sc = synth.random_octree_scene(7, max_level=4, p_split=0.4,
                                   grid_fn=synth.normal_grid(12.0, 2.0))
    cam = synth.orbit_camera(4, 40, 40, distance=1.6)
    fr, out, ins = run_gpu(sc, cam, K=2, t_stop=1e-2)
    ref = oracle.render(sc, cam, K=2, t_stop=1e-2)
    compare_images(out, ref)
    o = to_np(out)
    stopped = (ref["term_vox"] >= 0) & (ref["near_stop"] == 0)
    assert stopped.sum() > 20
    last = o["last"][stopped]
    vox = (ins["values"][last] & 0x1FFFFFFF).astype(np.int64)
    assert (vox == ref["term_vox"][stopped]).all()


@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (0.25, 0.5, 1.0)])
@pytest.mark.parametrize("t_stop", [0.0, 1e-4, 0.3])
def test_background_and_stop_threshold(bg, t_stop):
    sc = synth.random_octree_scene(11, max_level=4, p_split=0.5, max_cells=64,
                                   grid_fn=synth.normal_grid(3.0, 1.0))
    cam = synth.orbit_camera(9, 40, 24, distance=1.7)
    fr, out, ins = run_gpu(sc, cam, K=3, t_stop=t_stop, bg=bg)
    ref = oracle.render(sc, cam, K=3, t_stop=t_stop, bg=bg)
    compare_images(out, ref)


# ----------------------------------------------------------------- edge cases

def test_empty_scene():
    sc = synth.scenes.make_scene(synth.scenes.Cells.cat([]), synth.constant_grid(0.0), 0.3,
                                 np.random.default_rng(0))
    cam = synth.orbit_camera(0, 40, 24)
    fr, out, ins = run_gpu(sc, cam, K=1, bg=(0.1, 0.2, 0.3))
    o = to_np(out)
    assert ins["n_pairs"] == 0
    assert np.allclose(o["rgb"], np.array([0.1, 0.2, 0.3])[:, None, None])
    assert (o["alpha"] == 0).all() and (o["depth"] == 0).all() and (o["T_final"] == 1).all()
    assert (o["last"] == -1).all()


def test_scene_behind_camera():
    sc = synth.random_octree_scene(3, max_level=3, max_cells=40)
    cam = synth.look_at((0.5, 0.5, -2.0), (0.5, 0.5, -5.0), (0, 1, 0), 50, 32, 32)
    fr, out, ins = run_gpu(sc, cam, K=1)
    assert ins["n_pairs"] == 0 and (ins["count"] == 0).all()
    assert (to_np(out)["alpha"] == 0).all()


def test_camera_inside_scene():
    """Voxels crossing the near plane cover the whole image (conservative)."""
    sc = synth.random_octree_scene(5, max_level=3, p_split=0.4, max_cells=64,
                                   grid_fn=synth.normal_grid(0.5, 1.0))
    cam = synth.look_at((0.52, 0.47, 0.43), (0.9, 0.8, 0.95), (0, 1, 0), 70, 48, 32)
    fr, out, ins = run_gpu(sc, cam, K=2)
    compare_integers(sc, cam, ins)
    full = (ins["rect"][:, 1] - ins["rect"][:, 0] + 1) * (ins["rect"][:, 3] - ins["rect"][:, 2] + 1)
    assert (full == 3 * 2).any()
    ref = oracle.render(sc, cam, K=2)
    compare_images(out, ref)


def test_invalid_voxels_are_reported():
    from paper_2412_04459_gb300 import DeviceScene, Frame, _native as N
    sc = synth.dense_scene(2)
    sc.centre = sc.centre.copy()
    sc.centre[5, 1] += 0.4 * 0.25       # 0.4 of a level-2 cell off its lattice point
    fr = Frame(DeviceScene.from_host(sc), synth.dense_view_camera(32, 32))
    fr.preprocess()
    with pytest.raises(N.SvrError) as e:
        fr.bin_sort()
    assert e.value.code == N.SVR_ERR_INVALID
    sc = synth.dense_scene(2)
    sc.level = sc.level.copy()
    sc.level[3] = 4                      # above the declared maximum level 2
    fr = Frame(DeviceScene.from_host(sc, max_level=2), synth.dense_view_camera(32, 32))
    fr.preprocess()
    with pytest.raises(N.SvrError) as e:
        fr.bin_sort()
    assert e.value.code == N.SVR_ERR_INVALID


def test_capacity_overflow_reports_count_and_retries():
    from paper_2412_04459_gb300 import DeviceScene, Frame, _native as N
    import ctypes
    sc = dense5()
    cam = synth.dense_view_camera()
    fr = Frame(DeviceScene.from_host(sc), cam, K=1, pair_capacity=1000)
    fr.preprocess()
    n = ctypes.c_int64(0)
    rc = N.lib().svr_bin_sort(N.ref(fr.frame), N.ref(n), None)
    assert rc == N.SVR_ERR_CAPACITY and n.value > 1000
    flags, P = fr.status()
    assert flags & N.SVR_FLAG_CAPACITY and P == n.value
    # the Frame helper grows the workspace and redoes the view
    fr2 = Frame(DeviceScene.from_host(sc), cam, K=1, pair_capacity=1000)
    fr2.render()
    assert fr2.n_pairs == n.value and fr2.pair_capacity >= n.value
    _, out, _ = run_gpu(sc, cam, K=1, capacity=n.value)
    assert np.array_equal(to_np(out)["rgb"], to_np(fr2.forward())["rgb"])


def test_deterministic_outputs():
    sc = dense5()
    cam = synth.dense_view_camera()
    _, o1, i1 = run_gpu(sc, cam, K=3)
    _, o2, i2 = run_gpu(sc, cam, K=3)
    for k in ("keys", "values", "ranges", "rect", "count"):
        assert np.array_equal(i1[k], i2[k])
    for k in ("rgb", "depth", "alpha", "T_final", "last"):
        assert np.array_equal(to_np(o1)[k], to_np(o2)[k])


def test_max_level_16_sort_path():
    """A scene declared with max_level 16 keeps all 48 Morton bits in the keys
    and sorts each tile by (key, value) through the value-rank path; sorted
    pairs, ranges and images still equal the oracle's."""
    from paper_2412_04459_gb300 import DeviceScene, Frame
    sc = synth.random_octree_scene(12, max_level=4, p_split=0.6, grid_fn=synth.normal_grid(1.0, 1.0))
    cam = synth.orbit_camera(3, 96, 64, distance=1.8)
    fr = Frame(DeviceScene.from_host(sc, max_level=16), cam, K=2)
    fr.preprocess()
    fr.bin_sort()
    out = fr.forward()
    ins = fr.inspect()
    assert ins["n_pairs"] > 1500
    compare_integers(sc, cam, ins)
    compare_images(out, oracle.render(sc, cam, K=2))
