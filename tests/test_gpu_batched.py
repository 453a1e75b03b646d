"""Batched multi-view path (svr_preprocess_views / svr_render_batched): per
view it must equal the single-view path (which the parity tests hold to the
oracle), its compact keys must carry the same order, it must take more tiles
than the single-view key layout allows, and its whole step must replay from a
CUDA graph.  Tile sizes 8 and 32 are checked against the oracle directly."""
import numpy as np
import pytest

import oracle
import synth
from oracle import binning
from tests.conftest import cached
from tests.gpu_common import compare_images, compare_integers, compare_reordered, require_gpu, run_gpu, to_np

pytestmark = pytest.mark.gpu

SIZES = [(64, 48), (40, 40), (72, 56), (33, 65)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _scene():
    return cached("batched_scene", lambda: synth.random_octree_scene(
        17, max_level=5, p_split=0.5, grid_fn=synth.normal_grid(2.0, 1.5)))


def _cams(n, seed=30, sizes=SIZES, distance=1.8):
    return [synth.orbit_camera(seed + i, *sizes[i % len(sizes)], distance=distance) for i in range(n)]


def test_batched_views_equal_single_views():
    from paper_2412_04459_gb300 import DeviceScene, Frame
    sc = _scene()
    dev = DeviceScene.from_host(sc)
    cams = _cams(5)
    batch = Frame(dev, cams, K=3)
    out = batch.render()
    ib = batch.inspect()
    views = batch.views(out)
    S = int(batch.frame.key_shift)
    assert S == 3 * (sc.max_level + 1)
    total = 0
    for v, cam in enumerate(cams):
        single = Frame(dev, cam, K=3)
        o1 = single.render()
        i1 = single.inspect()
        total += i1["n_pairs"]
        a, b = to_np(views[v]), to_np(o1)
        for k in ("rgb", "depth", "alpha", "T_final"):
            assert np.array_equal(a[k], b[k]), (v, k)
        # `last` is a position in each path's own sorted list: same voxel
        ok = b["last"] >= 0
        assert np.array_equal(ok, a["last"] >= 0)
        assert np.array_equal(ib["values"][a["last"][ok]], i1["values"][b["last"][ok]])
        # per tile: same values in the same order; compact key = tile id over
        # the top S bits of the single-view key's Morton order
        tb = int(batch.frame.tile_base[v])
        nt = i1["ranges"].shape[0]
        for t in range(nt):
            b0, e0 = i1["ranges"][t]
            b1, e1 = ib["ranges"][tb + t]
            assert e0 - b0 == e1 - b1
            assert np.array_equal(i1["values"][b0:e0], ib["values"][b1:e1])
            k0 = i1["keys"][b0:e0] & np.uint64((1 << 48) - 1)
            want = (np.uint64(tb + t) << np.uint64(S)) | (k0 >> np.uint64(48 - S))
            assert np.array_equal(ib["keys"][b1:e1], want)
    assert ib["n_pairs"] == total


def test_batched_backward_sums_single_views():
    import torch
    from paper_2412_04459_gb300 import DeviceScene, Frame
    sc = _scene()
    dev = DeviceScene.from_host(sc)
    cams = _cams(4, seed=50)
    batch = Frame(dev, cams, K=2, bg=(0.1, 0.2, 0.3))
    out = batch.render()
    grads = [synth.upstream_grads(10 + v, c.height, c.width) for v, c in enumerate(cams)]
    flat = [torch.as_tensor(np.concatenate([g[i].reshape(-1) for g in grads]), device="cuda") for i in range(3)]
    dg_b, ds_b = batch.backward(flat[0], flat[1], flat[2], out)
    dg_s = torch.zeros_like(dg_b)
    ds_s = torch.zeros_like(ds_b)
    for v, cam in enumerate(cams):
        single = Frame(dev, cam, K=2, bg=(0.1, 0.2, 0.3))
        o1 = single.render()
        t = lambda a: torch.as_tensor(a, device="cuda")
        dg, ds = single.backward(t(grads[v][0]), t(grads[v][1]), t(grads[v][2]), o1)
        dg_s += dg
        ds_s += ds
    for a, b, name in ((dg_b, dg_s, "grid"), (ds_b, ds_s, "sh")):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        assert np.linalg.norm(a - b) <= 1e-5 * np.linalg.norm(b)
        compare_reordered(a, b, name)


def test_batched_beyond_single_view_tile_limit():
    """9 views of 1920x1080 at 16x16 tiles: 73,440 tiles, more than the
    single-view key's 16-bit tile id; the compact keys take them."""
    from paper_2412_04459_gb300 import DeviceScene, Frame
    sc = synth.random_octree_scene(23, max_level=4, p_split=0.5, max_cells=200)
    dev = DeviceScene.from_host(sc)
    cams = [synth.orbit_camera(60 + i, 1920, 1080, distance=2.2) for i in range(9)]
    batch = Frame(dev, cams, K=1)
    out = batch.render()
    assert int(batch.frame.total_tiles) == 9 * 120 * 68 > 65536
    views = batch.views(out)
    for v in (0, 8):
        o1 = Frame(dev, cams[v], K=1).render()
        assert np.array_equal(to_np(views[v])["rgb"], to_np(o1)["rgb"])


@pytest.mark.parametrize("tile", [8, 32])
def test_tile_sizes_against_oracle(tile):
    sc = synth.random_octree_scene(4, max_level=4, p_split=0.5, max_cells=64,
                                   grid_fn=synth.normal_grid(1.0, 1.5))
    cam = synth.orbit_camera(7, 70, 45, distance=1.7)
    from paper_2412_04459_gb300 import DeviceScene, Frame
    fr = Frame(DeviceScene.from_host(sc), cam, K=3, tile=tile)
    out = fr.render()
    compare_integers(sc, cam, fr.inspect(), tile=tile)
    compare_images(out, oracle.render(sc, cam, K=3))


def test_graph_replay_of_batched_step():
    """svr_render_batched captured once in a CUDA graph and replayed after the
    densities changed in place gives the eager result for the new values."""
    import torch
    from paper_2412_04459_gb300 import DeviceScene, Frame
    sc = _scene()
    dev = DeviceScene.from_host(sc)
    cams = _cams(4, seed=70)
    fr = Frame(dev, cams, K=3)
    fr.render()                                  # sizes the workspace
    fr.pair_capacity = fr.n_pairs * 2 + 1024
    out = fr.new_outputs()
    P = fr.n_pixels
    rng = np.random.default_rng(0)
    grads = [torch.as_tensor(rng.normal(size=n).astype(np.float32), device="cuda") for n in (3 * P, P, P)]
    d_grid = torch.zeros(sc.n_pts, device="cuda")
    d_sh = torch.empty(sc.n_vox, 48, device="cuda")
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        fr.render_batched(out, grads, d_grid, d_sh)          # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        d_grid.zero_()
        fr.render_batched(out, grads, d_grid, d_sh)
    new = torch.as_tensor(sc.grid + 0.5 * rng.normal(size=sc.n_pts).astype(np.float32), device="cuda")
    dev.grid.copy_(new)
    g.replay()
    torch.cuda.synchronize()
    got = {k: v.clone() for k, v in out.items()}
    got_dg, got_ds = d_grid.clone(), d_sh.clone()
    # eager, same inputs
    fr2 = Frame(dev, cams, K=3, pair_capacity=fr.pair_capacity)
    ref = fr2.render()
    dg2, ds2 = fr2.backward(grads[0], grads[1], grads[2], ref)
    for k in ("rgb", "depth", "alpha", "T_final"):
        assert torch.equal(got[k], ref[k]), k
    assert torch.linalg.norm(got_dg - dg2) <= 1e-5 * torch.linalg.norm(dg2)
    assert torch.linalg.norm(got_ds - ds2) <= 1e-5 * torch.linalg.norm(ds2)
    compare_reordered(got_dg.cpu().numpy(), dg2.cpu().numpy(), "grid")
    compare_reordered(got_ds.cpu().numpy(), ds2.cpu().numpy(), "sh")
    flags, _ = fr.status()
    assert flags == 0


@pytest.mark.parametrize("partitions", [1, 2])
def test_batched_renderer_partitions_equal_views(partitions, tmp_path, monkeypatch):
    """The graph-replayed BatchedRenderer, whole or split into sort
    partitions, gives each view's single-view images and the summed
    gradients; the autotuner returns one of its candidates."""
    import torch
    from paper_2412_04459_gb300 import DeviceScene, Frame
    from paper_2412_04459_gb300.autotune import BatchedRenderer, tune
    monkeypatch.setenv("SVR_TUNE_CACHE", str(tmp_path / "tune.json"))
    sc = _scene()
    dev = DeviceScene.from_host(sc)
    cams = _cams(3, seed=90)
    best = tune(dev, cams, K=2, tiles=(8, 16), partitions=(1, 3), reps=1)
    assert (best["tile"], best["partitions"]) in {(8, 1), (8, 3), (16, 1), (16, 3)}
    assert tune(dev, cams, K=2, tiles=(8, 16), partitions=(1, 3), reps=1) == best   # cached
    r = BatchedRenderer(dev, cams, K=2, tile=16, partitions=partitions)
    rng = np.random.default_rng(3)
    for x in r.grads:
        x.copy_(torch.as_tensor(rng.normal(size=x.numel()).astype(np.float32)))
    r.capture()
    r.step()
    torch.cuda.synchronize()
    dg = torch.zeros_like(r.d_grid)
    ds = torch.zeros_like(r.d_sh)
    for v, cam in enumerate(cams):
        a, b = int(r.pixel_base[v]), int(r.pixel_base[v + 1])
        fr = Frame(dev, cam, K=2)
        o = fr.render()
        assert torch.equal(r.out["rgb"][3 * a:3 * b].view(3, cam.height, cam.width), o["rgb"])
        g1, s1 = fr.backward(r.grads[0][3 * a:3 * b], r.grads[1][a:b], r.grads[2][a:b], o)
        dg += g1
        ds += s1
    # sums over views in another order
    assert torch.linalg.norm(r.d_grid - dg) <= 1e-5 * torch.linalg.norm(dg)
    assert torch.linalg.norm(r.d_sh - ds) <= 1e-5 * torch.linalg.norm(ds)
    compare_reordered(r.d_grid.cpu().numpy(), dg.cpu().numpy(), "grid")
    compare_reordered(r.d_sh.cpu().numpy(), ds.cpu().numpy(), "sh")
