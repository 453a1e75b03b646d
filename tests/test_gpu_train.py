"""The training step's pieces and the whole step against the oracle: Adam
with the paper's settings, the transmittance-concentration loss, the
distortion loss of every ray (forward and backward, also across split tile
lists), and TrainStep (batched render, optional supersampling, losses,
backward, Adam), eager and graph-replayed."""
import numpy as np
import pytest

import oracle
import synth
from oracle import antialias, training
from tests.conftest import cached
from tests.gpu_common import IMG_TOL, SEG_REL, compare_grads, near_stop_allowance, oracle_grads, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    require_gpu()


def _t(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, np.float32), device="cuda")


@pytest.mark.parametrize("period,head,lr,lr_rest", [(1, 1, training.LR_GRID, None),
                                                     (48, 3, training.LR_SH_DC, training.LR_SH_REST)])
def test_adam_kernel(period, head, lr, lr_rest):
    from paper_2412_04459_gb300.train import adam
    rng = np.random.default_rng(period)
    n = 48 * 1000 + (0 if period > 1 else 37)
    p = rng.normal(size=n).astype(np.float32)
    pg, mg, vg = _t(p), _t(np.zeros(n)), _t(np.zeros(n))
    p64, m64, v64 = p.astype(np.float64), np.zeros(n), np.zeros(n)
    lrs = np.where(np.arange(n) % period < head, lr, lr if lr_rest is None else lr_rest)
    for step in range(1, 6):
        g = (rng.normal(size=n) * rng.choice([1e-6, 1.0, 1e3], size=n)).astype(np.float32)
        adam(pg, _t(g), mg, vg, step, lr, lr_rest, period=period, head=head)
        p64, m64, v64 = training.adam_step(p64, g.astype(np.float64), m64, v64, step, lrs)
    err = np.abs(pg.cpu().numpy() - p64)
    assert (err <= 1e-6 * np.abs(p64) + 1e-4 * lrs).all(), err.max()


def test_t_concentration_and_weighted_mean():
    import torch
    from paper_2412_04459_gb300.train import t_concentration_loss, weighted_mean
    rng = np.random.default_rng(0)
    a = rng.random(100_003).astype(np.float32)
    a[:5] = [0.0, 1.0, 0.5, 1e-8, 1 - 1e-8]
    loss = torch.zeros(1, device="cuda")
    g = torch.empty(len(a), device="cuda")
    t_concentration_loss(_t(a), 0.01, loss, g)
    L, G = training.t_concentration(a.astype(np.float64))
    assert abs(loss.item() - 0.01 * L) <= 1e-5 * 0.01 * L
    assert np.allclose(g.cpu().numpy(), 0.01 * G, rtol=1e-4, atol=1e-12)
    x = rng.random(77_777).astype(np.float32)
    weighted_mean(_t(x), 0.1, loss)
    assert abs(loss.item() - 0.01 * L - 0.1 * x.astype(np.float64).mean()) <= 1e-5


def _back_heavy(front, back_mean, back_std=2.0, z_cut=0.5):
    def grid_fn(pos, rng):
        out = np.full(len(pos), front, dtype=np.float64)
        far = pos[:, 2] >= z_cut
        out[far] = rng.normal(back_mean, back_std, size=int(far.sum()))
        return out
    return grid_fn


CASES = {
    "tiny": (lambda: synth.random_octree_scene(73, max_level=4, p_split=0.5, max_cells=64,
                                               grid_fn=synth.normal_grid(1.0, 1.5)),
             lambda: synth.orbit_camera(17, 48, 40, distance=1.7), 3, 1e-4),
    "split": (lambda: cached("dense5_backheavy", lambda: synth.dense_scene(5, seed=3,
                                                                           grid_fn=_back_heavy(-4.0, 40.0, 5.0))),
              lambda: synth.dense_view_camera(), 2, 1e-3),
}


@pytest.mark.parametrize("name", list(CASES))
def test_distortion_forward_and_backward(name):
    import torch
    from paper_2412_04459_gb300 import DeviceScene, Frame, _native as N
    make_scene, make_cam, K, t_stop = CASES[name]
    sc, cam = make_scene(), make_cam()
    fr = Frame(DeviceScene.from_host(sc), cam, K=K, t_stop=t_stop)
    fr.preprocess()
    fr.bin_sort()
    H, W = cam.height, cam.width
    dist = torch.zeros(2, H, W, device="cuda")
    ex = N.SvrRenderExtras()
    ex.distortion = dist.data_ptr()
    out = fr.new_outputs()
    from paper_2412_04459_gb300.raster import _ptr, _stream
    N.check(N.lib().svr_render_fwd_ex(N.ref(fr.frame), _ptr(out["rgb"]), _ptr(out["depth"]), _ptr(out["alpha"]),
                                      _ptr(out["T_final"]), _ptr(out["last"]), N.ref(ex), _stream()), "fwd_ex")
    ref = oracle.render(sc, cam, K=K, t_stop=t_stop, distortion=True)
    keep = ref["near_stop"] == 0
    assert (~keep).sum() <= near_stop_allowance(keep.size)
    err = np.abs(dist[0].cpu().numpy() - ref["dist"])[keep].max()
    print(f"PARITY distortion {name}: {err:.3e}, max {ref['dist'].max():.3e}")
    assert err <= IMG_TOL and ref["dist"].max() > 1e-2
    if name == "split":
        lens = np.diff(fr.inspect()["ranges"].astype(np.int64), axis=1)
        assert lens.max() > 1024
    rng = np.random.default_rng(5)
    g_rgb = rng.normal(size=(3, H, W)) * keep
    g_a = rng.normal(size=(H, W)) * keep
    g_dist = rng.normal(size=(H, W)) * keep
    bx = N.SvrRenderExtras()
    bx.distortion = dist.data_ptr()
    gd = _t(g_dist)
    bx.d_distortion = gd.data_ptr()
    d_grid = torch.zeros(sc.n_pts, device="cuda")
    d_sh = torch.empty(sc.n_vox, 48, device="cuda")
    gr, ga = _t(g_rgb), _t(g_a)
    N.check(N.lib().svr_render_bwd_ex(N.ref(fr.frame), _ptr(gr), None, _ptr(ga), _ptr(out["T_final"]),
                                      _ptr(out["last"]), _ptr(d_grid), _ptr(d_sh), N.ref(bx), _stream()), "bwd_ex")
    og, osh, mag = oracle_grads(sc, cam, g_rgb, np.zeros((H, W)), g_a, K=K, t_stop=t_stop, g_dist=g_dist)
    compare_grads(d_grid.cpu().numpy(), og, name="grid", mag=(mag["grid"], mag["grid_seg"]))
    compare_grads(d_sh.cpu().numpy(), osh, name="sh", mag=(mag["sh"], mag["sh_seg"]))


def _train_case(h_ss):
    import torch
    from paper_2412_04459_gb300 import DeviceScene
    sc = synth.random_octree_scene(75, max_level=4, p_split=0.5, max_cells=300, grid_fn=synth.normal_grid(1.5, 1.5))
    cams = [synth.orbit_camera(40 + i, *wh, distance=1.8) for i, wh in enumerate([(48, 40), (40, 52)])]
    rng = np.random.default_rng(2)
    tgt_grid = sc.grid.astype(np.float64) + 0.3 * rng.normal(size=sc.n_pts)
    targets = []
    for c in cams:
        rc = antialias.supersampled_camera(c, h_ss) if h_ss else c
        img = oracle.render(sc, rc, K=2, grid=tgt_grid)["rgb"]
        targets.append(antialias.downsample(img, c.height, c.width) if h_ss else img)
    dev = DeviceScene.from_host(sc)
    return sc, cams, targets, dev, [torch.as_tensor(t.astype(np.float32), device="cuda") for t in targets]


@pytest.mark.parametrize("h_ss", [None, 1.5])
def test_train_step_against_oracle(h_ss):
    """Losses (MSE + 0.01 L_T + 0.1 mean distortion) against the oracle's;
    gradients against the oracle's for the upstream gradients the step's
    losses produced; the Adam update against the FP64 update of the same
    gradients."""
    import torch
    from paper_2412_04459_gb300.train import TrainStep
    sc, cams, targets, dev, tt = _train_case(h_ss)
    ts = TrainStep(dev, cams, tt, K=2, h_ss=h_ss, stats=True)
    grid0, sh0 = dev.grid.clone(), dev.sh.clone()
    ts.forward_backward()
    torch.cuda.synchronize()
    # the pruning statistic gathered by the step's backward
    mw_ref = np.zeros(sc.n_vox)
    for rc in ts.render_cams:
        oracle.render(sc, rc, K=2, max_weight=mw_ref)
    assert np.abs(ts.max_weight.cpu().numpy() - mw_ref).max() <= IMG_TOL
    assert float(ts.priority.sum()) > 0
    # the oracle's loss for the same parameters
    P = ts.frame.n_pixels
    mse_num, n_rgb, lt, ld = 0.0, 0, 0.0, 0.0
    alphas = []
    og, osh = np.zeros(sc.n_pts), np.zeros((sc.n_vox, 48))
    mg, ms = [np.zeros(sc.n_pts), np.zeros(sc.n_pts)], [np.zeros((sc.n_vox, 48)), np.zeros((sc.n_vox, 48))]
    pr_ref, pr_seg = np.zeros(sc.n_vox), np.zeros(sc.n_vox)
    outs = ts.frame.views(ts.out)
    for v, c in enumerate(cams):
        rc = ts.render_cams[v]
        ref = oracle.render(sc, rc, K=2, distortion=True)
        assert not ref["near_stop"].any()
        rgb = antialias.downsample(ref["rgb"], c.height, c.width) if h_ss else ref["rgb"]
        mse_num += ((rgb - targets[v]) ** 2).sum()
        n_rgb += rgb.size
        alphas.append(ref["alpha"].reshape(-1))
        ld += ref["dist"].sum()
    L_T, _ = training.t_concentration(np.concatenate(alphas))
    want = mse_num / n_rgb + training.LAMBDA_T * L_T + training.LAMBDA_DIST * ld / P
    assert abs(ts.loss.item() - want) <= 1e-4 * want, (ts.loss.item(), want)
    # gradients for the upstream gradients the GPU's losses handed the backward
    g_rgb_all = ts.g_rgb.cpu().numpy().astype(np.float64)
    g_a_all = ts.g_alpha.cpu().numpy().astype(np.float64)
    for v, c in enumerate(cams):
        rc = ts.render_cams[v]
        a, b = int(ts.frame.pixel_base[v]), int(ts.frame.pixel_base[v + 1])
        g_rgb = g_rgb_all[3 * a:3 * b].reshape(3, rc.height, rc.width)
        g_a = g_a_all[a:b].reshape(rc.height, rc.width)
        g_d = np.full((rc.height, rc.width), training.LAMBDA_DIST / P)
        x, y, m = oracle_grads(sc, rc, g_rgb, np.zeros_like(g_a), g_a, K=2, g_dist=g_d, priority=pr_ref)
        pr_seg += m["priority_seg"]
        og += x
        osh += y
        mg[0] += m["grid"]
        mg[1] += m["grid_seg"]
        ms[0] += m["sh"]
        ms[1] += m["sh_seg"]
    compare_grads(ts.d_grid.cpu().numpy(), og, name="grid", mag=mg)
    compare_grads(ts.d_sh.cpu().numpy(), osh, name="sh", mag=ms)
    # the subdivision priority gathered by the same backward (distortion term
    # included), at the relative bar plus its grazing segments' rounding
    p = ts.priority.cpu().numpy().astype(np.float64)
    rel = np.linalg.norm(p - pr_ref) / np.linalg.norm(pr_ref)
    ratio = np.abs(p - pr_ref) / (1e-3 * (pr_ref + 1e-3 * pr_ref.max()) + SEG_REL * pr_seg)
    print(f"PARITY priority train step: rel L2 {rel:.3e}, worst elementwise ratio {ratio.max():.3f}")
    assert rel <= 1e-3 and (ratio <= 1.0).all(), (rel, ratio.max())
    # Adam on the GPU's own gradients against the FP64 update
    dg, ds = ts.d_grid.cpu().numpy().astype(np.float64), ts.d_sh.cpu().numpy().astype(np.float64)
    ts.optimize()
    torch.cuda.synchronize()
    want_g, _, _ = training.adam_step(grid0.cpu().numpy(), dg, 0, 0, 1, training.LR_GRID)
    want_s, _, _ = training.adam_step(sh0.cpu().numpy(), ds, 0, 0, 1, training.sh_learning_rates(sc.n_vox))
    assert np.abs(dev.grid.cpu().numpy() - want_g).max() <= 1e-5
    assert np.abs(dev.sh.cpu().numpy() - want_s).max() <= 1e-5


def test_graph_replayed_steps_equal_eager_steps():
    """Three steps with the forward-backward replayed from a CUDA graph give
    the eager steps' losses and parameters (the same kernels, atomics in
    another order), and the loss decreases."""
    import torch
    from paper_2412_04459_gb300 import DeviceScene
    from paper_2412_04459_gb300.train import TrainStep
    sc, cams, targets, dev, tt = _train_case(None)
    dev2 = DeviceScene.from_host(sc)
    eager = TrainStep(dev, cams, tt, K=2)
    graph = TrainStep(dev2, cams, tt, K=2).capture()
    graph.scene.grid.copy_(eager.scene.grid)            # capture() ran one eager warm-up pass: no update
    losses = []
    for _ in range(3):
        le = eager.step().item()
        lg = graph.step().item()
        assert abs(le - lg) <= 1e-5 * abs(le)
        losses.append(le)
    assert torch.allclose(dev.grid, dev2.grid, rtol=0, atol=1e-5)
    assert torch.allclose(dev.sh, dev2.sh, rtol=0, atol=1e-5)
    assert losses[2] < losses[0]
