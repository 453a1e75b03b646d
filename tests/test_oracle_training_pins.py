"""Pins of the oracle's training-step pieces: the distortion loss (Sec. 3.2.3,
Mip-NeRF 360's loss) against closed forms and finite differences, the
transmittance-concentration loss against its values and derivative, and
Adam against a library implementation (torch.optim.Adam on the CPU in FP64)
and its first-step closed form.  No GPU."""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import training
from tests.test_oracle_extras_pins import _explin, _two_voxel_column


def test_distortion_closed_forms():
    """Two constant-density voxels in a column: per pixel L = 2 w_1 w_2 (m_2 -
    m_1) + (w_1^2 delta_1 + w_2^2 delta_2) / 3, w_1 = alpha_1, w_2 = (1 -
    alpha_1) alpha_2, with m and delta from the pixel's ray-box segments."""
    sc = _two_voxel_column(0.9, 2.4, 0.8, -0.5)
    cam = synth.look_at((0.375, 0.375, -2.0), (0.375, 0.375, 0.5), (0, 1, 0), 12.0, 14, 12)
    out = oracle.render(sc, cam, K=1, t_stop=0.0, distortion=True)
    n_both = 0
    for y in range(cam.height):
        for x in range(cam.width):
            ro, rd = oracle.pixel_ray(cam, x, y)
            segs = []
            for v in range(2):
                a, b, ok = oracle.ray_aabb(sc.centre[v].astype(np.float64), 0.25, ro, rd)
                if ok:
                    sigma = _explin(float(sc.grid[sc.corner_idx[v][0]]))
                    segs.append((a, b, 1.0 - math.exp(-sigma * (b - a) * np.linalg.norm(rd))))
            w, T = [], 1.0
            for a, b, al in segs:
                w.append(T * al)
                T *= 1 - al
            want = sum(wi * wi * (b - a) / 3 for wi, (a, b, _) in zip(w, segs))
            if len(segs) == 2:
                n_both += 1
                m = [(a + b) / 2 for a, b, _ in segs]
                want += 2 * w[0] * w[1] * (m[1] - m[0])
            assert abs(out["dist"][y, x] - want) <= 1e-12 * max(1.0, want), (x, y)
    assert n_both > 20


def test_distortion_gradient_matches_finite_differences():
    """d(sum_p g_p L_dist,p + colour terms) / d grid: the analytic backward
    against central differences of the oracle's own rendered losses."""
    sc = synth.random_octree_scene(63, max_level=3, p_split=0.4, max_cells=30, grid_fn=synth.normal_grid(0.8, 1.5))
    cam = synth.orbit_camera(11, 10, 9, distance=1.6)
    H, W = cam.height, cam.width
    rng = np.random.default_rng(8)
    g_rgb, g_a = rng.normal(size=(3, H, W)), rng.normal(size=(H, W))
    g_dist = rng.normal(size=(H, W))
    zero = np.zeros((H, W))
    d_grid, _ = oracle.render_grad(sc, cam, g_rgb, zero, g_a, K=2, t_stop=0.0, g_dist=g_dist)
    grid0 = sc.grid.astype(np.float64)

    def loss(grid):
        o = oracle.render(sc, cam, K=2, t_stop=0.0, grid=grid, distortion=True)
        return float((g_rgb * o["rgb"]).sum() + (g_a * o["alpha"]).sum() + (g_dist * o["dist"]).sum())

    h = 1e-6
    idx = rng.choice(len(grid0), 60, replace=False)
    fd = []
    for i in idx:
        gp, gm = grid0.copy(), grid0.copy()
        gp[i] += h
        gm[i] -= h
        fd.append((loss(gp) - loss(gm)) / (2 * h))
    fd = np.array(fd)
    scale = np.abs(fd).max()
    assert np.abs(d_grid[idx] - fd).max() <= 1e-6 * scale + 1e-9
    d0, _ = oracle.render_grad(sc, cam, g_rgb, zero, g_a, K=2, t_stop=0.0)
    assert np.abs(d0[idx] - fd).max() > 1e-3 * scale          # the distortion term is part of it


def test_t_concentration_values_and_derivative():
    a = np.array([0.5, 0.1, 0.9, 0.0, 1.0, 0.3])
    L, g = training.t_concentration(a)
    H = lambda T: -(T * math.log(T) + (1 - T) * math.log(1 - T))
    Tc = np.clip(1 - a, 1e-6, 1 - 1e-6)
    assert abs(L - np.mean([H(t) for t in Tc])) < 1e-14
    assert abs(H(0.5) - math.log(2)) < 1e-15
    # symmetric in T <-> 1 - T; zero derivative at 1/2 and where clamped
    assert abs(g[0]) < 1e-15 and g[3] == 0.0 and g[4] == 0.0
    assert abs(g[1] + g[2]) < 1e-15
    for i in (1, 2, 5):
        h = 1e-7
        ap, am = a.copy(), a.copy()
        ap[i] += h
        am[i] -= h
        fd = (training.t_concentration(ap)[0] - training.t_concentration(am)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-7


def test_adam_against_torch_and_first_step():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    p0 = rng.normal(size=50)
    p = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=training.LR_GRID, betas=(training.BETA1, training.BETA2), eps=training.ADAM_EPS)
    mine, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    for step in range(1, 8):
        g = rng.normal(size=50)
        if step == 1:
            first, _, _ = training.adam_step(mine, g, m, v, 1, training.LR_GRID)
            assert np.allclose(first, p0 - training.LR_GRID * np.sign(g), rtol=0, atol=1e-12)
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        mine, m, v = training.adam_step(mine, g, m, v, step, training.LR_GRID)
        assert np.allclose(mine, p.detach().numpy(), rtol=0, atol=1e-12)
    lr = training.sh_learning_rates(2)
    assert lr[0, 0] == lr[1, 2] == 0.01 and lr[0, 3] == lr[1, 47] == 0.00025
