"""Pins of the oracle's optional outputs: the normal modality (Eq. vox_normal,
Eq. interp_grad, Eq. interp_grad_grad) and the pruning / subdivision
statistics (Sec. 3.2.2: maximum blending weight, Eq. priority).

Each is tied to something other than the oracle's own formula: the trilinear
field written out from its textbook definition and differentiated by finite
differences, linear fields whose gradient is known, closed forms for one or
two constant-density voxels on the camera axis, and central differences of
the oracle's rendered normal image.  No GPU.
"""
import itertools
import math

import numpy as np
import pytest

import oracle
import synth


def _trilinear_textbook(V, q):
    """sum over corners (i, j, k) of V_ijk prod (q or 1 - q), corner index
    4 i + 2 j + k."""
    acc = 0.0
    for i, j, k in itertools.product((0, 1), repeat=3):
        w = (q[0] if i else 1 - q[0]) * (q[1] if j else 1 - q[1]) * (q[2] if k else 1 - q[2])
        acc += V[4 * i + 2 * j + k] * w
    return acc


def test_interp_grad_is_the_gradient_at_the_centre():
    """P9: the closed form of Eq. (interp_grad) equals the central-difference
    gradient of the trilinear field at q = (1/2, 1/2, 1/2), and the oracle's
    trilinear interpolation equals the textbook sum."""
    rng = np.random.default_rng(0)
    for _ in range(20):
        V = rng.normal(size=8)
        qc = np.full(3, 0.5)
        h = 1e-6
        fd = np.array([(_trilinear_textbook(V, qc + h * e) - _trilinear_textbook(V, qc - h * e)) / (2 * h)
                       for e in np.eye(3)])
        assert np.allclose(oracle.interp_grad_centre(V), fd, rtol=1e-8, atol=1e-9)
        q = rng.random(3)
        assert abs(oracle.trilinear(V, q) - _trilinear_textbook(V, q)) < 1e-14


def test_interp_grad_of_a_linear_field():
    """V_c = g . (x_c, y_c, z_c) + h (corner offsets 0/1) is its own trilinear
    interpolant, so the gradient anywhere, the centre included, is g."""
    g = np.array([0.7, -1.3, 2.1])
    V = np.array([g @ np.array([i, j, k]) + 0.4 for i, j, k in itertools.product((0, 1), repeat=3)])
    assert np.allclose(oracle.interp_grad_centre(V), g, rtol=1e-14)


def _linear_voxel_scene(grad, offset=0.3):
    """One level-1 voxel at lattice (1, 1, 1) whose corner values form a
    linear field with local gradient `grad`."""
    cells = synth.scenes.dense_cells(1)
    cells = cells.take(np.where((cells.ijk == (1, 1, 1)).all(1))[0])
    sc = synth.scenes.make_scene(cells, synth.constant_grid(0.0), 0.0, np.random.default_rng(0))
    bits = np.array([[(c >> 2) & 1, (c >> 1) & 1, c & 1] for c in range(8)], np.float64)
    sc.grid[sc.corner_idx[0]] = (bits @ np.asarray(grad) + offset).astype(np.float32)
    sc.sh[:] = 0.0
    return sc


def test_normal_image_of_a_linear_field():
    """A single voxel with a linear density field: every pixel that sees it
    composites N = alpha n with n = grad / |grad| (Eq. vox_normal), whatever
    its ray."""
    grad = np.array([0.5, -1.0, 2.0])
    sc = _linear_voxel_scene(grad)
    cam = synth.look_at((-0.8, 1.9, -1.1), (0.75, 0.75, 0.75), (0, 1, 0), 30.0, 20, 18)
    out = oracle.render(sc, cam, K=2, t_stop=0.0, normals=True)
    seen = out["alpha"] > 1e-3
    assert seen.sum() > 20
    n = grad / np.linalg.norm(grad)
    ratio = out["normal"][:, seen] / out["alpha"][seen]
    # the corner values are stored in float32: linear up to 1e-7 relative
    assert np.allclose(ratio, n[:, None], rtol=1e-6, atol=1e-9)
    assert np.ptp(ratio, axis=1).max() < 1e-12          # one normal for every ray
    assert (out["normal"][:, ~(out["alpha"] > 0)] == 0).all()


def test_normal_gradient_matches_finite_differences():
    """d(sum g_N . N + g_rgb . C + ...) / d grid by central differences of the
    oracle's own images vs its analytic backward through the normalisation and
    Eq. (interp_grad_grad), on a random tiny octree with two samples."""
    sc = synth.random_octree_scene(61, max_level=3, p_split=0.4, max_cells=30,
                                   grid_fn=synth.normal_grid(0.5, 1.5))
    cam = synth.orbit_camera(9, 10, 9, distance=1.6)
    H, W = cam.height, cam.width
    rng = np.random.default_rng(5)
    g_rgb, g_d, g_a = (rng.normal(size=(3, H, W)), rng.normal(size=(H, W)), rng.normal(size=(H, W)))
    g_n = rng.normal(size=(3, H, W))
    d_grid, _ = oracle.render_grad(sc, cam, g_rgb, g_d, g_a, K=2, t_stop=0.0, g_normal=g_n)
    grid0 = sc.grid.astype(np.float64)

    def loss(grid):
        o = oracle.render(sc, cam, K=2, t_stop=0.0, grid=grid, normals=True)
        return float((g_rgb * o["rgb"]).sum() + (g_d * o["depth"]).sum() + (g_a * o["alpha"]).sum()
                     + (g_n * o["normal"]).sum())

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
    assert scale > 0
    assert np.abs(d_grid[idx] - fd).max() <= 1e-6 * scale + 1e-9
    # the normal term is a real part of it: without g_normal the gradient differs
    d0, _ = oracle.render_grad(sc, cam, g_rgb, g_d, g_a, K=2, t_stop=0.0)
    assert np.abs(d0[idx] - fd).max() > 1e-3 * scale


# ------------------------------------------------ pruning / subdivision

def _two_voxel_column(x_front, x_back, sh_front, sh_back):
    """Level-2 voxels (1, 1, 0) and (1, 1, 2) on the axis of _axis_camera, with
    constant raw densities and constant (DC-only) colours."""
    cells = synth.scenes.dense_cells(2)
    pick = [np.where((cells.ijk == ijk).all(1))[0][0] for ijk in ((1, 1, 0), (1, 1, 2))]
    cells = cells.take(np.array(pick))
    sc = synth.scenes.make_scene(cells, synth.constant_grid(0.0), 0.0, np.random.default_rng(0), shuffle=False)
    sc.grid[sc.corner_idx[0]] = x_front
    sc.grid[sc.corner_idx[1]] = x_back
    sc.sh[:] = 0.0
    sc.sh[0, 0:3] = sh_front
    sc.sh[1, 0:3] = sh_back
    return sc


def _explin(x):
    return x if x > 1.1 else 1.1 * math.exp(x / 1.1 - 1.0)


def _column_alphas(cam, x, y, sc):
    """Closed-form alphas of the two voxels along pixel (x, y) (the camera
    axis is world +z, voxel z-extents [0, .25] and [.5, .75])."""
    ro, rd = oracle.pixel_ray(cam, x, y)
    out = []
    for v, (z0, z1) in enumerate(((0.0, 0.25), (0.5, 0.75))):
        a, b, ok = oracle.ray_aabb(sc.centre[v].astype(np.float64), 0.25, ro, rd)
        if not ok:
            out.append(0.0)
            continue
        sigma = _explin(float(sc.grid[sc.corner_idx[v][0]]))
        out.append(1.0 - math.exp(-sigma * (b - a) * np.linalg.norm(rd)))
    return out


def test_max_weight_and_priority_closed_forms():
    """Two constant-density voxels in a column: per pixel the weights are
    alpha_1 and (1 - alpha_1) alpha_2, and with L = g . C + g_A A,
    dL/dalpha_1 = T_1 (g . (c_1 - RC_1) + g_A (1 - alpha_2)), RC_1 = alpha_2 c_2
    + (1 - alpha_2) bg, and dL/dalpha_2 = (1 - alpha_1) (g . (c_2 - bg) + g_A);
    the maximum weight is the largest weight over the pixels and the priority
    the sum of |alpha dL/dalpha| (Eq. priority)."""
    sc = _two_voxel_column(0.9, 2.4, 0.8, -0.5)
    cam = synth.look_at((0.375, 0.375, -2.0), (0.375, 0.375, 0.5), (0, 1, 0), 12.0, 14, 12)
    bg = np.array([0.2, 0.1, 0.4], np.float32).astype(np.float64)   # the renderer's float32 inputs
    H, W = cam.height, cam.width
    rng = np.random.default_rng(2)
    g_rgb, g_a = rng.normal(size=(3, H, W)), rng.normal(size=(H, W))
    g_d = np.zeros((H, W))
    Y0 = 0.5 / math.sqrt(math.pi)
    c = [max(0.0, Y0 * float(sc.sh[0, 0])), max(0.0, Y0 * float(sc.sh[1, 0]))]   # DC colours, clamped
    mw = np.zeros(sc.n_vox)
    oracle.render(sc, cam, K=1, t_stop=0.0, bg=tuple(bg), max_weight=mw)
    pr = np.zeros(sc.n_vox)
    oracle.render_grad(sc, cam, g_rgb, g_d, g_a, K=1, t_stop=0.0, bg=tuple(bg), priority=pr)
    want_mw = np.zeros(2)
    want_pr = np.zeros(2)
    n_both = 0
    for y in range(H):
        for x in range(W):
            a1, a2 = _column_alphas(cam, x, y, sc)
            n_both += a1 > 0 and a2 > 0
            g = g_rgb[:, y, x]
            want_mw[0] = max(want_mw[0], a1)
            want_mw[1] = max(want_mw[1], (1 - a1) * a2)
            rc1 = a2 * c[1] + (1 - a2) * bg
            d1 = (g @ (c[0] - rc1)) + g_a[y, x] * (1 - a2)
            d2 = (1 - a1) * ((g @ (c[1] - bg)) + g_a[y, x])
            want_pr[0] += abs(a1 * d1) if a1 > 0 else 0.0
            want_pr[1] += abs(a2 * d2) if a2 > 0 else 0.0
    assert n_both > 20
    assert np.allclose(mw, want_mw, rtol=1e-12, atol=0)
    assert np.allclose(pr, want_pr, rtol=1e-10, atol=0)


def test_max_weight_accumulates_over_views_and_stops_with_the_walk():
    """The statistic is raised, never lowered, over successive views, and a
    voxel behind the one that stopped the walk gets no weight from that
    pixel (Sec. 3.1.2 early termination)."""
    sc = _two_voxel_column(60.0, 2.0, 0.5, 0.5)               # opaque front voxel: T < 1e-6 behind it
    cam = synth.look_at((0.375, 0.375, -2.0), (0.375, 0.375, 0.5), (0, 1, 0), 12.0, 14, 12)
    mw = np.zeros(sc.n_vox)
    oracle.render(sc, cam, K=1, t_stop=1e-4, max_weight=mw)
    assert mw[0] > 0.99 and mw[1] == 0.0
    mw2 = mw.copy()
    side = synth.look_at((0.375, 2.5, 0.625), (0.375, 0.375, 0.625), (0, 0, 1), 12.0, 14, 12)
    oracle.render(sc, side, K=1, t_stop=1e-4, max_weight=mw2)   # sees the back voxel alone
    assert mw2[0] == mw[0] and mw2[1] > 0.0
