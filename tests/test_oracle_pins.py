"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one part of the oracle to something other than itself: values
the paper prints, closed forms, invariants, brute force on tiny inputs or
finite differences.  No GPU.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import binning, morton
from tests.conftest import read_golden


# ----------------------------------------------------------------- Morton code

def test_octpath_hand_examples():
    """Worked examples of the bit interleaving (Sec. A.1)."""
    for i, j, k, l, code in read_golden("octpath_cases.txt"):
        assert int(morton.octpath(i, j, k, l)) == code, (i, j, k, l)


def test_octpath_round_trip_brute_force():
    """to_voxel_index(to_octpath(ijk, l), l) == ijk for every index, l <= 4, and
    codes of one level are distinct and ordered like the interleaved bits."""
    for l in range(1, 5):
        n = 1 << l
        i, j, k = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
        i, j, k = i.ravel(), j.ravel(), k.ravel()
        code = morton.octpath(i, j, k, l)
        ii, jj, kk = morton.voxel_index(code, l)
        assert (ii == i).all() and (jj == j).all() and (kk == k).all()
        assert len(np.unique(code)) == n ** 3
        # codes are left aligned: the low 3 (16 - l) bits are zero
        assert (code & np.uint64((1 << (3 * (16 - l))) - 1) == 0).all()


def test_order_table_matches_printed_table():
    """The oracle derives the table from geometry; the paper prints it."""
    printed = np.array(read_golden("order_table.txt"))
    assert (morton.order_table() == printed).all()


def test_printed_table_is_xor():
    """Sec. B.2 notes the table lookup is a single xor per code: table[s][b] = b ^ s."""
    printed = np.array(read_golden("order_table.txt"))
    s, b = np.meshgrid(np.arange(8), np.arange(8), indexing="ij")
    assert (printed == (s ^ b)).all()


def test_signbits_definition():
    rd = np.array([[1, 1, 1], [-1, 1, 1], [1, -1, 1], [1, 1, -1], [-1, -1, -1], [0.0, -0.0, 1]])
    assert list(morton.signbits(rd)) == [0, 4, 2, 1, 7, 0]


@pytest.mark.parametrize("seed", range(6))
def test_morton_order_equals_depth_order(seed):
    """Sec. B.3: for a non-overlapping octree, sorting the voxels a ray hits by
    the direction-dependent Morton order of the ray's sign pattern gives the
    near-to-far order (brute force on random octrees and random rays)."""
    rng = np.random.default_rng(seed)
    scene = synth.random_octree_scene(seed, max_level=6, p_split=0.45)
    code, ok = binning.voxel_octpath(scene)
    assert ok.all()
    checked = 0
    for _ in range(40):
        ro = np.array([0.5, 0.5, 0.5]) + rng.normal(size=3) * 1.5
        target = rng.uniform(0.1, 0.9, size=3)
        rd = target - ro
        a, b, v = oracle.ray_hits(scene, ro, rd)
        keep = (b - a) > 1e-9 * np.linalg.norm(rd)      # proper segments only
        a, b, v = a[keep], b[keep], v[keep]
        if len(v) < 2:
            continue
        s = int(morton.signbits(rd))
        order = morton.dir_dep_order(code[v], s)
        by_morton = v[np.argsort(order, kind="stable")]
        assert list(by_morton) == list(v), (seed, s)
        checked += 1
    assert checked > 10


# ------------------------------------------------------------------- lattice

def test_lattice_index_matches_generator():
    """Centres are read as cell centres w_c - w_s/2 + v_s (ijk + 1/2): the
    oracle recovers the generator's indices (made by recursive splitting)."""
    for scene in (synth.dense_scene(3), synth.random_octree_scene(3, max_level=7)):
        ijk, ok = binning.lattice_index(scene)
        assert ok.all()
        assert (ijk == scene.ijk).all()


def test_lattice_rejects_off_lattice_and_bad_level():
    scene = synth.dense_scene(2)
    bad = synth.scenes.Scene(**{**scene.__dict__})
    bad.centre = scene.centre.copy()
    bad.centre[3, 0] += 0.4 * 0.25      # 0.4 cell off
    bad.level = scene.level.copy()
    bad.level[5] = 17
    _, ok = binning.lattice_index(bad)
    assert not ok[3] and not ok[5] and ok.sum() == scene.n_vox - 2


# ------------------------------------------------------------------- camera

def test_pixel_ray_projects_back_to_pixel():
    """The pixel ray of (x, y) passes through pixel centre (x+.5, y+.5) at
    camera depth t, and the principal point's ray is the viewing axis."""
    cam = synth.orbit_camera(3, 64, 48)
    R = cam.w2c[:, :3].astype(np.float64)
    t = cam.w2c[:, 3].astype(np.float64)
    rng = np.random.default_rng(0)
    for _ in range(20):
        x, y = rng.integers(0, 64), rng.integers(0, 48)
        ro, rd = oracle.pixel_ray(cam, x, y)
        for depth in (0.5, 2.0):
            X = R @ (ro + depth * rd) + t
            assert abs(X[2] - depth) < 1e-6
            u = float(cam.fx) * X[0] / X[2] + float(cam.cx)
            v = float(cam.fy) * X[1] / X[2] + float(cam.cy)
            assert abs(u - (x + 0.5)) < 1e-5 and abs(v - (y + 0.5)) < 1e-5
    ro, rd = oracle.pixel_ray(cam, float(cam.cx) - 0.5, float(cam.cy) - 0.5)
    assert np.allclose(rd / np.linalg.norm(rd), R[2], atol=1e-6)


# ------------------------------------------------------------------- explin

def test_explin_properties():
    """Eq. (explin): identity above 1.1, exponential below, C^1 at 1.1."""
    assert oracle.explin(1.1) == pytest.approx(1.1, abs=1e-15)
    h = 1e-7
    left = (oracle.explin(1.1) - oracle.explin(1.1 - h)) / h
    right = (oracle.explin(1.1 + h) - oracle.explin(1.1)) / h
    assert left == pytest.approx(1.0, abs=1e-5) and right == pytest.approx(1.0, abs=1e-9)
    for x in (1.2, 3.0, 50.0):
        assert oracle.explin(x) == x
    # below the knee: multiplying by e every 1.1 units of x (exp(x/1.1 + const))
    for x in (-10.0, -1.0, 0.0, 1.0):
        assert oracle.explin(x) / oracle.explin(x - 1.1) == pytest.approx(math.e, rel=1e-12)
        assert oracle.explin(x) > 0
    # derivative against central differences (smooth away from the knee)
    for x in (-5.0, 0.3, 1.0, 2.0):
        fd = (oracle.explin(x + 1e-6) - oracle.explin(x - 1e-6)) / 2e-6
        assert oracle.explin_grad(x) == pytest.approx(fd, rel=1e-7)
    # shape of softplus: monotone, positive, asymptotically the identity
    xs = np.linspace(-8, 8, 200)
    e = np.array([oracle.explin(x) for x in xs])
    sp = np.log1p(np.exp(xs))
    assert (np.diff(e) > 0).all() and (e > 0).all()
    assert abs(e[-1] - sp[-1]) < 1e-3


# ----------------------------------------------------------------------- SH

def _sphere_quadrature(n_theta=24, n_phi=48):
    z, w = np.polynomial.legendre.leggauss(n_theta)
    phi = (np.arange(n_phi) + 0.5) * 2 * np.pi / n_phi
    Z, P = np.meshgrid(z, phi, indexing="ij")
    W = np.repeat(w[:, None], n_phi, 1) * (2 * np.pi / n_phi)
    s = np.sqrt(1 - Z ** 2)
    dirs = np.stack([s * np.cos(P), s * np.sin(P), Z], -1).reshape(-1, 3)
    return dirs, W.reshape(-1)


def test_sh_orthonormal():
    """The 16 real SH functions are orthonormal on the sphere (exact
    Gauss-Legendre x trapezoid quadrature for degree <= 6 polynomials)."""
    dirs, w = _sphere_quadrature()
    Y = np.array([oracle.sh_basis(d) for d in dirs])
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye(16)).max() < 1e-10


def test_sh_degree_structure():
    """Index l*l + l + m holds degree l, order m: Y_0^0 = 1/(2 sqrt(pi));
    zonal Y_l^0(+z) = sqrt((2l+1)/(4 pi)); degree 1 is proportional to
    (y, z, x); rotating about z by g maps (Y_l^m, Y_l^-m) by a rotation of
    angle m g (no Condon-Shortley phase: Y_l^l > 0 on +x)."""
    assert oracle.sh_basis([0, 0, 1])[0] == pytest.approx(0.5 / math.sqrt(math.pi), rel=1e-14)
    Yz = oracle.sh_basis([0, 0, 1])
    for l in range(4):
        assert Yz[l * l + l] == pytest.approx(math.sqrt((2 * l + 1) / (4 * math.pi)), rel=1e-13)
    c1 = math.sqrt(3 / (4 * math.pi))
    for d, expect in (([1, 0, 0], [0, 0, c1]), ([0, 1, 0], [c1, 0, 0]), ([0, 0, 1], [0, c1, 0])):
        assert np.allclose(oracle.sh_basis(d)[1:4], expect, atol=1e-14)
    rng = np.random.default_rng(0)
    for _ in range(10):
        d = rng.normal(size=3)
        g = rng.uniform(0, 2 * np.pi)
        Rz = np.array([[math.cos(g), -math.sin(g), 0], [math.sin(g), math.cos(g), 0], [0, 0, 1]])
        Y0 = oracle.sh_basis(d)
        Y1 = oracle.sh_basis(Rz @ d)
        for l in range(1, 4):
            for m in range(1, l + 1):
                cp, sp = Y0[l * l + l + m], Y0[l * l + l - m]
                rc = math.cos(m * g) * cp - math.sin(m * g) * sp
                rs = math.sin(m * g) * cp + math.cos(m * g) * sp
                assert Y1[l * l + l + m] == pytest.approx(rc, abs=1e-12)
                assert Y1[l * l + l - m] == pytest.approx(rs, abs=1e-12)
    for l in range(1, 4):
        assert oracle.sh_basis([1, 0, 0])[l * l + 2 * l] > 0


# ---------------------------------------------------- closed-form renderings

def _axis_camera(width=32, height=32, z_eye=-2.0, fov=20.0, target=(0.5, 0.5, 0.5)):
    """Camera on the -z side of the cube looking along +z (world z = camera z)."""
    return synth.look_at((target[0], target[1], z_eye), target, (0, 1, 0), fov, width, height)


def _front_back(cam, x, y, z0, z1):
    """Closed-form segment of a pixel ray between the planes z = z0 and z1 for
    a camera whose viewing axis is world +z: camera depth = world z - z_eye."""
    ro, rd = oracle.pixel_ray(cam, x, y)
    a = (z0 - ro[2]) / rd[2]
    b = (z1 - ro[2]) / rd[2]
    return ro, rd, a, b


def _single_voxel_scene(level, ijk, value, sh_dc=0.0):
    cells = synth.scenes.dense_cells(level)
    sel = np.where((cells.ijk == np.asarray(ijk)).all(1))[0]
    cells = cells.take(sel)
    rng = np.random.default_rng(0)
    sc = synth.scenes.make_scene(cells, synth.constant_grid(value), 0.0, rng)
    sc.sh[:] = 0.0
    sc.sh[:, 0:3] = sh_dc
    return sc


@pytest.mark.parametrize("K", [1, 2, 3])
@pytest.mark.parametrize("value", [-3.0, 0.5, 2.5])
def test_constant_density_voxel(K, value):
    """One voxel with all 8 corners = x: density explin(x) is constant, so
    alpha = 1 - exp(-explin(x) * l) for any K, and the voxel depth is the
    K-sample sum of Sec. A.4 with beta = 1 - exp(-explin(x) l / K)."""
    sc = _single_voxel_scene(1, (1, 1, 1), value, sh_dc=1.0)
    cam = _axis_camera()
    sigma = {-3.0: 1.1 * math.exp(-3.0 / 1.1 - 1.0), 0.5: 1.1 * math.exp(0.5 / 1.1 - 1.0), 2.5: 2.5}[value]
    # voxel (1,1,1) at level 1 spans [0.5, 1]^3; pick pixels whose rays cross
    # both the front and the back face
    pix = []
    for x in range(32):
        for y in range(32):
            ro, rd, a, b = _front_back(cam, x, y, 0.5, 1.0)
            pf, pb = ro + a * rd, ro + b * rd
            if (0.5 < pf[:2]).all() and (pf[:2] < 1).all() and (0.5 < pb[:2]).all() and (pb[:2] < 1).all():
                pix.append((x, y, a, b, np.linalg.norm(rd)))
    assert len(pix) > 5
    out = oracle.render(sc, cam, K=K, t_stop=0.0, pixels=[(p[0], p[1]) for p in pix])
    y00 = 0.5 / math.sqrt(math.pi)
    for n, (x, y, a, b, rdn) in enumerate(pix):
        ell = (b - a) * rdn
        alpha = 1 - math.exp(-sigma * ell)
        assert out["alpha"][n] == pytest.approx(alpha, rel=1e-12)
        beta = 1 - math.exp(-sigma * ell / K)
        tk = [a + (k - 0.5) / K * (b - a) for k in range(1, K + 1)]
        d = sum((1 - beta) ** (k - 1) * beta * tk[k - 1] for k in range(1, K + 1))
        assert out["depth"][n] == pytest.approx(d, rel=1e-12)
        assert out["rgb"][n] == pytest.approx([alpha * y00] * 3, rel=1e-12)


@pytest.mark.parametrize("K", [1, 2, 3])
def test_uniform_grid_transmittance(K):
    """Dense level-3 grid with every grid point = x: along a ray the optical
    depths of consecutive voxel segments telescope to sigma times the path
    length inside the cube, T_final = exp(-sigma * path), for any K, and a
    constant colour c composites to c (1 - T_final)."""
    x = 0.375                      # exact in float32, the inputs' precision
    sigma = 1.1 * math.exp(x / 1.1 - 1.0)
    sc = synth.dense_scene(3, grid_fn=synth.constant_grid(x), sh_std=0.0)
    sc.sh[:, 0:3] = 0.75
    cam = _axis_camera(48, 48, fov=20.0)
    pix = []
    for px in range(0, 48, 3):
        for py in range(0, 48, 3):
            ro, rd, a, b = _front_back(cam, px, py, 0.0, 1.0)
            pf, pb = ro + a * rd, ro + b * rd
            if (0 < pf[:2]).all() and (pf[:2] < 1).all() and (0 < pb[:2]).all() and (pb[:2] < 1).all():
                pix.append((px, py, (b - a) * np.linalg.norm(rd)))
    assert len(pix) > 20
    out = oracle.render(sc, cam, K=K, t_stop=0.0, pixels=[(p[0], p[1]) for p in pix])
    for n, (_, _, path) in enumerate(pix):
        T = math.exp(-sigma * path)
        assert out["t_final"][n] == pytest.approx(T, rel=1e-11)
        c = 0.75 * 0.5 / math.sqrt(math.pi)
        assert out["rgb"][n] == pytest.approx([c * (1 - T)] * 3, rel=1e-10)


def test_linear_field_midpoint_exact():
    """Corner values V_ijk = g.(i,j,k) + h, all > 1.1: the density is linear
    inside the voxel, trilinear interpolation reproduces it, and the K = 1
    midpoint rule is exact: alpha = 1 - exp(-l * sigma(midpoint))."""
    sc = _single_voxel_scene(1, (0, 0, 0), 0.0)
    g = np.array([0.7, -0.4, 1.3])
    h = 2.0
    bits = np.array([[(c >> 2) & 1, (c >> 1) & 1, c & 1] for c in range(8)], np.float64)
    grid = np.zeros(sc.n_pts)
    grid[sc.corner_idx[0]] = bits @ g + h
    cam = _axis_camera(32, 32, fov=20.0, target=(0.25, 0.25, 0.25))
    pix = []
    for x in range(32):
        for y in range(32):
            ro, rd, a, b = _front_back(cam, x, y, 0.0, 0.5)
            pf, pb = ro + a * rd, ro + b * rd
            if (0 < pf[:2]).all() and (pf[:2] < 0.5).all() and (0 < pb[:2]).all() and (pb[:2] < 0.5).all():
                mid = ro + 0.5 * (a + b) * rd
                q = mid / 0.5                          # local coordinates of the level-1 voxel at the origin
                pix.append((x, y, (b - a) * np.linalg.norm(rd), q @ g + h))
    assert len(pix) > 5
    out = oracle.render(sc, cam, K=1, t_stop=0.0, pixels=[(p[0], p[1]) for p in pix], grid=grid)
    for n, (_, _, ell, sig) in enumerate(pix):
        assert out["alpha"][n] == pytest.approx(1 - math.exp(-ell * sig), rel=1e-12)


def test_early_termination_rule():
    """Sec. 3.1.2: compositing stops after the voxel that leaves T < t_stop.
    With one constant colour c the stopped pixel is exactly c (1 - T_stop)."""
    sc = synth.dense_scene(3, grid_fn=synth.constant_grid(3.0), sh_std=0.0)
    sc.sh[:, 0:3] = 0.75
    c = 0.75 * 0.5 / math.sqrt(math.pi)
    cam = _axis_camera(16, 16, fov=20.0)
    full = oracle.render(sc, cam, K=2, t_stop=0.0)
    cut = oracle.render(sc, cam, K=2, t_stop=0.2)
    hit = full["n_comp"] > 0
    assert (cut["n_comp"][hit] < full["n_comp"][hit]).any()
    stopped = cut["term_vox"] >= 0
    assert stopped.any()
    assert (cut["t_final"][stopped] < 0.2).all()
    # T before the stopping voxel was still >= t_stop: undoing its alpha
    # (one voxel's optical depth, at most sigma * diagonal) lands above 0.2
    assert np.allclose(cut["rgb"], c * (1 - cut["t_final"])[None], rtol=0, atol=1e-12)
    assert (cut["t_final"][~stopped] == full["t_final"][~stopped]).all()


# ------------------------------------------------------------------ gradients

def _fd_check(sc, cam, K, t_stop, bg, seed, n_grid=None, n_sh=None, h=1e-6):
    H, W = cam.height, cam.width
    g_rgb, g_depth, g_alpha = synth.upstream_grads(seed, H, W)
    g_rgb = g_rgb.astype(np.float64)
    d_grid, d_sh = oracle.render_grad(sc, cam, g_rgb, g_depth, g_alpha, K=K, t_stop=t_stop, bg=bg)
    grid0 = sc.grid.astype(np.float64)
    sh0 = sc.sh.astype(np.float64)

    def loss(grid, sh):
        o = oracle.render(sc, cam, K=K, t_stop=t_stop, bg=bg, grid=grid, sh=sh)
        return float((g_rgb * o["rgb"]).sum() + (g_depth * o["depth"]).sum()
                     + (g_alpha * o["alpha"]).sum()), o

    _, base = loss(grid0, sh0)
    rng = np.random.default_rng(seed)
    gi = np.arange(len(grid0)) if n_grid is None else rng.choice(len(grid0), n_grid, replace=False)
    fd_g = []
    for i in gi:
        gp = grid0.copy(); gp[i] += h
        gm = grid0.copy(); gm[i] -= h
        lp, op = loss(gp, sh0)
        lm, om = loss(gm, sh0)
        assert (op["n_comp"] == base["n_comp"]).all() and (om["n_comp"] == base["n_comp"]).all()
        fd_g.append((lp - lm) / (2 * h))
    fd_g = np.array(fd_g)
    flat = sh0.reshape(-1)
    si = np.arange(len(flat)) if n_sh is None else rng.choice(len(flat), n_sh, replace=False)
    fd_s = []
    for i in si:
        sp = flat.copy(); sp[i] += h
        sm = flat.copy(); sm[i] -= h
        lp, _ = loss(grid0, sp.reshape(sh0.shape))
        lm, _ = loss(grid0, sm.reshape(sh0.shape))
        fd_s.append((lp - lm) / (2 * h))
    fd_s = np.array(fd_s)
    an_g = d_grid[gi]
    an_s = d_sh.reshape(-1)[si]
    scale_g = np.abs(fd_g).max() + 1e-30
    scale_s = np.abs(fd_s).max() + 1e-30
    assert np.abs(an_g - fd_g).max() <= 1e-6 * scale_g + 1e-9, np.abs(an_g - fd_g).max()
    assert np.abs(an_s - fd_s).max() <= 1e-6 * scale_s + 1e-9, np.abs(an_s - fd_s).max()
    assert np.linalg.norm(an_g - fd_g) <= 1e-6 * np.linalg.norm(fd_g) + 1e-9
    assert np.abs(fd_g).max() > 0 and np.abs(fd_s).max() > 0


@pytest.mark.parametrize("K,bg", [(1, (0.0, 0.0, 0.0)), (2, (0.2, -0.1, 0.5)), (3, (0.0, 0.3, 0.0))])
def test_gradient_matches_finite_differences(K, bg):
    """Analytic FP64 gradient (alpha form) vs central differences, h = 1e-6,
    on a random tiny octree: grid densities and every SH coefficient."""
    sc = synth.random_octree_scene(11 + K, max_level=3, p_split=0.4, max_cells=40,
                                   grid_fn=synth.normal_grid(0.5, 1.5))
    cam = synth.orbit_camera(5 + K, 12, 10, distance=1.6)
    _fd_check(sc, cam, K, 0.0, bg, seed=K, n_grid=None, n_sh=200)


def test_gradient_with_termination_matches_fd():
    """Same check with early termination active (no decision flips at h)."""
    sc = synth.random_octree_scene(21, max_level=3, p_split=0.5, max_cells=48,
                                   grid_fn=synth.normal_grid(4.0, 1.0))
    cam = synth.orbit_camera(2, 10, 10, distance=1.6)
    o = oracle.render(sc, cam, K=3, t_stop=0.3)
    assert (o["term_vox"] >= 0).any() and not o["near_stop"].any()
    _fd_check(sc, cam, 3, 0.3, (0.1, 0.1, 0.1), seed=7, n_grid=80, n_sh=80)


# ------------------------------------------------------- binning brute force

@pytest.mark.parametrize("seed", range(4))
def test_tile_lists_conservative_and_ordered(seed):
    """Brute force on tiny inputs (<= 64 voxels, small image): every voxel a
    pixel ray enters (proper segment) appears in that pixel's tile list with
    the pixel's sign bits, and the pixel's sub-list, in sorted key order,
    lists its hits near to far (Sec. B.1)."""
    sc = synth.random_octree_scene(seed, max_level=4, p_split=0.5, max_cells=64)
    cam = synth.orbit_camera(seed, 40, 24, distance=1.5 + 0.3 * seed)
    tile = 16
    ntx, nty = binning.tile_grid(cam, tile)
    masks, either = binning.tile_masks(cam, tile)
    keys, vals, counts = binning.emit_pairs(sc, cam, tile, masks)
    sk, sv = binning.sort_pairs(keys, vals)
    rng_ = binning.tile_ranges(sk, ntx * nty)
    assert counts.sum() == len(keys)
    ro, rd = binning.pixel_rays(cam)
    s_px = morton.signbits(rd)
    checked = 0
    for y in range(cam.height):
        for x in range(cam.width):
            t = (y // tile) * ntx + x // tile
            b, e = rng_[t]
            lst = sv[b:e]
            s = s_px[y, x]
            vox = (lst & 0x1FFFFFFF)[(lst >> 29) == s]
            a, bb, v = oracle.ray_hits(sc, ro, rd[y, x])
            proper = (bb - a) > 1e-9
            v = v[proper]
            assert set(v.tolist()) <= set(vox.tolist())
            pos = {int(u): i for i, u in enumerate(vox)}
            seq = [pos[int(u)] for u in v]
            assert seq == sorted(seq)
            checked += len(v)
    assert checked > 0
    # keys are sorted, unique, and the value carries the key's sign pattern
    assert (np.diff(sk.astype(np.float64)) >= 0).all()
    assert len(np.unique(sk)) == len(sk)


def test_key_layout():
    """key = tile << 48 | Morton order (48 bits); value = s << 29 | voxel id."""
    sc = synth.random_octree_scene(5, max_level=3, max_cells=30)
    cam = synth.dense_view_camera(64, 64)
    keys, vals, _ = binning.emit_pairs(sc, cam)
    code, _ = binning.voxel_octpath(sc)
    vid = (vals & 0x1FFFFFFF).astype(np.int64)
    s = (vals >> 29).astype(np.int64)
    assert ((keys & np.uint64((1 << 48) - 1)) == morton.dir_dep_order(code[vid], s)).all()
    assert ((keys >> np.uint64(48)) < np.uint64(16)).all()


def test_colour_uses_direction_to_voxel_centre():
    """Eq. (vox_color): one colour per voxel and view, from the SH evaluated
    toward normalize(centre - camera position), clamped at 0.  With only the
    (l=1, m=1) coefficient set, c = max(0, sqrt(3/(4 pi)) * dir_x) for every
    pixel that sees the voxel, whatever its own ray direction."""
    sc = _single_voxel_scene(2, (1, 2, 1), 20.0)          # opaque voxel
    sc.sh[:] = 0.0
    sc.sh[0, 3 * 3 + 0] = 1.0                              # red, index l*l + l + m = 3
    sc.sh[0, 3 * 3 + 1] = -1.0                             # green, negative: clamped to 0
    eye = np.array([-1.5, 0.9, -1.2])
    cam = synth.look_at(eye, (0.375, 0.625, 0.375), (0, 1, 0), 30.0, 24, 24)
    out = oracle.render(sc, cam, K=1, t_stop=0.0)
    centre = sc.centre[0].astype(np.float64)
    d = centre - eye
    d /= np.linalg.norm(d)
    c = math.sqrt(3 / (4 * math.pi)) * d[0]
    assert c > 0
    seen = out["alpha"] > 0.5
    assert seen.sum() > 10
    ratio = out["rgb"][0][seen] / out["alpha"][seen]
    assert np.allclose(ratio, c, rtol=1e-6)
    assert (out["rgb"][1] == 0).all() and (out["rgb"][2] == 0).all()


def test_gradient_magnitudes():
    """The oracle's contribution magnitudes (sum of |term| per gradient
    element): never below |gradient|; equal to it where an element has one
    term (one pixel through one voxel, K = 1); unchanged when every upstream
    gradient flips sign (the gradient flips); doubled when they double."""
    sc = _single_voxel_scene(2, (1, 2, 1), 1.5, sh_dc=0.7)
    sc.grid[:] = np.linspace(0.5, 2.5, sc.n_pts).astype(np.float32)
    cam = synth.look_at((-1.2, 0.8, -1.5), (0.375, 0.625, 0.375), (0, 1, 0), 25.0, 16, 16)
    ref = oracle.render(sc, cam, K=1, t_stop=0.0)
    y, x = np.unravel_index(np.argmax(ref["alpha"]), ref["alpha"].shape)
    assert ref["n_comp"][y, x] == 1
    px = np.array([[x, y]])
    up = (np.array([[0.3, -1.2, 0.8]]), np.array([0.5]), np.array([-0.7]))
    mag = {}
    g, s = oracle.render_grad(sc, cam, *up, K=1, t_stop=0.0, pixels=px, magnitudes=mag)
    assert np.allclose(mag["grid"], np.abs(g), rtol=1e-12, atol=0)
    assert np.allclose(mag["sh"], np.abs(s), rtol=1e-12, atol=0)
    # the segment-weighted magnitudes carry the condition number of the hit's
    # length b - a: perturbing the voxel's planes, the origin and the
    # direction by relative 1e-9 moves b - a by at most 1e-9 kappa (first
    # order), and some perturbation comes within a factor 4 of it
    ro, rd = oracle.pixel_ray(cam, x, y)
    vs = float(sc.world_size) / 4
    c0 = sc.centre[0].astype(np.float64)
    a, b, ok = oracle.ray_aabb(c0, vs, ro, rd)
    assert ok and b > a
    kappa = mag["grid_seg"][mag["grid"] > 0] / mag["grid"][mag["grid"] > 0]
    assert np.allclose(kappa, kappa[0], rtol=1e-12) and np.allclose(mag["sh_seg"][mag["sh"] > 0] /
                                                                    mag["sh"][mag["sh"] > 0], kappa[0], rtol=1e-12)
    kappa = kappa[0]
    eps, worst = 1e-9, 0.0
    rng = np.random.default_rng(0)
    for _ in range(2000):
        sgn = rng.choice([-1.0, 1.0], size=(4, 3))
        lo = (c0 - vs / 2) * (1 + eps * sgn[0])
        hi = (c0 + vs / 2) * (1 + eps * sgn[1])
        o = ro * (1 + eps * sgn[2])
        d = rd * (1 + eps * sgn[3])
        t0, t1 = (lo - o) / d, (hi - o) / d
        aa, bb = np.minimum(t0, t1).max(), np.maximum(t0, t1).min()
        worst = max(worst, abs((bb - aa) - (b - a)) / (b - a) / eps)
    assert worst <= kappa * 1.01 and worst >= kappa / 4, (worst, kappa)
    # a whole image: many terms per element
    G = synth.upstream_grads(3, cam.height, cam.width)
    m1 = {}
    g1, s1 = oracle.render_grad(sc, cam, G[0].astype(np.float64), G[1], G[2], K=2, t_stop=0.0, magnitudes=m1)
    assert (m1["grid"] >= np.abs(g1) - 1e-15).all() and (m1["sh"] >= np.abs(s1) - 1e-15).all()
    assert (m1["grid"] > 1.5 * np.abs(g1)).any()           # some elements cancel
    m2 = {}
    g2, s2 = oracle.render_grad(sc, cam, -G[0].astype(np.float64), -G[1], -G[2], K=2, t_stop=0.0, magnitudes=m2)
    assert np.allclose(g2, -g1, rtol=1e-12, atol=1e-300) and np.allclose(m2["grid"], m1["grid"], rtol=1e-12)
    m3 = {}
    oracle.render_grad(sc, cam, 2 * G[0].astype(np.float64), 2 * G[1], 2 * G[2], K=2, t_stop=0.0, magnitudes=m3)
    assert np.allclose(m3["grid"], 2 * m1["grid"], rtol=1e-12) and np.allclose(m3["sh"], 2 * m1["sh"], rtol=1e-12)
