"""Pins of the oracle's tile binning that do not restate it.

Sec. 3.1.2 ("Projection to image space") assigns a voxel to every tile the
2-D bounding box of its eight projected corners overlaps; Sec. B.1
duplicates it once per ray sign pattern present in the tile.  The oracle's
``binning.voxel_rects`` and ``binning.tile_masks`` are held here to:

* hand-worked values (``tests/golden/rect_cases.txt``,
  ``tests/golden/tile_mask_cases.txt``), each derived in the file's comments;
* brute force by another route: pixel rays by inverting the 4x4 world-to-
  camera matrix instead of transposing R, corner projections through the
  3x4 matrix K [R | t] in homogeneous coordinates, and the tile set by
  enumerating every tile and intersecting rectangles, so a rectangle one
  tile too wide or too narrow, a missing clamp, or a mask with an extra or a
  missing bit fails.
No GPU.
"""
import numpy as np
import pytest

import synth
from oracle import binning
from tests.conftest import read_golden


def _camera(R, t, f, cx, cy, W, H):
    w2c = np.zeros((3, 4), np.float32)
    w2c[:, :3] = R
    w2c[:, 3] = t
    return synth.cameras.Camera(np.float32(f), np.float32(f), np.float32(cx), np.float32(cy), w2c, W, H)


def _one_voxel(wc, ws, level, ijk):
    """Scene of one voxel of `level` at lattice index ijk."""
    vs = ws * 2.0 ** -level
    centre = np.asarray(wc, np.float64) - 0.5 * ws + vs * (np.asarray(ijk, np.float64) + 0.5)
    cells = synth.scenes.Cells(ijk=np.array([ijk], np.int64), level=np.array([level], np.int64),
                               centre=centre[None], size=np.array([vs]))
    sc = synth.scenes.make_scene(cells, synth.constant_grid(0.0), 0.0, np.random.default_rng(0),
                                 center=wc, size=ws, shuffle=False)
    return sc


# ------------------------------------------------------------- hand-worked

def test_tile_masks_hand_worked():
    for row in read_golden("tile_mask_cases.txt"):
        rx, rz, W, H, f, cx, cy, tile = row[:8]
        want = row[8:]
        cam = _camera(np.diag([rx, 1, rz]).astype(np.float32), (0, 0, 0), f, cx, cy, W, H)
        mask, either = binning.tile_masks(cam, tile)
        assert not either.any()
        assert mask.tolist() == want, (row, mask.tolist())


def test_voxel_rects_hand_worked():
    cam = _camera(np.eye(3, dtype=np.float32), (0, 0, 0), 90, 60, 70, 128, 128)
    for row in read_golden("rect_cases.txt"):
        wc, ws, level, ijk, tile = row[0:3], row[3], row[4], row[5:8], row[8]
        want = row[9:13]
        sc = _one_voxel(wc, float(ws), level, ijk)
        rect, amb = binning.voxel_rects(sc, cam, tile)
        assert not amb[0], row
        assert rect[0].tolist() == want, (row, rect[0].tolist())


# ------------------------------------------------------------- brute force

def _rays_by_inverse(cam):
    """Per-pixel ray direction from the inverted 4x4 [R | t]: the world point
    of the pixel at camera depth 1 minus the camera centre."""
    M = np.eye(4)
    M[:3, :] = np.asarray(cam.w2c, np.float32).astype(np.float64)
    Minv = np.linalg.inv(M)
    centre = Minv[:3, 3]
    fx, fy, cx, cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    dirs = np.zeros((cam.height, cam.width, 3))
    for y in range(cam.height):
        for x in range(cam.width):
            pc = np.array([(x + 0.5 - cx) / fx, (y + 0.5 - cy) / fy, 1.0, 1.0])
            dirs[y, x] = (Minv @ pc)[:3] - centre
    return dirs


@pytest.mark.parametrize("seed,tile", [(0, 16), (1, 16), (2, 8), (3, 32), (4, 16)])
def test_tile_masks_exact_by_brute_force(seed, tile):
    """Bit s of a tile's mask is set exactly when some in-image pixel of the
    tile has a ray with sign pattern s (no extra and no missing bit)."""
    W, H = 56, 40                                      # ragged for every tile size
    cam = synth.orbit_camera(seed, W, H, distance=2.0 + 0.2 * seed)
    # shift the principal point so that sign changes fall inside tiles
    cam = _camera(cam.R, cam.t, float(cam.fx), 0.37 * W + 3 * seed, 0.61 * H - 2 * seed, W, H)
    dirs = _rays_by_inverse(cam)
    ntx, nty = -(-W // tile), -(-H // tile)
    want = np.zeros(ntx * nty, np.int64)
    for y in range(H):
        for x in range(W):
            d = dirs[y, x]
            s = (4 if d[0] < 0 else 0) + (2 if d[1] < 0 else 0) + (1 if d[2] < 0 else 0)
            want[(y // tile) * ntx + x // tile] |= 1 << s
    mask, either = binning.tile_masks(cam, tile)
    assert (mask[~either] == want[~either]).all()
    assert either.sum() <= 1
    # the case mixes sign patterns, within a tile too
    assert max(bin(int(m)).count("1") for m in want) >= 2


def _projected_box(cam, corners):
    """(u_min, u_max, v_min, v_max, n_behind) of corners [8, 3] through the
    3x4 matrix K [R | t] in homogeneous coordinates."""
    Kmat = np.array([[float(np.float32(cam.fx)), 0.0, float(np.float32(cam.cx))],
                     [0.0, float(np.float32(cam.fy)), float(np.float32(cam.cy))],
                     [0.0, 0.0, 1.0]])
    P = Kmat @ np.asarray(cam.w2c, np.float32).astype(np.float64)
    us, vs, nb = [], [], 0
    for c in corners:
        h = P @ np.append(c, 1.0)
        if h[2] <= 1e-3:          # camera depth: the third row of P is the third row of [R | t]
            nb += 1
            continue
        us.append(h[0] / h[2])
        vs.append(h[1] / h[2])
    if nb:
        return None, None, None, None, nb
    return min(us), max(us), min(vs), max(vs), 0


def _overlapping_tiles(box, cam, tile):
    """Tiles whose pixel square [T tx, T tx + T) x [T ty, ...) and the image
    [0, W) x [0, H) both meet the closed box, by enumeration."""
    u0, u1, v0, v1 = box
    ntx, nty = -(-cam.width // tile), -(-cam.height // tile)
    out = set()
    for ty in range(nty):
        for tx in range(ntx):
            lo_u = max(u0, tile * tx, 0.0)
            hi_u = min(tile * (tx + 1), cam.width)
            lo_v = max(v0, tile * ty, 0.0)
            hi_v = min(tile * (ty + 1), cam.height)
            if lo_u < hi_u and lo_u <= u1 and lo_v < hi_v and lo_v <= v1:
                out.add((tx, ty))
    return out


def _near_edge(box, cam, tile, margin=1e-3):
    """True if a bound of the box lies within `margin` pixels of a tile edge
    or an image edge (where FP rounding may decide either way)."""
    for val, ext in ((box[0], cam.width), (box[1], cam.width), (box[2], cam.height), (box[3], cam.height)):
        r = val - tile * np.floor(val / tile)
        if r < margin or tile - r < margin or abs(val - ext) < margin or abs(val) < margin:
            return True
    return False


@pytest.mark.parametrize("seed,tile,dist", [(0, 16, 1.1), (1, 8, 1.35), (2, 32, 1.6), (3, 16, 1.85), (1, 16, 0.3),
                                           (3, 8, 0.3)])
def test_voxel_rects_tight_by_brute_force(seed, tile, dist):
    """The oracle's rectangle holds exactly the tiles the projected box
    overlaps inside the image: no tile too many (tightness) and none too few;
    a voxel with some corners behind the near plane takes the whole image and
    one with all of them behind, or with its box off the image, none."""
    sc = synth.random_octree_scene(seed + 40, max_level=4, p_split=0.5, max_cells=200)
    W, H = 72, 40
    # close: some voxels cross the image edges; at 0.3 the camera sits inside
    # the octree and many voxels cross the near plane
    cam = synth.orbit_camera(seed + 7, W, H, distance=dist)
    rect, amb = binning.voxel_rects(sc, cam, tile)
    ntx, nty = -(-W // tile), -(-H // tile)
    bits = np.array([[(b >> 2) & 1, (b >> 1) & 1, b & 1] for b in range(8)], np.float64)
    lv = sc.level.astype(np.int64)
    vs = float(sc.world_size) * 2.0 ** -lv
    lo = np.asarray(sc.world_center, np.float64) - 0.5 * float(sc.world_size)
    n_checked = n_skipped = n_partial = n_empty = 0
    for i in range(sc.n_vox):
        corners = lo + vs[i] * (sc.ijk[i].astype(np.float64) + bits)       # from the generator's lattice index
        u0, u1, v0, v1, nb = _projected_box(cam, corners)
        if nb == 8:
            assert rect[i, 0] > rect[i, 1], i
            n_empty += 1
            continue
        if nb > 0:
            assert rect[i].tolist() == [0, ntx - 1, 0, nty - 1], i
            n_partial += 1
            continue
        box = (u0, u1, v0, v1)
        if _near_edge(box, cam, tile):
            n_skipped += 1
            continue
        want = _overlapping_tiles(box, cam, tile)
        got = set()
        if rect[i, 0] <= rect[i, 1] and rect[i, 2] <= rect[i, 3]:
            got = {(tx, ty) for ty in range(rect[i, 2], rect[i, 3] + 1) for tx in range(rect[i, 0], rect[i, 1] + 1)}
        assert got == want, (i, box, rect[i].tolist())
        n_checked += 1
        n_empty += not want
    assert n_checked > 100 and n_skipped <= 0.02 * sc.n_vox
    assert amb.sum() <= 0.02 * sc.n_vox          # the oracle's own "either" set stays small
    assert n_empty > 0
    if dist < 0.5:
        assert n_partial > 10
