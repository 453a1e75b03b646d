"""Tile binning and sorting keys (oracle side, FP64 numpy).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Follows Sec. 3.1.2 ("Projection to image space", "Sorting voxels") and
Sec. B.1 (key/value layout):

* lattice index of each voxel from its centre and level (Eq. vox_coord, with
  the centre read as the cell centre: w_c - w_s/2 + v_s (ijk + 1/2));
* per-pixel ray sign bits, and per tile the set of sign patterns present
  among its in-image pixel rays (8-bit mask);
* per voxel the tile rectangle covered by the 2-D bounding box of its eight
  projected corners (all corners behind z = 1e-3: culled; some behind: the
  whole image);
* one (key, value) pair per (voxel, tile of the rectangle, sign pattern of
  the tile), emitted in voxel / row-major tile / sign order, with
  key = tile << 48 | dir_dep_order(octpath, s), value = s << 29 | voxel id;
* the pairs sorted by (key, value) and the [begin, end) range of each tile.

Rounding-sensitive decisions (a floor near a tile boundary, a cull test near
its threshold, a ray component near zero) are reported as "either" flags so a
comparison with FP32 results can exclude them.
"""
from __future__ import annotations

import numpy as np

from . import morton

NEAR = 1e-3
PX_MARGIN = 1e-3      # pixels, plus REL_MARGIN * |u|
REL_MARGIN = 1e-5
SIGN_MARGIN = 1e-6    # relative ray component treated as "zero"


def lattice_index(scene):
    """(ijk [N, 3] int64, ok [N] bool): nearest lattice cell of each centre and
    whether the centre lies within a quarter cell of it."""
    c = np.asarray(scene.centre, np.float32).astype(np.float64)
    lv = np.asarray(scene.level, np.int64)
    ws = float(np.float32(scene.world_size))
    wc = np.asarray(scene.world_center, np.float32).astype(np.float64)
    vs = ws * np.exp2(-lv.astype(np.float64))
    f = (c - (wc - 0.5 * ws)[None]) / vs[:, None] - 0.5
    ijk = np.rint(f)
    ok = (np.abs(f - ijk) <= 0.25).all(axis=1) & (lv >= 1) & (lv <= 16)
    ok &= ((ijk >= 0) & (ijk < np.exp2(lv)[:, None])).all(axis=1)
    return ijk.astype(np.int64), ok


def voxel_octpath(scene):
    ijk, ok = lattice_index(scene)
    lv = np.asarray(scene.level, np.int64)
    return morton.octpath(ijk[:, 0], ijk[:, 1], ijk[:, 2], np.clip(lv, 1, 16)), ok


def pixel_rays(cam):
    """ro [3], rd [H, W, 3] in FP64 (camera-space direction has z = 1)."""
    w2c = np.asarray(cam.w2c, np.float32).astype(np.float64)
    R, t = w2c[:, :3], w2c[:, 3]
    fx, fy, cx, cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    x = np.arange(cam.width, dtype=np.float64)
    y = np.arange(cam.height, dtype=np.float64)
    dx = (x + 0.5 - cx) / fx
    dy = (y + 0.5 - cy) / fy
    d = np.stack(np.broadcast_arrays(dx[None, :], dy[:, None], np.ones((1, 1))), axis=-1)
    rd = d @ R          # row vector times R == (R^T d)^T
    ro = -(R.T @ t)
    return ro, rd


def tile_grid(cam, tile=16):
    return (cam.width + tile - 1) // tile, (cam.height + tile - 1) // tile


def tile_masks(cam, tile=16):
    """mask [ntiles] uint8 (bit s set if some in-image pixel of the tile has
    sign pattern s), either [ntiles] bool (a pixel ray component is ~0)."""
    ntx, nty = tile_grid(cam, tile)
    _, rd = pixel_rays(cam)
    s = morton.signbits(rd)
    near0 = (np.abs(rd) < SIGN_MARGIN * np.linalg.norm(rd, axis=-1, keepdims=True)).any(-1)
    ty = np.arange(cam.height)[:, None] // tile
    tx = np.arange(cam.width)[None, :] // tile
    tid = (ty * ntx + tx).reshape(-1)
    mask = np.zeros(ntx * nty, np.uint8)
    np.bitwise_or.at(mask, tid, (1 << s.reshape(-1)).astype(np.uint8))
    either = np.zeros(ntx * nty, bool)
    np.logical_or.at(either, tid, near0.reshape(-1))
    return mask, either


def _floor_amb(u, tile):
    """floor(u / tile) and whether u is within the margin of a tile edge."""
    f = np.floor(u / tile)
    m = PX_MARGIN + REL_MARGIN * np.abs(u)
    r = u - f * tile
    amb = (r < m) | (tile - r < m)
    return f, amb


def voxel_rects(scene, cam, tile=16):
    """Per voxel: rect int64 [N, 4] = (tx0, tx1, ty0, ty1), empty when
    tx0 > tx1; amb [N] bool (a rounding-sensitive decision).  Voxels whose
    lattice check fails get an empty rect."""
    ntx, nty = tile_grid(cam, tile)
    W, H = cam.width, cam.height
    w2c = np.asarray(cam.w2c, np.float32).astype(np.float64)
    R, t = w2c[:, :3], w2c[:, 3]
    fx, fy, cx, cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    c = np.asarray(scene.centre, np.float32).astype(np.float64)
    lv = np.clip(np.asarray(scene.level, np.int64), 1, 16)
    vs = float(np.float32(scene.world_size)) * np.exp2(-lv.astype(np.float64))
    bits = np.array([[(b >> 2) & 1, (b >> 1) & 1, b & 1] for b in range(8)], np.float64)
    corners = c[:, None, :] + (bits[None] - 0.5) * vs[:, None, None]      # [N, 8, 3]
    X = corners @ R.T + t[None, None]                                      # [N, 8, 3]
    Z = X[..., 2]
    behind = Z <= NEAR
    amb = (np.abs(Z - NEAR) < 1e-5).any(axis=1)
    nb = behind.sum(axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        u = fx * X[..., 0] / Z + cx
        v = fy * X[..., 1] / Z + cy
    u = np.where(behind, np.nan, u)
    v = np.where(behind, np.nan, v)
    n = len(c)
    rect = np.zeros((n, 4), np.int64)
    rect[:, 1] = -1
    rect[:, 3] = -1
    full = (nb > 0) & (nb < 8)
    front = nb == 0
    rect[full] = (0, ntx - 1, 0, nty - 1)
    if front.any():
        uf, vf = u[front], v[front]
        umin, umax = uf.min(1), uf.max(1)
        vmin, vmax = vf.min(1), vf.max(1)
        m_u = PX_MARGIN + REL_MARGIN * np.maximum(np.abs(umin), np.abs(umax))
        m_v = PX_MARGIN + REL_MARGIN * np.maximum(np.abs(vmin), np.abs(vmax))
        cull = (umax < 0) | (umin >= W) | (vmax < 0) | (vmin >= H)
        camb = ((np.abs(umax) < m_u) | (np.abs(umin - W) < m_u)
                | (np.abs(vmax) < m_v) | (np.abs(vmin - H) < m_v))
        fx0, a0 = _floor_amb(umin, tile)
        fx1, a1 = _floor_amb(umax, tile)
        fy0, a2 = _floor_amb(vmin, tile)
        fy1, a3 = _floor_amb(vmax, tile)
        tx0 = np.clip(fx0, 0, ntx - 1)
        tx1 = np.clip(fx1, 0, ntx - 1)
        ty0 = np.clip(fy0, 0, nty - 1)
        ty1 = np.clip(fy1, 0, nty - 1)
        # an ambiguous floor only matters if the clamp does not hide it
        a0 &= (fx0 > 0) & (fx0 <= ntx - 1)
        a1 &= (fx1 >= 0) & (fx1 < ntx - 1)
        a2 &= (fy0 > 0) & (fy0 <= nty - 1)
        a3 &= (fy1 >= 0) & (fy1 < nty - 1)
        r = np.stack([tx0, tx1, ty0, ty1], 1).astype(np.int64)
        r[cull] = (0, -1, 0, -1)
        rect[front] = r
        amb[front] |= camb | (~cull & (a0 | a1 | a2 | a3))
    _, ok = lattice_index(scene)
    rect[~ok] = (0, -1, 0, -1)
    return rect, amb


_SIGN_LIST = [[s for s in range(8) if (m >> s) & 1] for m in range(256)]
_POPC = np.array([len(x) for x in _SIGN_LIST], np.int64)
_SIGN_TAB = np.full((256, 8), -1, np.int64)
for _m, _l in enumerate(_SIGN_LIST):
    _SIGN_TAB[_m, :len(_l)] = _l


def emit_pairs(scene, cam, tile=16, masks=None, rects=None):
    """All (key, value) pairs in emission order, plus the per-voxel counts."""
    ntx, nty = tile_grid(cam, tile)
    if masks is None:
        masks, _ = tile_masks(cam, tile)
    if rects is None:
        rects, _ = voxel_rects(scene, cam, tile)
    code, ok = voxel_octpath(scene)
    n = scene.n_vox
    wx = np.maximum(rects[:, 1] - rects[:, 0] + 1, 0)
    wy = np.maximum(rects[:, 3] - rects[:, 2] + 1, 0)
    area = wx * wy
    vox = np.repeat(np.arange(n), area)
    start = np.repeat(np.cumsum(area) - area, area)
    local = np.arange(len(vox)) - start
    tx = rects[vox, 0] + local % np.maximum(wx[vox], 1)
    ty = rects[vox, 2] + local // np.maximum(wx[vox], 1)
    tid = ty * ntx + tx
    m = masks[tid].astype(np.int64)
    pc = _POPC[m]
    counts = np.bincount(vox, weights=pc, minlength=n).astype(np.int64)
    vox2 = np.repeat(vox, pc)
    tid2 = np.repeat(tid, pc)
    st2 = np.repeat(np.cumsum(pc) - pc, pc)
    j = np.arange(len(vox2)) - st2
    s = _SIGN_TAB[np.repeat(m, pc), j]
    order = morton.dir_dep_order(code[vox2], s)
    keys = (tid2.astype(np.uint64) << np.uint64(48)) | order
    vals = ((s.astype(np.uint64) << np.uint64(29)) | vox2.astype(np.uint64)).astype(np.uint32)
    return keys, vals, counts


def sort_pairs(keys, vals):
    order = np.lexsort((vals, keys))
    return keys[order], vals[order]


def tile_ranges(sorted_keys, ntiles):
    tid = (np.asarray(sorted_keys, np.uint64) >> np.uint64(48)).astype(np.int64)
    beg = np.searchsorted(tid, np.arange(ntiles), side="left")
    end = np.searchsorted(tid, np.arange(ntiles), side="right")
    rng = np.stack([beg, end], 1).astype(np.int64)
    rng[beg == end] = 0
    return rng
