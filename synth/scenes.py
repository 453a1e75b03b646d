"""Seeded synthetic sparse-voxel scenes.

A scene is a set of octree leaf voxels stored in arbitrary order, each with
its level, its world-space centre, the indices of its 8 corner grid points and
48 spherical-harmonic coefficients ([16][3], coefficient-major, RGB inner).
Grid points are shared by voxels of the same level that touch at a corner; a
grid point is identified by (level, integer corner coordinates).  Corner j of
a voxel has x, y, z offsets (j >> 2 & 1, j >> 1 & 1, j & 1), the order of
V_000 ... V_111 in the trilinear interpolation of the paper (Sec. A.2).

Voxels are made by splitting cubes: the root cube (centre c, size s) has eight
children with centres c + (b - 1/2) s / 2 and size s / 2, for b in {0, 1}^3,
and child grid index 2 * ijk + b.  The random numbers come from numpy's
default_rng(seed) or from a counter-based splitmix64 hash of (seed, tag,
integers), so a scene depends only on its arguments.

This module only builds inputs.  It holds none of the rasterizer's arithmetic.
"""
from __future__ import annotations

import concurrent.futures
import dataclasses
import hashlib
import os

import numpy as np

# ---------------------------------------------------------------------------
# counter-based hash (splitmix64), used for per-cell and per-lattice-point draws
# ---------------------------------------------------------------------------

_U64 = np.uint64


def _mix(x: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        x = (x + _U64(0x9E3779B97F4A7C15)).astype(np.uint64)
        z = x
        z = (z ^ (z >> _U64(30))) * _U64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> _U64(27))) * _U64(0x94D049BB133111EB)
        return z ^ (z >> _U64(31))


def hash_uniform(seed: int, tag: int, *ints: np.ndarray) -> np.ndarray:
    """Uniform [0, 1) numbers, one per element of the broadcast integer arrays."""
    h = _mix(np.full(np.broadcast(*ints).shape if ints else (), seed, dtype=np.uint64))
    h = _mix(h ^ _U64(tag))
    for a in ints:
        h = _mix(h ^ np.asarray(a).astype(np.int64).astype(np.uint64))
    return (h >> _U64(11)).astype(np.float64) * (1.0 / (1 << 53))


# ---------------------------------------------------------------------------
# octree cells
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Cells:
    ijk: np.ndarray     # int64 [n, 3]
    level: np.ndarray   # int64 [n]
    centre: np.ndarray  # float64 [n, 3]
    size: np.ndarray    # float64 [n]

    def __len__(self) -> int:
        return len(self.level)

    def take(self, m) -> "Cells":
        return Cells(self.ijk[m], self.level[m], self.centre[m], self.size[m])

    @staticmethod
    def cat(parts) -> "Cells":
        parts = list(parts)
        if not parts:
            return Cells(np.zeros((0, 3), np.int64), np.zeros(0, np.int64),
                         np.zeros((0, 3)), np.zeros(0))
        return Cells(np.concatenate([p.ijk for p in parts]),
                     np.concatenate([p.level for p in parts]),
                     np.concatenate([p.centre for p in parts]),
                     np.concatenate([p.size for p in parts]))


_BITS = np.array([[(b >> 2) & 1, (b >> 1) & 1, b & 1] for b in range(8)], np.int64)


def root(center, size) -> Cells:
    return Cells(np.zeros((1, 3), np.int64), np.zeros(1, np.int64),
                 np.asarray(center, np.float64)[None], np.array([float(size)]))


def split(c: Cells) -> Cells:
    """The eight children of every cell, child b of cell i at row 8 i + b."""
    n = len(c)
    ijk = (2 * c.ijk[:, None, :] + _BITS[None]).reshape(n * 8, 3)
    half = c.size[:, None, None] * 0.5
    centre = (c.centre[:, None, :] + (_BITS[None] - 0.5) * half).reshape(n * 8, 3)
    level = np.repeat(c.level + 1, 8)
    size = np.repeat(c.size * 0.5, 8)
    return Cells(ijk, level, centre, size)


def dense_cells(level: int, center=(0.5, 0.5, 0.5), size=1.0) -> Cells:
    c = root(center, size)
    for _ in range(level):
        c = split(c)
    return c


# ---------------------------------------------------------------------------
# scene container
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class Scene:
    world_center: np.ndarray  # float32 [3]
    world_size: np.float32
    centre: np.ndarray        # float32 [N, 3]
    level: np.ndarray         # uint8 [N]
    corner_idx: np.ndarray    # int32 [N, 8]
    grid: np.ndarray          # float32 [Pts]
    sh: np.ndarray            # float32 [N, 48]
    ijk: np.ndarray           # int32 [N, 3], generator bookkeeping
    grid_pos: np.ndarray      # float64 [Pts, 3], world position of each grid point

    @property
    def n_vox(self) -> int:
        return int(self.level.shape[0])

    @property
    def n_pts(self) -> int:
        return int(self.grid.shape[0])

    @property
    def max_level(self) -> int:
        return int(self.level.max()) if self.n_vox else 0


_N26 = np.array([(a, b, c) for a in (-1, 0, 1) for b in (-1, 0, 1) for c in (-1, 0, 1)
                 if (a, b, c) != (0, 0, 0)], np.int64)


def _unique(x: np.ndarray) -> np.ndarray:
    """Sorted distinct values of a 1-D integer array (np.unique's result; a
    plain sort and a neighbour comparison, much faster on large arrays)."""
    s = np.sort(np.asarray(x).ravel())
    if len(s) == 0:
        return s
    keep = np.empty(len(s), bool)
    keep[0] = True
    np.not_equal(s[1:], s[:-1], out=keep[1:])
    return s[keep]


def _isin_sorted(x: np.ndarray, table: np.ndarray) -> np.ndarray:
    """x's elements that occur in `table` (sorted, distinct): np.isin's result."""
    if len(table) == 0:
        return np.zeros(np.shape(x), bool)
    i = np.minimum(np.searchsorted(table, x), len(table) - 1)
    return table[i] == x


def _unique_first_inverse(x: np.ndarray):
    """np.unique(x, return_index=True, return_inverse=True) of a 1-D integer
    array: distinct values, the index of each one's first occurrence, and the
    position of every element's value among them."""
    order = np.argsort(x)
    s = x[order]
    new = np.empty(len(s), bool)
    if not len(s):
        return s, order, order
    new[0] = True
    np.not_equal(s[1:], s[:-1], out=new[1:])
    inv = np.empty(len(s), np.int64)
    inv[order] = np.cumsum(new) - 1
    starts = np.flatnonzero(new)
    return s[starts], np.minimum.reduceat(order, starts), inv


def _cell_key(level, ijk: np.ndarray) -> np.ndarray:
    level = np.broadcast_to(np.asarray(level, np.int64), ijk.shape[:1])
    return (level << 51) | (ijk[:, 0] << 34) | (ijk[:, 1] << 17) | ijk[:, 2]


def balance_levels(cells: Cells, max_diff: int) -> Cells:
    """Split leaves until no two leaves that touch (share a face, edge or
    corner) differ by more than max_diff levels.

    A leaf B at level l touches a leaf coarser than l - max_diff exactly when
    one of the 26 neighbours of B's level-(l - max_diff) ancestor is not a node
    of the tree (it lies inside a coarser leaf); that coarser leaf is split,
    and the check repeats until nothing changes.
    """
    if len(cells) == 0:
        return cells
    mask = np.int64((1 << 17) - 1)

    def ijk_of(keys):
        return np.stack([(keys >> 34) & mask, (keys >> 17) & mask, keys & mask], axis=1)

    while True:
        lmin, lmax = int(cells.level.min()), int(cells.level.max())
        by_level = {l: cells.ijk[cells.level == l] for l in range(lmin, lmax + 1)}
        leaf_keys = {l: _unique(_cell_key(l, v)) for l, v in by_level.items()}
        # nodes (leaves and their ancestors) of each level
        nodes = {}
        for m in range(lmin, lmax + 1):
            parts = [_cell_key(m, by_level[l] >> (l - m)) for l in range(m, lmax + 1) if len(by_level[l])]
            nodes[m] = _unique(np.concatenate(parts)) if parts else np.zeros(0, np.int64)
        split_keys = []
        for l in range(lmin + max_diff + 1, lmax + 1):
            if not len(by_level[l]):
                continue
            m = l - max_diff
            anc = ijk_of(_unique(_cell_key(m, by_level[l] >> max_diff)))
            nb = (anc[:, None, :] + _N26[None]).reshape(-1, 3)
            nb = nb[((nb >= 0) & (nb < (1 << m))).all(axis=1)]
            kb = _unique(_cell_key(m, nb))
            missing = ijk_of(kb[~_isin_sorted(kb, nodes[m])])
            for m2 in range(m - 1, lmin - 1, -1):
                if not len(missing):
                    break
                up = missing >> (m - m2)
                hit = _isin_sorted(_cell_key(m2, up), leaf_keys[m2])
                if hit.any():
                    split_keys.append(_unique(_cell_key(m2, up[hit])))
                missing = missing[~hit]
        if not split_keys:
            return cells
        go = _isin_sorted(_cell_key(cells.level, cells.ijk), _unique(np.concatenate(split_keys)))
        cells = Cells.cat([cells.take(~go), split(cells.take(go))])


def corner_points(cells: Cells):
    """Shared grid points of a leaf set: (corner_idx [N, 8], positions [Pts, 3])."""
    n = len(cells)
    if n == 0:
        return np.zeros((0, 8), np.int32), np.zeros((0, 3))
    cijk = cells.ijk[:, None, :] + _BITS[None]                     # [n, 8, 3]
    key = ((cells.level[:, None] << 51) | (cijk[..., 0] << 34)
           | (cijk[..., 1] << 17) | cijk[..., 2])
    uniq, first, inv = _unique_first_inverse(key.reshape(-1))
    pos = (cells.centre[:, None, :] + (_BITS[None] - 0.5) * cells.size[:, None, None])
    pos = pos.reshape(-1, 3)[first]
    return inv.reshape(n, 8).astype(np.int32), pos


def make_scene(cells: Cells, grid_fn, sh_std: float, rng: np.random.Generator,
               center=(0.5, 0.5, 0.5), size=1.0, shuffle=True) -> Scene:
    """Assemble a Scene from leaf cells.

    grid_fn(positions [Pts, 3], rng) -> raw densities [Pts].  The voxel order
    is shuffled (the representation stores voxels in arbitrary order).
    """
    if shuffle and len(cells):
        cells = cells.take(rng.permutation(len(cells)))
    corner_idx, pos = corner_points(cells)
    grid = np.asarray(grid_fn(pos, rng), np.float32)
    sh = (rng.normal(size=(len(cells), 48)) * sh_std).astype(np.float32)
    return Scene(np.asarray(center, np.float32), np.float32(size),
                 cells.centre.astype(np.float32), cells.level.astype(np.uint8),
                 corner_idx, grid, sh, cells.ijk.astype(np.int32), pos)


def normal_grid(mean: float, std: float):
    return lambda pos, rng: rng.normal(mean, std, size=len(pos))


def constant_grid(value: float):
    return lambda pos, rng: np.full(len(pos), value)


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------

def dense_scene(level: int = 5, seed: int = 0, grid_fn=None, sh_std: float = 0.3,
                center=(0.5, 0.5, 0.5), size=1.0, shuffle=True) -> Scene:
    """Every voxel of one octree level (the dense level-5 workload: 32^3 voxels,
    33^3 grid points with raw densities ~ N(0, 1), SH ~ N(0, 0.3))."""
    rng = np.random.default_rng(seed)
    cells = dense_cells(level, center, size)
    return make_scene(cells, grid_fn or normal_grid(0.0, 1.0), sh_std, rng,
                      center, size, shuffle)


def random_octree_cells(seed: int, max_level: int, p_split: float = 0.5,
                        p_keep: float = 1.0, max_cells: int | None = None,
                        center=(0.5, 0.5, 0.5), size=1.0) -> Cells:
    """A random non-overlapping leaf set: split from the root (every level-1
    cell exists), each cell split again with probability p_split up to
    max_level, then each leaf kept with probability p_keep."""
    rng = np.random.default_rng(seed)
    active = split(root(center, size))
    leaves = []
    while len(active):
        can = active.level < max_level
        go = can & (rng.random(len(active)) < p_split)
        leaves.append(active.take(~go))
        active = split(active.take(go)) if go.any() else active.take(go)
    cells = Cells.cat(leaves)
    keep = rng.random(len(cells)) < p_keep
    cells = cells.take(keep)
    if max_cells is not None and len(cells) > max_cells:
        cells = cells.take(np.sort(rng.choice(len(cells), max_cells, replace=False)))
    return cells


def random_octree_scene(seed: int, max_level: int = 3, p_split: float = 0.5,
                        p_keep: float = 1.0, max_cells: int | None = None,
                        grid_fn=None, sh_std: float = 0.3,
                        center=(0.5, 0.5, 0.5), size=1.0) -> Scene:
    cells = random_octree_cells(seed, max_level, p_split, p_keep, max_cells, center, size)
    rng = np.random.default_rng(seed + 1000003)
    return make_scene(cells, grid_fn or normal_grid(0.0, 1.0), sh_std, rng, center, size)


# --- noisy sphere shell ----------------------------------------------------

def value_noise(p: np.ndarray, freq: float, seed: int, octave: int) -> np.ndarray:
    """Lattice value noise in [-1, 1]: hashed lattice values, smoothstep
    trilinear interpolation, `freq` lattice cells per unit length.  The
    lattice values over the points' bounding box are hashed once into a table
    and gathered (the same values as hashing per point)."""
    g = p * freq
    i0 = np.floor(g).astype(np.int64)
    f = g - i0
    s = f * f * (3.0 - 2.0 * f)
    if len(p) == 0:
        return np.zeros(0)
    lo = i0.min(axis=0)
    ext = i0.max(axis=0) - lo + 2
    ax = [np.arange(lo[a], lo[a] + ext[a]) for a in range(3)]
    li, lj, lk = np.meshgrid(ax[0], ax[1], ax[2], indexing="ij")
    table = (2.0 * hash_uniform(seed, 7919 + octave, li.ravel(), lj.ravel(), lk.ravel()) - 1.0)
    rel = i0 - lo
    base = (rel[:, 0] * ext[1] + rel[:, 1]) * ext[2] + rel[:, 2]
    out = np.zeros(len(p))
    for b in range(8):
        o = _BITS[b]
        w = np.prod(np.where(o[None] == 1, s, 1.0 - s), axis=1)
        out += w * table[base + (o[0] * ext[1] + o[1]) * ext[2] + o[2]]
    return out


def shell_radius(p: np.ndarray, seed: int, radius: float, amp: float,
                 octaves=((4.0, 1.0), (8.0, 0.5), (16.0, 0.25))) -> np.ndarray:
    """radius + n(p): three octaves of value noise, weights normalised so the
    largest possible deviation is `amp`."""
    tot = sum(a for _, a in octaves)
    n = sum(a * value_noise(p, f, seed, o) for o, (f, a) in enumerate(octaves))
    return radius + amp * n / tot


_CHUNK = 1 << 18


def shell_distance(p: np.ndarray, seed: int, centers, radii, amp: float) -> np.ndarray:
    """Distance-like measure | |p - c| - r(p) | to the nearest of several shells.

    Large point sets are cut into chunks evaluated on a thread pool (NumPy
    releases the GIL in its loops); every point's value depends only on the
    point, so the result is the same."""
    if len(p) <= _CHUNK:
        return _shell_distance(p, seed, centers, radii, amp)
    chunks = [p[i:i + _CHUNK] for i in range(0, len(p), _CHUNK)]
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(len(chunks), os.cpu_count() or 1)) as ex:
        return np.concatenate(list(ex.map(lambda c: _shell_distance(c, seed, centers, radii, amp), chunks)))


def _shell_distance(p: np.ndarray, seed: int, centers, radii, amp: float) -> np.ndarray:
    d = np.full(len(p), np.inf)
    for s, (c, r) in enumerate(zip(centers, radii)):
        rr = shell_radius(p, seed * 31 + s, r, amp)
        d = np.minimum(d, np.abs(np.linalg.norm(p - np.asarray(c)[None], axis=1) - rr))
    return d


def _shell_cells(seed, p_split, base_level, max_level, centers, radii, band, amp,
                 count_only=False):
    """Band-limited random subdivision.

    Start from the dense base_level grid; a cell of level < max_level whose
    centre lies within band + half its diagonal of a shell is split with
    probability p_split (a hash of (seed, level, ijk), so the leaf count grows
    monotonically with p_split).
    """
    active = dense_cells(base_level)
    leaves = []
    n_leaves = 0
    while len(active):
        lvl = int(active.level[0])
        if lvl >= max_level:
            go = np.zeros(len(active), bool)
        else:
            d = shell_distance(active.centre, seed, centers, radii, amp)
            near = d <= band + active.size * (np.sqrt(3.0) * 0.5)
            u = hash_uniform(seed, 104729 + lvl, active.ijk[:, 0], active.ijk[:, 1],
                             active.ijk[:, 2])
            go = near & (u < p_split)
        if count_only:
            n_leaves += int((~go).sum())
        else:
            leaves.append(active.take(~go))
        active = split(active.take(go)) if go.any() else active.take(go)
    return n_leaves if count_only else Cells.cat(leaves)


# Split probabilities found by calibrate_shell(): the ~1M-voxel single-shell
# workload (1,051,072 leaves at seed 0) and the ~8M-voxel three-shell one
# (8,035,861 leaves at seed 0).
_SHELL_P = {}
KNOWN_SPLIT_P = {("one", 0, 1 << 20): 0.58203125, ("three", 0, 8_000_000): 0.505859375}


def calibrate_shell(target: int, seed: int = 0, **kw) -> float:
    """Bisect the split probability so the leaf count is within 1% of target."""
    lo, hi = 0.0, 1.0
    for _ in range(30):
        mid = 0.5 * (lo + hi)
        n = _shell_cells(seed, mid, count_only=True, **kw)
        if abs(n - target) <= 0.01 * target:
            return mid
        if n < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


SHELL_ONE = dict(base_level=4, max_level=9, centers=((0.5, 0.5, 0.5),), radii=(0.4,),
                 band=0.02, amp=0.05)
SHELL_THREE = dict(base_level=4, max_level=11,
                   centers=((0.47, 0.5, 0.52), (0.53, 0.48, 0.5), (0.5, 0.52, 0.47)),
                   radii=(0.25, 0.33, 0.41), band=0.01, amp=0.05, max_level_diff=4)


def shell_scene(seed: int = 0, target: int = 1 << 20, p_split: float | None = None,
                spec: dict | None = None, sh_std: float = 0.3,
                near_mean: float = 2.0, near_std: float = 1.0, far_value: float = -4.0) -> Scene:
    """Adaptive octree around noisy sphere shells (the ~1M-voxel workload).

    Leaves of a level-4 background grid, split toward the shells up to
    spec['max_level'].  Grid points within spec['band'] of a shell get raw
    densities ~ N(near_mean, near_std), all others far_value.
    """
    name = "one" if spec is None or spec == SHELL_ONE else "three" if spec == SHELL_THREE else None
    if p_split is None and (name, seed, target) in KNOWN_SPLIT_P:
        p_split = KNOWN_SPLIT_P[(name, seed, target)]
    cache = _cache_path("shell", seed, target, p_split, spec, sh_std, near_mean, near_std, far_value)
    if cache and os.path.exists(cache):
        return _load(cache)
    scene = _shell_scene(seed, target, p_split, spec, sh_std, near_mean, near_std, far_value)
    if cache:
        _save(cache, scene)
    return scene


def _cache_path(*key):
    """File under $SVR_SCENE_CACHE for a generated scene (None if unset)."""
    d = os.environ.get("SVR_SCENE_CACHE")
    if not d:
        return None
    os.makedirs(d, exist_ok=True)
    h = hashlib.sha1(repr(key).encode()).hexdigest()[:16]
    return os.path.join(d, f"scene_{h}.npz")


def _save(path, scene):
    tmp = path + f".{os.getpid()}.tmp.npz"
    np.savez(tmp, **{k: np.asarray(v) for k, v in dataclasses.asdict(scene).items()})
    os.replace(tmp, path)


def _load(path):
    z = np.load(path)
    kw = {k: z[k] for k in z.files}
    kw["world_size"] = np.float32(kw["world_size"])
    return Scene(**kw)


def _shell_scene(seed, target, p_split, spec, sh_std, near_mean, near_std, far_value):
    spec = dict(SHELL_ONE if spec is None else spec)
    max_diff = spec.pop("max_level_diff", None)
    if p_split is None:
        key = (seed, target, tuple(sorted((k, str(v)) for k, v in spec.items())))
        if key not in _SHELL_P:
            _SHELL_P[key] = calibrate_shell(target, seed, **spec)
        p_split = _SHELL_P[key]
    cells = _shell_cells(seed, p_split, **spec)
    if max_diff is not None:
        cells = balance_levels(cells, max_diff)
    rng = np.random.default_rng(seed)

    def grid_fn(pos, rng):
        d = shell_distance(pos, seed, spec["centers"], spec["radii"], spec["amp"])
        near = d <= spec["band"]
        out = np.full(len(pos), far_value)
        out[near] = rng.normal(near_mean, near_std, size=int(near.sum()))
        return out

    return make_scene(cells, grid_fn, sh_std, rng)


# ---------------------------------------------------------------------------
# helpers for tests
# ---------------------------------------------------------------------------

def subscene(scene: Scene, idx: np.ndarray) -> Scene:
    """The voxels `idx` of a scene, with their grid points renumbered."""
    idx = np.asarray(idx)
    ci = scene.corner_idx[idx]
    used, inv = np.unique(ci.reshape(-1), return_inverse=True)
    return Scene(scene.world_center, scene.world_size, scene.centre[idx], scene.level[idx],
                 inv.reshape(-1, 8).astype(np.int32), scene.grid[used], scene.sh[idx],
                 scene.ijk[idx], scene.grid_pos[used])


def upstream_grads(seed: int, height: int, width: int):
    """Seeded upstream gradients (dL/drgb [3, H, W], dL/ddepth, dL/dalpha)."""
    rng = np.random.default_rng(seed)
    g_rgb = rng.normal(size=(3, height, width)).astype(np.float32)
    g_depth = rng.normal(size=(height, width)).astype(np.float32)
    g_alpha = rng.normal(size=(height, width)).astype(np.float32)
    return g_rgb, g_depth, g_alpha
