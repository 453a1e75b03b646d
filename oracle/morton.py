"""Morton codes and the direction-dependent Morton order (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

* ``octpath`` / ``voxel_index``: the bit interleaving of Sec. A.1 (listing
  "conversion_octpath_ijk"): level n of the index, finest first, becomes the
  n-th 3-bit triple (x bit most significant), and the code is then shifted
  left by 3 (16 - l), so the coarsest level sits in the top triple.
* ``order_table``: the eight per-triple permutations of Sec. B.2, built here
  from geometry rather than written out: for ray sign pattern s, the eight
  children of a cube are ranked by their centre's projection on a direction
  with the signs of s whose x component dominates y, which dominates z.  That
  is the base case of the ordering proof (Sec. B.3): along +x the -x half
  comes first, inside it the -y half, inside that the -z child.
* ``dir_dep_order``: maps every triple of a code through the table of its
  sign pattern (Sec. B.2), triple by triple, over all 16 triples.
* ``signbits``: 4 (rd.x < 0) + 2 (rd.y < 0) + (rd.z < 0) (Sec. B.2).
"""
from __future__ import annotations

import numpy as np

MAX_LEVEL = 16
_U = np.uint64


def octpath(i, j, k, lv) -> np.ndarray:
    """Morton code of grid index (i, j, k) at level lv (vectorised)."""
    i = np.asarray(i, np.int64).astype(np.uint64)
    j = np.asarray(j, np.int64).astype(np.uint64)
    k = np.asarray(k, np.int64).astype(np.uint64)
    lv = np.asarray(lv, np.int64)
    code = np.zeros(np.broadcast(i, j, k, lv).shape, np.uint64)
    for n in range(MAX_LEVEL):
        bits = _U(4) * (i & _U(1)) + _U(2) * (j & _U(1)) + (k & _U(1))
        code |= np.where(n < lv, bits << _U(3 * n), _U(0))
        i = i >> _U(1)
        j = j >> _U(1)
        k = k >> _U(1)
    return code << (3 * (MAX_LEVEL - lv)).astype(np.uint64)


def voxel_index(code, lv):
    """Inverse of octpath: (i, j, k) of a Morton code at level lv."""
    code = np.asarray(code, np.uint64) >> (3 * (MAX_LEVEL - np.asarray(lv, np.int64))).astype(np.uint64)
    lv = np.asarray(lv, np.int64)
    i = np.zeros(code.shape, np.uint64)
    j = np.zeros(code.shape, np.uint64)
    k = np.zeros(code.shape, np.uint64)
    for n in range(MAX_LEVEL):
        on = n < lv
        i |= np.where(on, ((code >> _U(2)) & _U(1)) << _U(n), _U(0))
        j |= np.where(on, ((code >> _U(1)) & _U(1)) << _U(n), _U(0))
        k |= np.where(on, (code & _U(1)) << _U(n), _U(0))
        code = code >> _U(3)
    return i.astype(np.int64), j.astype(np.int64), k.astype(np.int64)


def signbits(rd) -> np.ndarray:
    rd = np.asarray(rd)
    return (4 * (rd[..., 0] < 0) + 2 * (rd[..., 1] < 0) + (rd[..., 2] < 0)).astype(np.int64)


def order_table() -> np.ndarray:
    """table[s][b]: rank of child b among the 8 children for ray signs s."""
    eps = 1e-3
    table = np.zeros((8, 8), np.int64)
    for s in range(8):
        sx = -1.0 if (s >> 2) & 1 else 1.0
        sy = -1.0 if (s >> 1) & 1 else 1.0
        sz = -1.0 if s & 1 else 1.0
        d = np.array([sx, sy * eps, sz * eps * eps])
        centres = np.array([[(b >> 2) & 1, (b >> 1) & 1, b & 1] for b in range(8)], np.float64) - 0.5
        proj = centres @ d
        order = np.argsort(proj, kind="stable")      # children, near to far
        table[s, order] = np.arange(8)
    return table


_TABLE = order_table()


def dir_dep_order(code, s) -> np.ndarray:
    """Direction-dependent Morton order of a 48-bit code for sign pattern s."""
    code = np.asarray(code, np.uint64)
    s = np.broadcast_to(np.asarray(s, np.int64), code.shape)
    out = np.zeros(code.shape, np.uint64)
    for n in range(MAX_LEVEL):
        tri = ((code >> _U(3 * n)) & _U(7)).astype(np.int64)
        out |= _TABLE[s, tri].astype(np.uint64) << _U(3 * n)
    return out
