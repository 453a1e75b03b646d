"""Input generators: the level balancing of the large workload's octree."""
import numpy as np

from synth import scenes as S


def _max_touching_level_gap(cells):
    lo = cells.centre - cells.size[:, None] / 2
    hi = cells.centre + cells.size[:, None] / 2
    gap = 0
    for i in range(len(cells)):
        touch = ((lo[i] <= hi + 1e-12) & (hi[i] >= lo - 1e-12)).all(axis=1)
        touch[i] = False
        if touch.any():
            gap = max(gap, int(np.abs(cells.level[touch] - cells.level[i]).max()))
    return gap


def test_balance_levels_bounds_touching_levels():
    """Brute force over all pairs of leaves of a random octree with large
    level jumps: after balancing, leaves that touch (face, edge or corner)
    differ by at most max_diff levels, and the leaves still tile the cube."""
    cells = S.random_octree_cells(5, 7, 0.35)
    assert _max_touching_level_gap(cells) > 2
    for max_diff in (2, 3):
        b = S.balance_levels(cells, max_diff)
        assert _max_touching_level_gap(b) <= max_diff
        assert np.isclose((b.size ** 3).sum(), 1.0)
        assert len(np.unique(S._cell_key(b.level, b.ijk))) == len(b)
