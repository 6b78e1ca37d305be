"""The layout property check itself (CPU): it accepts split trees and rejects
orders that are not."""
import numpy as np

from layout_props import check_cell_layout, pairwise_separated, runs_from


def test_sorted_line_is_separated_and_shuffled_is_not():
    rng = np.random.default_rng(0)
    x = np.sort(rng.uniform(0, 1, 256))
    P = np.stack([x, rng.uniform(0, 0.01, 256), rng.uniform(0, 0.01, 256)], 1)   # no flat axis
    assert pairwise_separated(P, runs_from(0, 256, 32))
    Q = P[rng.permutation(256)]
    assert not pairwise_separated(Q, runs_from(0, 256, 32))


def test_lattice_quadrants_are_separated():
    """A 16 x 16 lattice ordered as 4 x 8 blocks (a split tree: halves, then
    quarters, ...) passes; swapping two nodes of different blocks fails."""
    i, j = np.meshgrid(np.arange(16), np.arange(16), indexing="ij")
    order = []
    for bi in range(4):           # blocks of 4 rows x 8 columns
        for bj in range(2):
            order += [(r, c) for r in range(4 * bi, 4 * bi + 4) for c in range(8 * bj, 8 * bj + 8)]
    rng = np.random.default_rng(1)
    P = np.array([[r, c, rng.uniform(0, 0.1)] for r, c in order])    # z varies: no flat axis
    assert pairwise_separated(P, runs_from(0, 256, 32))
    assert pairwise_separated(P, runs_from(0, 256, 128))
    # interleaving two blocks breaks the property
    Q = P.copy()
    Q[[5, 40]] = Q[[40, 5]]
    assert not pairwise_separated(Q, runs_from(0, 256, 32))


def test_check_cell_layout_walks_cells_and_chunks():
    x = np.arange(300, dtype=float)
    P = np.stack([x, x, x], 1)
    assert check_cell_layout(P, [0, 100], [100, 300], chunk=64, tile=16, leaf=8) == 2 + 4
