"""Property checks of the library's internal centre layout (test helper).

Inside each cell the library reorders the stably sorted centres so that runs of
32 (source blocks) and 128 (target tiles), counted from the cell start within
runs of at most 4096, are subtrees of recursive median splits.  That layout is
a design choice of the library, not part of the method, so the tests check it
by a property any such split tree has - two subtrees are separated along the
axis of the split that divides them - instead of against a second copy of the
construction."""
import numpy as np


def runs_from(start: int, end: int, length: int):
    """[(s, e)] runs of at most ``length`` positions counted from ``start``."""
    return [(s, min(s + length, end)) for s in range(start, end, length)]


def pairwise_separated(P: np.ndarray, runs) -> bool:
    """True when every two runs of rows of P (m x 3) are separated along some
    axis: max of one <= min of the other in that coordinate."""
    if len(runs) < 2:
        return True
    lo = np.array([P[s:e].min(0) for s, e in runs])
    hi = np.array([P[s:e].max(0) for s, e in runs])
    # sep[a, b, d]: run a lies entirely at or below run b along axis d
    sep = hi[:, None, :] <= lo[None, :, :]
    ok = sep.any(2) | sep.transpose(1, 0, 2).any(2)
    np.fill_diagonal(ok, True)
    return bool(ok.all())


def check_cell_layout(P_sorted: np.ndarray, cell_start, cell_end, chunk=4096, tile=128, leaf=32):
    """Every run of ``chunk`` of every cell: its runs of ``tile`` and of ``leaf``
    are pairwise separated.  Returns the number of chunks checked."""
    checked = 0
    for cs, ce in zip(cell_start, cell_end):
        if ce - cs <= leaf:
            continue
        for c0, c1 in runs_from(int(cs), int(ce), chunk):
            for length in (tile, leaf):
                runs = [(s - c0, e - c0) for s, e in runs_from(c0, c1, length)]
                assert pairwise_separated(P_sorted[c0:c1], runs), (cs, ce, c0, length)
            checked += 1
    return checked
