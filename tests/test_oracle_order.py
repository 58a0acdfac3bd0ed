"""Pins of the particle orders of oracle/order.py (the Hilbert curve and the
recursive coordinate bisection that cut particles into tiles):

* the Hilbert index is a bijection of the cells, consecutive indices are
  face-adjacent cells (the curve's defining property), and every aligned
  octree cell is one contiguous index range;
* the bisection order is a permutation whose splits, re-derived from it,
  put the lower part of the longest axis first, cut at whole tiles, and
  end in leaves of at most one tile; on a row of particles it reduces to the
  sorted order along that row.
"""
import numpy as np
import pytest

from oracle import crk as O
from oracle import order as R


def _grid(bits):
    g = np.arange(1 << bits)
    c = np.stack(np.meshgrid(g, g, g, indexing="ij"), -1).reshape(-1, 3)
    return c


def test_hilbert_index_is_a_face_adjacent_bijection():
    for bits in (1, 2, 3, 4):
        c = _grid(bits)
        k = R.hilbert_index(c, bits)
        assert np.array_equal(np.sort(k), np.arange(len(c)))
        walk = c[np.argsort(k)]
        step = np.abs(np.diff(walk, axis=0)).sum(axis=1)
        assert np.all(step == 1), bits
        # aligned cubes of side 2^j are contiguous index ranges
        for j in range(1, bits):
            cube = (walk >> j) @ np.array([1 << (2 * (bits - j)), 1 << (bits - j), 1])
            changes = np.count_nonzero(np.diff(cube))
            assert changes == (1 << (3 * (bits - j))) - 1, (bits, j)


def test_hilbert_order_keeps_level_cells_contiguous():
    rng = np.random.default_rng(4)
    pos = np.empty((5000, 4), np.float32)
    pos[:, :3] = O._wrap_f32(rng.random((5000, 3)))
    pos[:, 3] = 0.05
    perm = R.hilbert_order(pos)
    q, _ = O.fixed_point(pos)
    for k in (1, 2, 3, 4):
        cell = (q[perm].astype(np.int64) >> (32 - k)) @ np.array([1 << (2 * k), 1 << k, 1])
        assert np.count_nonzero(np.diff(cell)) == len(np.unique(cell)) - 1, k


def _splits(perm, q, leaf=R.TILE):
    """Re-derive every split of a bisection order and check it."""
    segs = [(0, len(perm))]
    leaves = 0
    while segs:
        a, b = segs.pop()
        size = b - a
        if size <= leaf:
            leaves += 1
            continue
        x = q[perm[a:b]].astype(np.int64)
        ext = x.max(0) - x.min(0)
        ax = int(np.argmax(ext))
        nl = R.split_left(size)
        assert nl % R.TILE == 0 and 0 < nl < size
        sl = ((x[:, ax] - x[:, ax].min()) * 256) // (ext[ax] + 1)
        assert sl[:nl].max() <= sl[nl:].min()         # the lower part goes first
        segs += [(a, a + nl), (a + nl, b)]
    return leaves


def test_bisection_order_splits():
    rng = np.random.default_rng(9)
    c = rng.random((6, 3))
    for n in (1, 33, 100, 3000):
        x = (c[rng.integers(0, 6, n)] + 0.04 * rng.standard_normal((n, 3))) % 1.0
        pos = np.empty((n, 4), np.float32)
        pos[:, :3] = O._wrap_f32(x)
        pos[:, 3] = 0.05
        perm = R.bisection_order(pos)
        assert np.array_equal(np.sort(perm), np.arange(n))
        q, _ = O.fixed_point(pos)
        leaves = _splits(perm, q)
        assert leaves >= (n + R.TILE - 1) // R.TILE


@pytest.mark.parametrize("leaf", [128, 256])
def test_bisection_to_the_papers_leaf_sizes(leaf):
    """Leaves of at most 128 or 256 particles (Sec. 2.3, N_ppl): every split
    re-derived (longest axis, lower part first, whole tiles on the left), and
    the one-tile bisection's order is that of the larger leaves refined
    further: its first splits are the same."""
    rng = np.random.default_rng(19)
    c = rng.random((6, 3))
    n = 3000
    x = (c[rng.integers(0, 6, n)] + 0.04 * rng.standard_normal((n, 3))) % 1.0
    pos = np.empty((n, 4), np.float32)
    pos[:, :3] = O._wrap_f32(x)
    pos[:, 3] = 0.05
    perm = R.bisection_order(pos, leaf=leaf)
    assert np.array_equal(np.sort(perm), np.arange(n))
    q, _ = O.fixed_point(pos)
    leaves = _splits(perm, q, leaf)
    assert (n + leaf - 1) // leaf <= leaves < (n + leaf - 1) // leaf * 2 + 1
    # the same particles in the same leaves as the one-tile bisection groups
    # at that level: each leaf of `leaf` particles is a union of its tiles
    fine = R.bisection_order(pos)
    segs, a = [], 0
    def leaf_segments(a, b):
        if b - a <= leaf:
            return [(a, b)]
        nl = R.split_left(b - a)
        return leaf_segments(a, a + nl) + leaf_segments(a + nl, b)
    for a, b in leaf_segments(0, n):
        assert set(perm[a:b].tolist()) == set(fine[a:b].tolist())


def test_bisection_of_a_row_is_the_sorted_row():
    n = 256
    rng = np.random.default_rng(2)
    x = rng.permutation(n) / n + 0.5 / n
    pos = np.zeros((n, 4), np.float32)
    pos[:, 0] = x
    pos[:, 1] = 0.25
    pos[:, 2] = 0.75
    pos[:, 3] = 0.05
    perm = R.bisection_order(pos)
    # 256 distinct slices of 256 evenly spaced points: every tile holds the
    # next 32 of the sorted row
    tiles = np.sort(x[perm].reshape(-1, 32), axis=1)
    assert np.array_equal(tiles.ravel(), np.sort(x))
