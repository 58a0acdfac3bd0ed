"""Particle orders that cut the particles into 32-particle tiles (CRK-HACC
Sec. 2.3: the chaining-mesh order and the recursive-coordinate-bisection
leaves of its short-range trees), as plain numpy definitions.

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product path.
Shares no code with the CUDA library.

  * Morton order: oracle.crk.cells (stable sort by the 30-bit Morton key).
  * Hilbert order: stable sort by the index along the Hilbert curve through
    the 2^10 cells per axis of the top 10 fixed-point bits.  The index is
    computed with Skilling's transposed form of the curve (J. Skilling,
    "Programming the Hilbert curve", AIP Conf. Proc. 707, 2004): the axes
    are rotated and reflected level by level, Gray-decoded, and their bits
    interleaved with x most significant.
  * Bisection order (the paper's leaves, here one tile each): starting from
    the Morton order, every segment of more than 32 particles splits at
    nl = 32 ceil(ceil(size/2) / 32) along the longest axis of its fixed-point
    box (first axis on ties); the particles are binned into 256 equal slices
    of the box along that axis, floor((c - lo) 256 / (extent + 1)); the slice
    holding the nl-th particle is the median slice; a stable partition puts
    the slices below it, then the median slice, then the slices above, so the
    first nl particles are the lower part.
"""
import numpy as np

from . import crk as O

TILE = 32


def hilbert_index(cells, bits=10):
    """Hilbert index of integer cell coordinates (m, 3) in [0, 2^bits)."""
    X = [np.asarray(cells[:, a], np.int64).copy() for a in range(3)]
    M = 1 << (bits - 1)
    Q = M
    while Q > 1:
        P = Q - 1
        for i in range(3):
            hit = (X[i] & Q) != 0
            t = np.where(hit, 0, (X[0] ^ X[i]) & P)
            X[0] = np.where(hit, X[0] ^ P, X[0] ^ t)
            X[i] = np.where(hit, X[i], X[i] ^ t)
        Q >>= 1
    for i in range(1, 3):
        X[i] = X[i] ^ X[i - 1]
    t = np.zeros_like(X[0])
    Q = M
    while Q > 1:
        t = np.where((X[2] & Q) != 0, t ^ (Q - 1), t)
        Q >>= 1
    key = np.zeros_like(X[0])
    for b in range(bits - 1, -1, -1):
        for i in range(3):
            key = (key << 1) | (((X[i] ^ t) >> b) & 1)
    return key


def hilbert_order(pos_h):
    """Sorted slot -> particle of the Hilbert order (stable in the index)."""
    q, _ = O.fixed_point(pos_h)
    key = hilbert_index(q.astype(np.int64) >> 22)
    return np.argsort(key, kind="stable").astype(np.int64)


def split_left(size):
    return ((size + 1) // 2 + TILE - 1) // TILE * TILE


def bisection_order(pos_h, leaf=TILE):
    """Sorted slot -> particle of the bisection order: segments of more than
    `leaf` particles split (leaves of one tile by default; 128 or 256, the
    paper's N_ppl range of Sec. 2.3, whose tiles are cut from the order the
    splits leave inside each leaf)."""
    _, perm, _, _ = O.cells(pos_h)
    perm = perm.astype(np.int64)
    q, _ = O.fixed_point(pos_h)
    q = q.astype(np.uint64)
    segs = [(0, len(perm))]
    while True:
        nxt, split = [], False
        for a, b in segs:
            size = b - a
            if size <= leaf:
                nxt.append((a, b))
                continue
            split = True
            ix = perm[a:b]
            x = q[ix]
            lo, hi = x.min(axis=0), x.max(axis=0)
            ext = hi - lo
            ax = int(np.argmax(ext))
            c = x[:, ax]
            sl = ((c - lo[ax]) * np.uint64(256)) // (ext[ax] + np.uint64(1))
            nl = split_left(size)
            cum = np.cumsum(np.bincount(sl.astype(np.int64), minlength=256))
            m = int(np.searchsorted(cum, nl))
            perm[a:b] = np.concatenate([ix[sl < m], ix[sl == m], ix[sl > m]])
            nxt += [(a, a + nl), (a + nl, b)]
        segs = nxt
        if not split:
            return perm
