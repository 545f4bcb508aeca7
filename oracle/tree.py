"""Quad/oct trees with Z-order over a point set (oracle).

Sec. 3.1: the domain cube is split recursively into 2^d children; the nodes of
level l are ordered along a Z-order (Morton) curve, node i at level l has the
children 2^d i + t, t = 0..2^d-1 (Fig. 6).  Reading of Fig. 6 adopted here:
the child digit is t = 2 bit(x1) + bit(x2) in 2D (x1 the more significant
axis), t = 4 bit(x1) + 2 bit(x2) + bit(x3) in 3D.  Sec. 3.6: empty nodes are
discarded, so a level lists only the nodes holding points, and point counts
per node may differ.  Points inside a node keep ascending input order.

Parity: pinned in tests by the 16-node layout of Fig. 6 and by counting
(every point in exactly one node per level; children partition parents).
"""
from __future__ import annotations

import numpy as np


def interleave(cells: np.ndarray, bits: int) -> np.ndarray:
    """Morton code of integer cell coordinates (npts, d), axis 0 most significant."""
    npts, d = cells.shape
    code = np.zeros(npts, dtype=np.int64)
    for bit in range(bits - 1, -1, -1):
        for k in range(d):
            code = (code << 1) | ((cells[:, k] >> bit) & 1)
    return code


class Tree:
    """Levels 0..L of a 2^d-ary tree; nodes[l] maps Z-index -> point indices."""

    def __init__(self, pts: np.ndarray, L: int, box=None):
        pts = np.asarray(pts, dtype=np.float64)
        self.d = pts.shape[1]
        self.b = 2 ** self.d
        self.L = L
        if box is None:
            lo = pts.min(axis=0)
            side = float((pts.max(axis=0) - lo).max())
            side = side if side > 0 else 1.0
        else:
            lo, side = np.asarray(box[0], dtype=np.float64), float(box[1])
        self.lo, self.side = lo, side
        cells = np.floor((pts - lo) / side * (2 ** L)).astype(np.int64)
        cells = np.clip(cells, 0, 2 ** L - 1)
        zL = interleave(cells, L) if L > 0 else np.zeros(pts.shape[0], dtype=np.int64)
        self.nodes = []
        for lev in range(L + 1):
            z = zL >> (self.d * (L - lev))
            order = np.lexsort((np.arange(z.size), z))
            zs = z[order]
            uniq, start = np.unique(zs, return_index=True)
            stops = list(start[1:]) + [zs.size]
            self.nodes.append({int(u): order[a:b] for u, a, b in zip(uniq, start, stops)})

    def level(self, lev: int):
        """Z-indices present at level lev, ascending."""
        return sorted(self.nodes[lev].keys())

    def points(self, lev: int, z: int) -> np.ndarray:
        return self.nodes[lev][z]

    def children(self, lev: int, z: int):
        """Non-empty children (at level lev+1) of node z at level lev, in Z-order."""
        nxt = self.nodes[lev + 1]
        return [self.b * z + t for t in range(self.b) if self.b * z + t in nxt]

    def ancestor(self, lev: int, z: int, up_lev: int) -> int:
        """Z-index at level up_lev of the ancestor of node z at level lev."""
        return z >> (self.d * (lev - up_lev))

    def descendants(self, lev: int, z: int, down_lev: int):
        """Non-empty descendants of (lev, z) at level down_lev, in Z-order."""
        shift = self.d * (down_lev - lev)
        lo, hi = z << shift, (z + 1) << shift
        return [u for u in self.level(down_lev) if lo <= u < hi]
