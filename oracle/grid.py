"""Adaptive grid structure of Section 2.2 (oracle; test infrastructure only).

Omega = prod_i [0, shape_i - 1] in Z^d.  Leaves are closed integer boxes that
tile Omega and share facets.  Sample points are the union of the corners of
the cells; since every corner of a refined cell is a corner of one of its
children, the corners of the leaves give the same set.  Points are indexed in
lexicographic order of their coordinates.

* cells(p_k)  = leaves C with p_k in C (closed containment; a hanging node on
  the edge of a coarse leaf therefore belongs to that coarse leaf too),
* U_k         = union of cells(p_k) (the blocky neighbourhood),
* nbrs(k)     = { j : some leaf contains both p_k and p_j }, with k in nbrs(k).
"""
from __future__ import annotations

import itertools
from typing import List

import numpy as np


def box_corners(lo, hi) -> List[tuple]:
    """corners(C) = prod_i {c_min^i, c_max^i} (Section 1.3)."""
    return [tuple(c) for c in itertools.product(*[sorted({int(a), int(b)}) for a, b in zip(lo, hi)])]


def box_midpoint(lo, hi) -> tuple:
    """Approximate midpoint: nearest integer to (c_max + c_min)/2, ties rounded down."""
    return tuple((int(a) + int(b)) // 2 for a, b in zip(lo, hi))


class Grid:
    def __init__(self, shape, cells):
        self.shape = tuple(int(s) for s in shape)
        self.d = len(self.shape)
        self.cells = np.asarray(cells, dtype=np.int64).reshape(-1, 2, self.d)
        self._validate()
        pts = set()
        for lo, hi in self.cells:
            pts.update(box_corners(lo, hi))
        self.points = np.array(sorted(pts), dtype=np.int64).reshape(-1, self.d)
        self.r = len(self.points)
        self.index = {tuple(p): k for k, p in enumerate(self.points)}
        # membership[c, k] = p_k in C (closed)
        lo = self.cells[:, 0, :][:, None, :]
        hi = self.cells[:, 1, :][:, None, :]
        P = self.points[None, :, :]
        self.member = np.all((P >= lo) & (P <= hi), axis=-1)          # [nc, r]
        self.cells_of = [np.nonzero(self.member[:, k])[0] for k in range(self.r)]
        self.points_of = [np.nonzero(self.member[c, :])[0] for c in range(len(self.cells))]
        nb = [set() for _ in range(self.r)]
        for c in range(len(self.cells)):
            ks = self.points_of[c]
            for k in ks:
                nb[k].update(int(j) for j in ks)
        self.nbrs = [np.array(sorted(s), dtype=np.int64) for s in nb]
        self.bbox_lo = np.array([self.cells[self.cells_of[k], 0, :].min(axis=0) for k in range(self.r)])
        self.bbox_hi = np.array([self.cells[self.cells_of[k], 1, :].max(axis=0) for k in range(self.r)])

    def _validate(self):
        """The leaves tile Omega (Section 2.2): boxes of positive extent
        inside it, every unit cube of Omega in exactly one leaf, so that
        leaves meet only on facets."""
        cnt = np.zeros(tuple(int(n) - 1 for n in self.shape), dtype=np.int64)
        for lo, hi in self.cells:
            if np.any(lo < 0) or np.any(hi >= np.array(self.shape)):
                raise ValueError("leaf cell outside the box")
            if np.any(hi <= lo):
                raise ValueError("degenerate leaf cell")
            cnt[tuple(slice(int(a), int(b)) for a, b in zip(lo, hi))] += 1
        if np.any(cnt == 0):
            raise ValueError("leaves do not cover the box")
        if np.any(cnt > 1):
            raise ValueError("leaves overlap")

    def bbox_shape(self, k):
        return tuple(int(h - l + 1) for l, h in zip(self.bbox_lo[k], self.bbox_hi[k]))

    def U_mask(self, k) -> np.ndarray:
        """Indicator of U_k on bbox(U_k)."""
        m = np.zeros(self.bbox_shape(k), dtype=bool)
        for c in self.cells_of[k]:
            lo, hi = self.cells[c]
            sl = tuple(slice(int(a - o), int(b - o) + 1) for a, b, o in zip(lo, hi, self.bbox_lo[k]))
            m[sl] = True
        return m

    def U_mask_full(self, k) -> np.ndarray:
        """Indicator of U_k on Omega."""
        m = np.zeros(self.shape, dtype=bool)
        for c in self.cells_of[k]:
            lo, hi = self.cells[c]
            m[tuple(slice(int(a), int(b) + 1) for a, b in zip(lo, hi))] = True
        return m
