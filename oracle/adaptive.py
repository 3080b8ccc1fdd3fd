"""Adaptive construction of A~ (Algorithm 1), oracle side (test
infrastructure only).  Built from the oracle's grid, weights, extension,
adjoint apply and estimator, in the algorithm's order:

1. Z (q probes) and Y = A* Z are given (the caller's random matrix and its
   q applications of A*).
2. The tree starts as Omega subdivided once in each coordinate direction.
3. Each pass builds U_k, w_k, phi_k = A delta_{p_k} (the caller's impulse
   callback, cached per point), phi_k^E, Y~ = A~* Z and the local
   estimators eta_C (Eq. randomized_estimator_ec).
4. Overall estimator: eta_Omega = sqrt(sum_C eta_C^2) / (||Y||_F / sqrt(q))
   (relative; a point on a shared facet counts in each cell holding it).
5. While eta_Omega > tau: the cell with the largest eta_C is subdivided in
   the direction i (Section 2.7) in which the averaged extended impulse
   responses of its front and back corners differ most,
       phi^{i+-} = 2^{1-d} sum {phi_k^E : p_k corner of C, p_k^i = c_max^i / c_min^i},
       || phi^{i+} - phi^{i-} ||_{l2(Omega - c_mid)},
   among directions with c_max^i - c_min^i > 2, at floor((c_min + c_max)/2).
   Values within a relative 1e-9 of the largest count as a tie, won by the
   lowest direction index.

   In 3D a split can break the two sides of a facet crosswise (one side
   split along one axis, the other side along another); the pieces of that
   facet then have corners that are no cell's corner, where the recursive
   construction of Section 2.4 has no value.  Such a split is skipped: the
   cell takes the next direction in the order above whose split leaves every
   facet piece with sample points at its corners, and a cell with none is
   passed over for the next cell by eta_C.  (In 2D a facet is a segment and
   its pieces end at sample points, so every split qualifies.)

`batch` > 1 refines up to that many cells per pass (largest eta_C first),
all chosen from one pass's estimates; batch = 1 is Algorithm 1 as printed.
"""
from __future__ import annotations

from itertools import product
from typing import Callable, List

import numpy as np

from .apply import PCOracle
from .estimator import eta_from_adjoints
from .grid import Grid, box_midpoint
from .weights import facet_pieces


def split_directions(grid: Grid, phiE: np.ndarray, R: int, c: int) -> List[int]:
    """Section 2.7: the directions in which leaf cell c may be subdivided
    (extent > 2), best first: each is the one of largest
    || phi^{i+} - phi^{i-} || among those not yet listed, values within a
    relative 1e-9 of it counting as a tie won by the lowest index."""
    lo, hi = grid.cells[c]
    d = grid.d
    W = 2 * R + 1
    index = {tuple(p): k for k, p in enumerate(grid.points)}
    mid = np.array(box_midpoint(lo, hi))
    # window offsets z with c_mid + z in Omega
    zs = np.array(list(product(range(-R, R + 1), repeat=d)))
    inside = np.all((mid + zs >= 0) & (mid + zs < np.array(grid.shape)), axis=1)
    vals = []
    for i in range(d):
        if hi[i] - lo[i] <= 2:
            vals.append(None)
            continue
        plus, minus = np.zeros(W ** d), np.zeros(W ** d)
        for corner in product(*[(lo[a], hi[a]) for a in range(d)]):
            k = index[tuple(int(v) for v in corner)]
            if corner[i] == hi[i]:
                plus += phiE[k]
            else:
                minus += phiE[k]
        diff = (plus - minus) / 2 ** (d - 1)
        vals.append(float(np.sqrt(np.sum(diff[inside] ** 2))))
    left = [i for i, v in enumerate(vals) if v is not None]
    order = []
    while left:
        top = max(vals[i] for i in left)
        best = min(i for i in left if vals[i] >= top - 1e-9 * top)
        order.append(best)
        left.remove(best)
    return order


def split_direction(grid: Grid, phiE: np.ndarray, R: int, c: int) -> int:
    """The best subdivision direction of leaf cell c, or -1 if no direction
    is big enough to refine."""
    order = split_directions(grid, phiE, R, c)
    return order[0] if order else -1


def pieces_have_sample_corners(shape, cells) -> bool:
    """Whether every facet piece of every leaf (Section 2.4: a facet, or its
    intersections with the facets of the leaves across it) has sample points
    at all its corners."""
    grid = Grid(shape, cells)
    points = {tuple(int(v) for v in p) for p in grid.points}
    for c in range(len(grid.cells)):
        for a in range(grid.d):
            for side in (0, 1):
                for plo, phi in facet_pieces(grid, c, a, side):
                    for corner in product(*[(int(plo[b]), int(phi[b])) for b in range(grid.d)]):
                        if corner not in points:
                            return False
    return True


def subdivide(cells: np.ndarray, c: int, i: int) -> np.ndarray:
    lo, hi = cells[c]
    m = (int(lo[i]) + int(hi[i])) // 2
    a_hi = hi.copy()
    a_hi[i] = m
    b_lo = lo.copy()
    b_lo[i] = m
    out = [cells[j] for j in range(len(cells)) if j != c]
    out += [np.array([lo, a_hi]), np.array([b_lo, hi])]
    return np.array(out)


def initial_cells(shape) -> np.ndarray:
    d = len(shape)
    cells = []
    for half in product((0, 1), repeat=d):
        lo, hi = [], []
        for a in range(d):
            m = (shape[a] - 1) // 2
            lo.append(0 if half[a] == 0 else m)
            hi.append(m if half[a] == 0 else shape[a] - 1)
        cells.append([lo, hi])
    return np.array(cells, dtype=np.int64)


def construct(shape, impulse: Callable[[np.ndarray], np.ndarray], R: int, Z: np.ndarray, Y: np.ndarray,
              tau: float, max_passes: int = 100, batch: int = 1, stats: dict = None):
    """Returns (cells, history) with history = [(r, eta_Omega)] per pass.  If
    `stats` is a dict it counts "skipped_splits" (a direction whose split
    would break a facet crosswise) and "fallbacks" (cells split in a later
    direction than their first)."""
    Z = np.asarray(Z, dtype=np.float64).reshape(len(Z), -1)
    Y = np.asarray(Y, dtype=np.float64).reshape(len(Y), -1)
    q = Z.shape[0]
    ynorm = np.linalg.norm(Y) / np.sqrt(q)
    cells = initial_cells(shape)
    cache = {}
    history: List[tuple] = []
    for _ in range(max_passes):
        grid = Grid(shape, cells)
        new = [tuple(int(v) for v in p) for p in grid.points if tuple(int(v) for v in p) not in cache]
        if new:
            phis = impulse(np.array(new))
            for p, ph in zip(new, phis):
                cache[p] = np.asarray(ph, dtype=np.float64).ravel()
        phi = np.array([cache[tuple(int(v) for v in p)] for p in grid.points])
        orc = PCOracle(shape, cells, phi, R)
        eta_c = eta_from_adjoints(grid, orc.apply_adjoint(Z), Y)
        eta_o = float(np.sqrt(np.sum(eta_c ** 2)) / ynorm)
        history.append((grid.r, eta_o))
        if eta_o <= tau:
            break
        order = sorted(range(len(cells)), key=lambda c: (-eta_c[c], c))
        chosen = []
        trial = cells          # the cells as split so far this pass
        for c in order:
            for i in split_directions(grid, orc.phiE, R, c):
                at = next(j for j, box in enumerate(trial) if np.array_equal(box, cells[c]))
                nxt = subdivide(trial, at, i)
                if grid.d == 2 or pieces_have_sample_corners(shape, nxt):
                    trial = nxt
                    chosen.append((c, i))
                    if stats is not None and i != split_direction(grid, orc.phiE, R, c):
                        stats["fallbacks"] = stats.get("fallbacks", 0) + 1
                    break
                if stats is not None:
                    stats["skipped_splits"] = stats.get("skipped_splits", 0) + 1
            if len(chosen) == batch:
                break
        if not chosen:
            break
        # subdivide from the highest index down so earlier indices stay valid
        for c, i in sorted(chosen, key=lambda ci: -ci[0]):
            cells = subdivide(cells, c, i)
    return cells, history
