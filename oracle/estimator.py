"""Randomized a-posteriori error estimator (Section 2.6), oracle side (test
infrastructure only).

    e_C   = || (A~ - A)[Omega, C] ||                    (Eq. relative_error)
    eta_C = (1/sqrt(q)) || Y~[C, .] - Y[C, .] ||        (Eq. randomized_estimator_ec)

with Y = A* Z and Y~ = A~* Z for a probe matrix Z with q columns (the paper
draws Z ~ N(0,1)^{N x q}; the estimator is the sample average approximation
of Eq. saa_XZ).  Cells are the grid's closed leaf boxes, in grid order, so a
point on a shared facet counts in every cell that contains it.  Norms are
Frobenius norms over the cell's points and all q columns, in FP64.
"""
from __future__ import annotations

import numpy as np


def cell_point_indices(grid, c: int) -> np.ndarray:
    """Flat C-order indices of the points of leaf cell c (closed box)."""
    lo, hi = grid.cells[c]
    axes = [np.arange(int(a), int(b) + 1) for a, b in zip(lo, hi)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.ravel_multi_index([m.ravel() for m in mesh], grid.shape)


def eta_from_adjoints(grid, ytilde: np.ndarray, y: np.ndarray) -> np.ndarray:
    """eta_C for every cell from Y~ = A~* Z and Y = A* Z, both [q][N]."""
    yt = np.asarray(ytilde, dtype=np.float64).reshape(len(ytilde), -1)
    yy = np.asarray(y, dtype=np.float64).reshape(len(y), -1)
    q = yt.shape[0]
    out = np.zeros(len(grid.cells))
    for c in range(len(grid.cells)):
        idx = cell_point_indices(grid, c)
        d = yt[:, idx] - yy[:, idx]
        out[c] = np.sqrt(np.sum(d * d) / q)
    return out


def eta(orc, z: np.ndarray, y: np.ndarray) -> np.ndarray:
    """eta_C with Y~ = A~* Z computed by the oracle's adjoint apply."""
    return eta_from_adjoints(orc.grid, orc.apply_adjoint(z), y)


def true_cell_errors(grid, A_tilde: np.ndarray, A: np.ndarray) -> np.ndarray:
    """e_C = ||(A~ - A)[Omega, C]||_F from dense matrices (tiny boxes)."""
    D = np.asarray(A_tilde, dtype=np.float64) - np.asarray(A, dtype=np.float64)
    return np.array([np.linalg.norm(D[:, cell_point_indices(grid, c)]) for c in range(len(grid.cells))])
