"""Adaptive construction of A~ (Algorithm 1) on the library.

The caller supplies the matrix-free access the paper assumes:
  impulse(points) -> phi_k = A delta_{p_k} on the window [-R, R]^d for each
      new sample point (one application of A per point),
  Z, Y = A* Z: q probe vectors and their images under A* (q applications of
      A*), as CUDA tensors [q, *box] in the operator's precision.
Each pass builds the operator on the current leaf cells (U_k, harmonic
weights w_k, extended impulse responses phi_k^E and spectra in libpc),
estimates eta_C for every leaf (pc_estimate_cell_errors: A~* Z on the GPU,
FP64 cell norms) and refines.

Each pass then calls pc_refine, which computes the overall estimator
eta_Omega = sqrt(sum_C eta_C^2) / (||Y||_F / sqrt(q)) (a relative error
estimate; a point on a shared facet counts in each cell that holds it) and,
while eta_Omega > tau, splits the leaf with the largest eta_C (Section 2.7)
in the direction of largest change of phi^E, at floor((c_min + c_max) / 2);
batch > 1 splits up to that many leaves per pass (largest eta_C first),
batch = 1 is Algorithm 1 as printed.  In 3D a split that would break the two
sides of a facet crosswise is skipped for the leaf's next direction
(pc_split_is_admissible): the facet's pieces would meet at a point that is
no cell's corner, where the recursive weights of Section 2.4 have no value.
All of this is libpc's host code; this module only marshals.

Each pass rebuilds the operator (geometry, weights and spectra in libpc).
Y~ = A~* Z is updated incrementally, as Algorithm 1 does (`incremental`,
the default): the correlations flip(phi_k^E) * Z of sample points whose
phi_k^E and bbox(U_k) are unchanged are kept from the previous pass, and
only new points and points with a new neighbour are recomputed
(pc_estimator_update).  With incremental=False, and for 3D boxes, every
pass recomputes all of them (pc_estimate_cell_errors).  3D leaves with
hanging nodes get their harmonic weights through the facet pieces of
Section 2.4 (the library handles them when it builds each pass's operator).
"""
from __future__ import annotations

from itertools import product
from typing import Callable, List, Tuple

import numpy as np

from .binding import Estimator, Operator, pc_refine, pc_sample_points


def _first_cells(shape) -> List[Tuple[List[int], List[int]]]:
    """Omega split once along every axis at floor((0 + n - 1) / 2)."""
    d = len(shape)
    mids = [(n - 1) // 2 for n in shape]
    out = []
    for side in product((0, 1), repeat=d):
        lo = [0 if s == 0 else mids[a] for a, s in enumerate(side)]
        hi = [mids[a] if s == 0 else shape[a] - 1 for a, s in enumerate(side)]
        out.append((lo, hi))
    return out


def construct(ctx, shape, impulse: Callable[[np.ndarray], np.ndarray], R: int, Z, Y, tau: float,
              precision: str = "fp32", max_passes: int = 100, batch: int = 1, incremental: bool = True,
              stats: dict = None, **tune):
    """Algorithm 1.  Returns (operator, cells [n][2][d], history [(r, eta_Omega)]).
    If `stats` is a dict it receives "recomputed": the number of sample
    points whose correlations each pass computed."""
    shape = tuple(int(n) for n in shape)
    q = Z.shape[0]
    # the incremental estimator covers 2D boxes; 3D passes re-estimate in full
    est = Estimator(ctx, shape, Z, Y, precision) if incremental and len(shape) == 2 else None
    recomputed = []
    # y_rms = ||Y||_F / sqrt(q), from the caller's A* Z
    y_rms = float(np.linalg.norm(Y.reshape(q, -1).double().cpu().numpy())) / np.sqrt(q)
    cells = np.array(_first_cells(shape), dtype=np.int32)
    known = {}
    history = []
    op = None
    for _ in range(max_passes):
        pts = pc_sample_points(shape, cells)
        fresh = [tuple(int(v) for v in p) for p in pts if tuple(int(v) for v in p) not in known]
        if fresh:
            for p, ph in zip(fresh, impulse(np.array(fresh))):
                known[p] = np.asarray(ph, dtype=np.float64).ravel()
        phi = np.stack([known[tuple(int(v) for v in p)] for p in pts])
        if op is not None:
            op.close()
        op = Operator(ctx, shape, cells, R, phi, precision=precision, **tune)
        if est is not None:
            eta_c, nrec = est.update(op, len(cells))
        else:
            eta_c, nrec = op.estimate_cell_errors(Z, Y, len(cells)), len(pts)
        recomputed.append(nrec)
        # eta_Omega and the refinement (leaf choice, direction, admissibility): libpc
        eta_o, nxt = pc_refine(shape, cells, R, phi, eta_c, y_rms, tau, batch)
        history.append((len(pts), eta_o))
        if eta_o <= tau or len(nxt) == len(cells):
            break
        cells = nxt
    if est is not None:
        est.close()
    if stats is not None:
        stats["recomputed"] = recomputed
    return op, np.asarray(cells), history
