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

Overall estimator: eta_Omega = sqrt(sum_C eta_C^2) / (||Y||_F / sqrt(q)),
a relative error estimate (a point on a shared facet counts in each cell
that holds it).  While eta_Omega > tau, the leaf with the largest eta_C is
split (Section 2.7) in the direction i, among those with c_max^i - c_min^i
> 2, that maximises || phi^{i+} - phi^{i-} || over the window offsets z with
c_mid + z in Omega, where phi^{i+-} averages phi_k^E over the cell's corners
on its front / back face in direction i; values within a relative 1e-9 of
the largest are a tie, won by the lowest i.  The split is at
floor((c_min + c_max) / 2).  batch > 1 splits up to that many leaves per
pass (largest eta_C first); batch = 1 is Algorithm 1 as printed.

In 3D a split can break the two sides of a facet crosswise (one side split
along one axis, the other along another): the facet's pieces then meet at a
point that is no cell's corner, where the recursive weights of Section 2.4
have no value (libpc refuses such grids with PC_ERR_GRID).  A leaf therefore
takes its directions in the order above (each the best of those left) and
splits in the first one that keeps every facet piece's corners at sample
points; a leaf with none is passed over for the next by eta_C.  In 2D facets
are segments and every split qualifies.

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

from .binding import Estimator, Operator, pc_extend_impulse, pc_sample_points


def _first_cells(shape) -> List[Tuple[List[int], List[int]]]:
    d = len(shape)
    mids = [(n - 1) // 2 for n in shape]
    out = []
    for side in product((0, 1), repeat=d):
        lo = [0 if s == 0 else mids[a] for a, s in enumerate(side)]
        hi = [mids[a] if s == 0 else shape[a] - 1 for a, s in enumerate(side)]
        out.append((lo, hi))
    return out


def _directions(shape, lo, hi, point_index, phiE, R) -> List[int]:
    d = len(shape)
    W = 2 * R + 1
    cmid = [(a + b) // 2 for a, b in zip(lo, hi)]
    grids = np.meshgrid(*[np.arange(-R, R + 1)] * d, indexing="ij")
    mask = np.ones((W,) * d, dtype=bool)
    for a in range(d):
        mask &= (cmid[a] + grids[a] >= 0) & (cmid[a] + grids[a] < shape[a])
    mask = mask.ravel()
    scores = {}
    for i in range(d):
        if hi[i] - lo[i] <= 2:
            continue
        front = np.zeros(W ** d)
        back = np.zeros(W ** d)
        for corner in product(*[(lo[a], hi[a]) for a in range(d)]):
            k = point_index[corner]
            if corner[i] == hi[i]:
                front += phiE[k]
            else:
                back += phiE[k]
        delta = (front - back) * (2.0 ** (1 - d))
        scores[i] = float(np.linalg.norm(delta[mask]))
    out = []
    while scores:
        top = max(scores.values())
        i = min(j for j, v in scores.items() if v >= top - 1e-9 * top)
        out.append(i)
        del scores[i]
    return out


def _split(cells, box, i):
    """cells with leaf `box` replaced by its halves along axis i."""
    lo, hi = box
    m = (lo[i] + hi[i]) // 2
    out = [c for c in cells if not (list(c[0]) == list(lo) and list(c[1]) == list(hi))]
    out.append((list(lo), [m if a == i else hi[a] for a in range(len(lo))]))
    out.append(([m if a == i else lo[a] for a in range(len(lo))], list(hi)))
    return out


def _pieces_end_at_points(cells, new_boxes) -> bool:
    """Whether every facet piece of the leaves `new_boxes` (their facets'
    intersections of positive area with the facets of the leaves across)
    has cell corners at its corners.  Pieces away from them are unchanged by
    a split."""
    d = len(cells[0][0])
    corners = set()
    for lo, hi in cells:
        corners.update(product(*[(lo[a], hi[a]) for a in range(d)]))
    for lo, hi in new_boxes:
        for a in range(d):
            for plane, far in ((lo[a], 1), (hi[a], 0)):
                for nlo, nhi in cells:
                    # a leaf across: its opposite facet lies on the same plane
                    if (nhi[a] if far else nlo[a]) != plane or (nlo[a] if far else nhi[a]) == plane:
                        continue
                    plo = [max(lo[b], nlo[b]) for b in range(d)]
                    phi = [min(hi[b], nhi[b]) for b in range(d)]
                    plo[a] = phi[a] = plane
                    if any(plo[b] >= phi[b] for b in range(d) if b != a):
                        continue
                    for corner in product(*[(plo[b], phi[b]) for b in range(d)]):
                        if corner not in corners:
                            return False
    return True


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
    ynorm = float(np.linalg.norm(Y.reshape(q, -1).double().cpu().numpy())) / np.sqrt(q)
    cells = _first_cells(shape)
    known = {}
    history = []
    op = None
    for _ in range(max_passes):
        arr = np.array(cells, dtype=np.int32)
        pts = pc_sample_points(shape, arr)
        fresh = [tuple(int(v) for v in p) for p in pts if tuple(int(v) for v in p) not in known]
        if fresh:
            for p, ph in zip(fresh, impulse(np.array(fresh))):
                known[p] = np.asarray(ph, dtype=np.float64).ravel()
        phi = np.stack([known[tuple(int(v) for v in p)] for p in pts])
        if op is not None:
            op.close()
        op = Operator(ctx, shape, arr, R, phi, precision=precision, **tune)
        if est is not None:
            eta_c, nrec = est.update(op, len(cells))
        else:
            eta_c, nrec = op.estimate_cell_errors(Z, Y, len(cells)), len(pts)
        recomputed.append(nrec)
        eta_o = float(np.sqrt(np.sum(eta_c ** 2))) / ynorm
        history.append((len(pts), eta_o))
        if eta_o <= tau:
            break
        phiE = pc_extend_impulse(shape, arr, R, phi)
        point_index = {tuple(int(v) for v in p): k for k, p in enumerate(pts)}
        picks = []
        trial = list(cells)   # the leaves as split so far this pass
        for c in sorted(range(len(cells)), key=lambda c: (-eta_c[c], c)):
            for i in _directions(shape, cells[c][0], cells[c][1], point_index, phiE, R):
                nxt = _split(trial, cells[c], i)
                if len(shape) == 2 or _pieces_end_at_points(nxt, nxt[-2:]):
                    trial = nxt
                    picks.append((c, i))
                    break
            if len(picks) == batch:
                break
        if not picks:
            break
        for c, i in sorted(picks, key=lambda ci: -ci[0]):
            lo, hi = cells.pop(c)
            m = (lo[i] + hi[i]) // 2
            cells.append((lo, [m if a == i else hi[a] for a in range(len(shape))]))
            cells.append(([m if a == i else lo[a] for a in range(len(shape))], hi))
    if est is not None:
        est.close()
    if stats is not None:
        stats["recomputed"] = recomputed
    return op, np.array(cells), history
