"""Harmonic partition-of-unity weights of Section 2.4 (oracle; test infrastructure only).

For each leaf cell C and each sample point p_k in C, w_k on C is built
recursively in dimension (Fig. harmonic and the text beside it):

* 0-dim boxes (sample points): w_k[p_j] = delta_kj.
* 1-dim boxes (edges of C, split at every sample point lying on them): the
  discrete 1D Laplace equation with the endpoint values as Dirichlet data.
* m-dim boxes (faces, then the cell itself): the discrete Laplace equation
  with the graph Laplacian (positive definite, the Kronecker-sum five/seven
  point stencil) and the already computed boundary values as Dirichlet data.

Each Dirichlet problem is solved exactly (to rounding) in the eigenbasis of
the 1D Dirichlet Laplacian tridiag(-1, 2, -1) of size m, whose eigenvectors
are the orthonormal sine vectors S_ij = sqrt(2/(m+1)) sin(pi i j/(m+1)) with
eigenvalues 2 - 2 cos(pi i/(m+1)); the Kronecker-sum operator is diagonal in
the tensor product of these bases.  Dense matrix products only, no FFT.

w_k on Omega is the union of its pieces on the cells of cells(p_k); pieces on
shared facets agree because both cells solve the same lower-dimensional
problems.

Broken facets (Section 2.4): a facet of a 3D leaf that finer leaves across
it divide is replaced by its constituent smaller boxes, the intersections of
the facet with the facets of the leaves across it.  Each piece gets the
harmonic extension of its own (node-split) edges, and the leaf's interior the
3D extension of the union of its pieces.  In 2D the facets are edges, and
splitting them at every sample point on them is the same construction.
"""
from __future__ import annotations

import functools
from typing import Dict, List, Tuple

import numpy as np

from .grid import Grid, box_corners


@functools.lru_cache(maxsize=None)
def _sine_basis(m: int) -> Tuple[np.ndarray, np.ndarray]:
    i = np.arange(1, m + 1, dtype=np.float64)
    S = np.sqrt(2.0 / (m + 1)) * np.sin(np.pi * np.outer(i, i) / (m + 1))
    lam = 2.0 - 2.0 * np.cos(np.pi * i / (m + 1))
    return S, lam


def dirichlet_laplace(V: np.ndarray) -> np.ndarray:
    """Given values V on a box (any dim, every axis of extent >= 2) whose
    boundary layer holds Dirichlet data, return V with the interior replaced by
    the solution of the discrete graph-Laplace equation."""
    V = np.array(V, dtype=np.float64)
    m = V.ndim
    inner = tuple(slice(1, -1) for _ in range(m))
    shp = tuple(s - 2 for s in V.shape)
    if any(s <= 0 for s in shp):
        return V
    Vb = V.copy()
    Vb[inner] = 0.0
    # right-hand side: sum of the boundary neighbours of each interior node
    b = np.zeros(shp)
    for a in range(m):
        lo = [slice(1, -1)] * m
        hi = [slice(1, -1)] * m
        lo[a] = slice(0, -2)
        hi[a] = slice(2, None)
        b += Vb[tuple(lo)] + Vb[tuple(hi)]
    # solve (sum_a T_a) U = b in the sine eigenbasis
    U = b
    lam_sum = np.zeros(shp)
    for a in range(m):
        S, lam = _sine_basis(shp[a])
        U = np.moveaxis(np.tensordot(S, np.moveaxis(U, a, 0), axes=(1, 0)), 0, a)
        sh = [1] * m
        sh[a] = shp[a]
        lam_sum = lam_sum + lam.reshape(sh)
    U = U / lam_sum
    for a in range(m):
        S, _ = _sine_basis(shp[a])
        U = np.moveaxis(np.tensordot(S, np.moveaxis(U, a, 0), axes=(1, 0)), 0, a)
    V[inner] = U
    return V


def _segment_values(lo: np.ndarray, hi: np.ndarray, axis: int, nodes: Dict[tuple, float]) -> np.ndarray:
    """Values on the 1-dim box [lo, hi] (varying along `axis`): split at every
    node on it, 1D Laplace on each piece."""
    n = int(hi[axis] - lo[axis] + 1)
    out = np.full(n, np.nan)
    pos = sorted(int(p[axis]) for p in nodes
                 if all(p[a] == lo[a] for a in range(len(lo)) if a != axis) and lo[axis] <= p[axis] <= hi[axis])
    if pos[0] != lo[axis] or pos[-1] != hi[axis]:
        raise ValueError("edge endpoints must be sample points")
    for a, b in zip(pos[:-1], pos[1:]):
        pa = list(lo)
        pa[axis] = a
        pb = list(lo)
        pb[axis] = b
        seg = np.zeros(b - a + 1)
        seg[0] = nodes[tuple(pa)]
        seg[-1] = nodes[tuple(pb)]
        seg = dirichlet_laplace(seg)
        out[a - lo[axis]: b - lo[axis] + 1] = seg
    return out


def harmonic_on_box(lo, hi, nodes: Dict[tuple, float]) -> np.ndarray:
    """Harmonic extension of the node values over the box [lo, hi]; returns an
    array of the box's full d-dim shape (degenerate axes kept with extent 1)."""
    lo = np.asarray(lo, dtype=np.int64)
    hi = np.asarray(hi, dtype=np.int64)
    d = len(lo)
    shape = tuple(int(h - l + 1) for l, h in zip(lo, hi))
    axes = [a for a in range(d) if hi[a] > lo[a]]
    m = len(axes)
    if m == 0:
        return np.full(shape, nodes[tuple(int(v) for v in lo)])
    if m == 1:
        return _segment_values(lo, hi, axes[0], nodes).reshape(shape)
    # a sample point in the relative interior of a box of dimension >= 2 would
    # make it a broken box: those are split into pieces before they get here
    interior = [p for p in nodes if all(lo[a] <= p[a] <= hi[a] for a in range(d))
                and all(lo[a] < p[a] < hi[a] for a in axes)]
    if interior:
        raise ValueError("a sample point inside a %d-dim box: split it into its constituent boxes" % m)
    V = np.full(shape, np.nan)
    # boundary facets: fix one non-degenerate axis at its min or max
    for a in axes:
        for side in (0, 1):
            flo = lo.copy()
            fhi = hi.copy()
            if side == 0:
                fhi[a] = lo[a]
            else:
                flo[a] = hi[a]
            fv = harmonic_on_box(flo, fhi, nodes)
            sl = [slice(None)] * d
            sl[a] = slice(0, 1) if side == 0 else slice(shape[a] - 1, shape[a])
            V[tuple(sl)] = fv
    sq = tuple(a for a in range(d) if a not in axes)
    Vs = V.squeeze(axis=sq) if sq else V
    Vs = dirichlet_laplace(Vs)
    return Vs.reshape(shape)


def facet_pieces(grid: Grid, c: int, a: int, side: int) -> List[Tuple[np.ndarray, np.ndarray]]:
    """The boxes that make up facet (axis a, side 0 = min, 1 = max) of leaf c
    (Section 2.4): the facet itself on the boundary of Omega, else its
    intersections, of positive area, with the facets of the leaves across it."""
    lo, hi = (np.array(v, dtype=np.int64) for v in grid.cells[c])
    plane = int(hi[a] if side else lo[a])
    flo, fhi = lo.copy(), hi.copy()
    flo[a] = fhi[a] = plane
    if (side == 0 and plane == 0) or (side == 1 and plane == grid.shape[a] - 1):
        return [(flo, fhi)]
    others = [b for b in range(grid.d) if b != a]
    out = []
    for n, (nlo, nhi) in enumerate(grid.cells):
        if n == c or (side == 1 and nlo[a] != plane) or (side == 0 and nhi[a] != plane):
            continue
        plo, phi = flo.copy(), fhi.copy()
        for b in others:
            plo[b], phi[b] = max(lo[b], nlo[b]), min(hi[b], nhi[b])
        if all(plo[b] < phi[b] for b in others):
            out.append((plo, phi))
    area = sum(int(np.prod([phi[b] - plo[b] for b in others])) for plo, phi in out)
    if area != int(np.prod([hi[b] - lo[b] for b in others])):
        raise ValueError("the leaves across a facet do not tile it")
    return out


def cell_weights(grid: Grid, c: int) -> Dict[int, np.ndarray]:
    """w_k restricted to leaf c, for every sample point p_k in c."""
    lo, hi = grid.cells[c]
    ks = grid.points_of[c]
    out = {}
    for k in ks:
        nodes = {tuple(int(v) for v in grid.points[j]): (1.0 if j == k else 0.0) for j in ks}
        if grid.d == 3:
            # facets as their constituent boxes, then the 3D interior
            shape = tuple(int(h - l + 1) for l, h in zip(lo, hi))
            V = np.full(shape, np.nan)
            for a in range(3):
                for side in (0, 1):
                    for plo, phi in facet_pieces(grid, c, a, side):
                        sl = tuple(slice(int(x - o), int(y - o) + 1) for x, y, o in zip(plo, phi, lo))
                        V[sl] = harmonic_on_box(plo, phi, nodes)
            out[int(k)] = dirichlet_laplace(V)
        else:
            out[int(k)] = harmonic_on_box(lo, hi, nodes)
    return out


def harmonic_weights(grid: Grid) -> List[np.ndarray]:
    """w_k on bbox(U_k) for k = 0..r-1 (zero outside U_k)."""
    W = [np.zeros(grid.bbox_shape(k)) for k in range(grid.r)]
    seen = [np.zeros(grid.bbox_shape(k), dtype=bool) for k in range(grid.r)]
    for c in range(len(grid.cells)):
        lo, hi = grid.cells[c]
        for k, vals in cell_weights(grid, c).items():
            sl = tuple(slice(int(a - o), int(b - o) + 1) for a, b, o in zip(lo, hi, grid.bbox_lo[k]))
            prev = W[k][sl]
            m = seen[k][sl]
            if np.any(m) and np.max(np.abs(prev[m] - vals[m])) > 1e-12:
                raise AssertionError("harmonic pieces disagree on a shared facet")
            W[k][sl] = vals
            seen[k][sl] = True
    return W


def weight_on_omega(grid: Grid, W: List[np.ndarray], k: int) -> np.ndarray:
    full = np.zeros(grid.shape)
    full[tuple(slice(int(a), int(b) + 1) for a, b in zip(grid.bbox_lo[k], grid.bbox_hi[k]))] = W[k]
    return full
