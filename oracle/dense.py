"""Dense operators on tiny boxes (oracle; test infrastructure only).

* A~[y, x] = sum_{k: x in U_k} w_k[x] phi_k^E[y - x]              Eq. conv_matrix_entries
* W_k[y, x] = sum_{j in nbrs(k)} w_j[x] v_j^(k)[y - x]             Eq. Wj_def
* F_k[y, x] = A[y - x + p_k, p_k] - A[y, x]                       Eq. translation_failure_operator
* mu_k^E = {(y, x): x in U_k^E, y in Omega, y - x + p_k in Omega}  Eq. skew_cylinder_set
  with U_k^E = union_{j in nbrs(k)} U_j
* F[y, x] = max_{k: (y, x) in mu_k^E} |F_k[y, x]|                  Eq. defn_of_F

Rows are outputs y, columns inputs x, C-order flattening of Omega.
"""
from __future__ import annotations

import numpy as np

from .extension import extension_weights
from .weights import weight_on_omega


def _coords(shape):
    return np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij"), axis=-1).reshape(-1, len(shape))


def _window_lookup(win: np.ndarray, Z: np.ndarray, R: int) -> np.ndarray:
    """win on [-R, R]^d, evaluated at offsets Z=[..., d]; zero outside the window."""
    d = Z.shape[-1]
    inside = np.all(np.abs(Z) <= R, axis=-1)
    idx = np.clip(Z + R, 0, 2 * R)
    w = win.reshape((2 * R + 1,) * d)
    return np.where(inside, w[tuple(idx[..., a] for a in range(d))], 0.0)


def dense_pc(orc) -> np.ndarray:
    """A~ from its entries (Eq. conv_matrix_entries)."""
    g = orc.grid
    X = _coords(g.shape)
    N = len(X)
    Z = X[:, None, :] - X[None, :, :]                 # y - x, [N(y), N(x), d]
    A = np.zeros((N, N))
    for k in range(g.r):
        Uk = g.U_mask_full(k).ravel()
        wk = weight_on_omega(g, orc.W, k).ravel()
        col = np.where(Uk, wk, 0.0)
        A += col[None, :] * _window_lookup(orc.phiE[k], Z, orc.R)
    return A


def dense_W(orc):
    """[r][N][N] partition-of-unity weights W_k of Proposition 4.3."""
    g = orc.grid
    X = _coords(g.shape)
    Z = X[:, None, :] - X[None, :, :]
    # v_j^(k) lives on all of Z^d, not only on the kernel window: build it on a
    # window that covers every difference y - x of the box
    Rb = max(g.shape) - 1
    V = extension_weights(g, Rb)                      # V[j][k] = v_j^(k)
    wfull = [weight_on_omega(g, orc.W, j).ravel() for j in range(g.r)]
    out = np.zeros((g.r, len(X), len(X)))
    for k in range(g.r):
        for j in g.nbrs[k]:
            j = int(j)
            out[k] += wfull[j][None, :] * _window_lookup(V[j][k], Z, Rb)
    return out


def mu_E(grid):
    """Indicators [r][N][N] of mu_k^E."""
    X = _coords(grid.shape)
    shp = np.asarray(grid.shape)
    out = np.zeros((grid.r, len(X), len(X)), dtype=bool)
    for k in range(grid.r):
        UE = np.zeros(grid.shape, dtype=bool)
        for j in grid.nbrs[k]:
            UE |= grid.U_mask_full(int(j))
        q = X[:, None, :] - X[None, :, :] + grid.points[k]
        ok = np.all((q >= 0) & (q < shp), axis=-1)
        out[k] = ok & UE.ravel()[None, :]
    return out


def dense_F(grid, Adense: np.ndarray):
    """[r][N][N] F_k on mu_k^E (zero elsewhere) and F."""
    X = _coords(grid.shape)
    shp = np.asarray(grid.shape)
    mu = mu_E(grid)
    N = len(X)
    Fk = np.zeros((grid.r, N, N))
    strides = np.array([int(np.prod(grid.shape[a + 1:])) for a in range(grid.d)])
    for k in range(grid.r):
        q = X[:, None, :] - X[None, :, :] + grid.points[k]
        ok = np.all((q >= 0) & (q < shp), axis=-1)
        qi = np.clip(q, 0, shp - 1) @ strides
        pk = int(grid.points[k] @ strides)
        vals = np.where(ok, Adense[qi, pk], 0.0) - Adense
        Fk[k] = np.where(mu[k], vals, 0.0)
    F = np.max(np.abs(Fk), axis=0)
    return Fk, F, mu
