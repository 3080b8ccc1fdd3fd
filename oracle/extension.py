"""Extended impulse responses phi_k^E of Section 2.5 (oracle; test infrastructure only).

All functions of z live on the window Z = [-R, R]^d (C order, index z + R);
the truncated operator makes every phi_j vanish outside it, so every phi_k^E
does too.  Following the text literally:

  c_k      = 1_{Omega - p_k} + sum_{j in nbrs(k), j != k} 1_{(Omega - p_j) \\ (Omega - p_k)}
  v_k      = 1 / c_k on supp(c_k), else 0
  v_k^(j)  = v_k 1_{Omega - p_k}                          (j = k)
           = v_k 1_{(Omega - p_j) \\ (Omega - p_k)}       (j in nbrs(k), j != k)   [Eq. vj_def]
  phi_k^E  = sum_{j in nbrs(k)} v_k^(j) phi_j                                        [Eq. def_varphiE]

supp(phi_j) is the domain Omega - p_j (Section 1.3: the largest set on which
the function could be non-zero), not the set where the truncated kernel
happens to be non-zero.  With extend=False the routine returns phi_k itself
(extension by zero), which the tests use to show the boundary artifact of
Fig. 1d_conv.
"""
from __future__ import annotations

from typing import Dict, List, Tuple

import numpy as np

from .grid import Grid


def window_offsets(d: int, R: int) -> np.ndarray:
    return np.stack(np.meshgrid(*[np.arange(-R, R + 1)] * d, indexing="ij"), axis=-1)


def domain_indicator(grid: Grid, p: np.ndarray, R: int) -> np.ndarray:
    """1_{Omega - p} on the window."""
    z = window_offsets(grid.d, R)
    y = z + np.asarray(p)
    return np.all((y >= 0) & (y < np.asarray(grid.shape)), axis=-1)


def extension_weights(grid: Grid, R: int) -> List[Dict[int, np.ndarray]]:
    """v_k^(j) on the window for every k and j in nbrs(k)."""
    ind = [domain_indicator(grid, grid.points[k], R) for k in range(grid.r)]
    out = []
    for k in range(grid.r):
        c = ind[k].astype(np.float64)
        for j in grid.nbrs[k]:
            if j != k:
                c = c + (ind[j] & ~ind[k])
        v = np.where(c > 0, 1.0 / np.where(c > 0, c, 1.0), 0.0)
        vk = {}
        for j in grid.nbrs[k]:
            j = int(j)
            if j == k:
                vk[j] = v * ind[k]
            else:
                vk[j] = v * (ind[j] & ~ind[k])
        out.append(vk)
    return out


def extend_impulse_responses(grid: Grid, phi: np.ndarray, R: int, extend: bool = True) -> np.ndarray:
    """phi: [r][(2R+1)^d] impulse responses (zero outside Omega - p_k).
    Returns phi^E with the same layout."""
    d = grid.d
    w = 2 * R + 1
    phi = np.asarray(phi, dtype=np.float64).reshape((grid.r,) + (w,) * d)
    if not extend:
        return phi.reshape(grid.r, -1).copy()
    V = extension_weights(grid, R)
    out = np.zeros_like(phi)
    for k in range(grid.r):
        acc = np.zeros((w,) * d)
        for j, vkj in V[k].items():
            acc = acc + vkj * phi[j]
        out[k] = acc
    return out.reshape(grid.r, -1)
