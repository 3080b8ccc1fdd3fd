"""Oracle operator object: grid + weights + extension + direct-sum apply
(test infrastructure only)."""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

from .build import build
from .extension import extend_impulse_responses
from .grid import Grid
from .weights import harmonic_weights

_lib = None


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        _lib.pc_oracle_apply.restype = ctypes.c_int
        _lib.pc_oracle_apply_adjoint.restype = ctypes.c_int
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class PCOracle:
    """A~ = sum_k phi_k^E * (w_k . f) on a box (Eq. conv_op_approx_main) and its
    adjoint A~* = sum_k w_k . (flip(phi_k^E) * f) (Eq. adjoint_random_z), FP64."""

    def __init__(self, shape: Sequence[int], cells, phi: np.ndarray, R: int, extend: bool = True,
                 weights=None):
        self.grid = Grid(shape, cells)
        self.shape = self.grid.shape
        self.d = self.grid.d
        self.R = int(R)
        self.W = harmonic_weights(self.grid) if weights is None else [np.asarray(w, np.float64) for w in weights]
        self.phi = np.asarray(phi, dtype=np.float64).reshape(self.grid.r, -1)
        self.phiE = extend_impulse_responses(self.grid, self.phi, self.R, extend=extend)

    @classmethod
    def from_workload(cls, wl, extend: bool = True):
        from workloads import impulse_windows
        g = Grid(wl.shape, wl.cells)
        phi = impulse_windows(wl.shape, g.points, wl.kernel)
        return cls(wl.shape, wl.cells, phi, wl.radius, extend=extend)

    # ------------------------------------------------------------------
    def _pad3(self, v, fill):
        v = list(v)
        return [fill] * (3 - len(v)) + v

    def _args(self):
        shape3 = np.array(self._pad3(self.shape, 1), dtype=np.int64)
        lo = np.array([self._pad3(self.grid.bbox_lo[k], 0) for k in range(self.grid.r)], dtype=np.int64)
        hi = np.array([self._pad3(self.grid.bbox_hi[k], 0) for k in range(self.grid.r)], dtype=np.int64)
        sizes = [w.size for w in self.W]
        off = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
        wcat = np.ascontiguousarray(np.concatenate([w.ravel() for w in self.W]).astype(np.float64))
        win = np.array(self._pad3([2 * self.R + 1] * self.d, 1), dtype=np.int64)
        phiE = np.ascontiguousarray(self.phiE, dtype=np.float64)
        return shape3, lo, hi, off, wcat, win, phiE

    def _run(self, fn, f, points, nthreads):
        f = np.ascontiguousarray(np.asarray(f, dtype=np.float64).reshape(-1, int(np.prod(self.shape))))
        B = f.shape[0]
        shape3, lo, hi, off, wcat, win, phiE = self._args()
        if points is None:
            ny = f.shape[1]
            yl = None
        else:
            yl = np.ascontiguousarray(np.asarray(points, dtype=np.int64).ravel())
            ny = yl.size
        out = np.zeros((B, ny))
        rc = fn(_p(shape3), ctypes.c_int32(self.grid.r), _p(lo), _p(hi), _p(off), _p(wcat), _p(win), _p(phiE),
                ctypes.c_int32(B), _p(f), ctypes.c_int64(ny), _p(yl) if yl is not None else ctypes.c_void_p(0),
                _p(out), ctypes.c_int32(nthreads))
        if rc != 0:
            raise MemoryError("oracle apply failed to allocate")
        if points is None:
            return out.reshape((B,) + self.shape)
        return out

    def apply(self, f: np.ndarray, points: Optional[np.ndarray] = None, nthreads: int = 0) -> np.ndarray:
        """f: [B][*shape] (any float dtype; promoted to FP64).  Returns [B][*shape],
        or [B][len(points)] when points (flat C-order indices) is given."""
        return self._run(_load().pc_oracle_apply, f, points, nthreads)

    def apply_adjoint(self, f: np.ndarray, points: Optional[np.ndarray] = None, nthreads: int = 0) -> np.ndarray:
        """A~* f (Eq. adjoint_random_z, real data: w_k times the correlation of
        f with phi_k^E); same shapes as apply."""
        return self._run(_load().pc_oracle_apply_adjoint, f, points, nthreads)
