"""Blocks of A~ and A~* applied to vectors (Section 3.3), oracle side.

TEST INFRASTRUCTURE ONLY.  Boxes are closed, T = [t_lo, t_hi] (targets) and
S = [s_lo, s_hi] (sources); vectors on a box are C-order arrays of its shape.

* :func:`apply_block` is the definition: x_S extended by zero to Omega, the
  oracle's direct-sum A~ (or A~*), restricted to T.
* :func:`translated_convolution` is the translation identity of Section 3.3:
  for f supported on S, (phi * f)[T] = (phi_0 * f_0)[T'] with f_0 = f moved
  from s_min to the origin, phi_0 = phi on G = T - S moved from g_min to the
  origin, T' = T - t_min + s_max - s_min.  One linear convolution of shape
  |S| + |G| - 1 per axis, formed with an FFT (the library primitive).
* :func:`apply_block_translated` sums that identity over the terms that can
  be non-zero: k with U_k meeting S for A~[T, S] (Eq. conv_op_approx_main),
  k with U_k meeting T for (A~*)[T, S] (Eq. adjoint_random_z), in ascending k.
"""
from __future__ import annotations

import numpy as np

from .weights import weight_on_omega


def _box(lo, hi):
    lo = np.asarray(lo, dtype=np.int64)
    hi = np.asarray(hi, dtype=np.int64)
    if lo.shape != hi.shape or np.any(hi < lo):
        raise ValueError("a box needs lo <= hi on every axis")
    return lo, hi


def _slices(lo, hi):
    return tuple(slice(int(a), int(b) + 1) for a, b in zip(lo, hi))


def apply_block(orc, t_lo, t_hi, s_lo, s_hi, xS: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """[B][*T] = A~[T, S] x_S (or (A~*)[T, S] x_S) for xS of shape [B][*S]."""
    t_lo, t_hi = _box(t_lo, t_hi)
    s_lo, s_hi = _box(s_lo, s_hi)
    sS = tuple(int(v) for v in s_hi - s_lo + 1)
    xS = np.asarray(xS, dtype=np.float64).reshape((-1,) + sS)
    full = np.zeros((xS.shape[0],) + orc.shape)
    full[(slice(None),) + _slices(s_lo, s_hi)] = xS
    y = orc.apply_adjoint(full) if adjoint else orc.apply(full)
    return y[(slice(None),) + _slices(t_lo, t_hi)]


def translated_convolution(phi_win: np.ndarray, R: int, f: np.ndarray, s_lo, s_hi, t_lo, t_hi) -> np.ndarray:
    """(phi * f)[T] for phi given on the window [-R, R]^d (zero outside) and
    f given on S (shape of S), by the translation identity of Section 3.3."""
    s_lo, s_hi = _box(s_lo, s_hi)
    t_lo, t_hi = _box(t_lo, t_hi)
    d = len(s_lo)
    g_lo, g_hi = t_lo - s_hi, t_hi - s_lo                 # G = T - S
    nS = s_hi - s_lo + 1
    nG = g_hi - g_lo + 1
    nT = t_hi - t_lo + 1
    # phi_0[z0] = phi[z0 + g_min] on G_0, zero where G leaves the window
    phi0 = np.zeros(tuple(int(v) for v in nG))
    w = np.asarray(phi_win, dtype=np.float64).reshape((2 * R + 1,) * d)
    a = np.maximum(g_lo, -R)
    b = np.minimum(g_hi, R)
    if np.any(b < a):
        return np.zeros(tuple(int(v) for v in nT))
    phi0[_slices(a - g_lo, b - g_lo)] = w[_slices(a + R, b + R)]
    f0 = np.asarray(f, dtype=np.float64).reshape(tuple(int(v) for v in nS))
    full = tuple(int(v) for v in nS + nG - 1)
    ax = tuple(range(d))
    conv = np.fft.irfftn(np.fft.rfftn(f0, full, ax) * np.fft.rfftn(phi0, full, ax), full, ax)
    # T' = T - t_min + s_max - s_min
    off = s_hi - s_lo
    return conv[_slices(off, off + nT - 1)]


def _meets(lo, hi, blo, bhi) -> bool:
    return bool(np.all(np.maximum(lo, blo) <= np.minimum(hi, bhi)))


def block_terms(orc, t_lo, t_hi, s_lo, s_hi, adjoint: bool = False):
    """The k whose terms can be non-zero: U_k meets S (adjoint: T)."""
    lo, hi = _box(t_lo, t_hi) if adjoint else _box(s_lo, s_hi)
    g = orc.grid
    out = []
    for k in range(g.r):
        if any(_meets(g.cells[c][0], g.cells[c][1], lo, hi) for c in g.cells_of[k]):
            out.append(k)
    return out


def apply_block_translated(orc, t_lo, t_hi, s_lo, s_hi, xS: np.ndarray, adjoint: bool = False) -> np.ndarray:
    """Same result as apply_block, one translated small convolution per term."""
    t_lo, t_hi = _box(t_lo, t_hi)
    s_lo, s_hi = _box(s_lo, s_hi)
    g = orc.grid
    d = g.d
    sS = tuple(int(v) for v in s_hi - s_lo + 1)
    sT = tuple(int(v) for v in t_hi - t_lo + 1)
    xS = np.asarray(xS, dtype=np.float64).reshape((-1,) + sS)
    out = np.zeros((xS.shape[0],) + sT)
    for k in block_terms(orc, t_lo, t_hi, s_lo, s_hi, adjoint):
        wk = np.where(g.U_mask_full(k), weight_on_omega(g, orc.W, k), 0.0)
        phi = orc.phiE[k].reshape((2 * orc.R + 1,) * d)
        if adjoint:
            psi = phi[(slice(None, None, -1),) * d]      # flip(phi_k^E)[z] = phi_k^E[-z]
            wT = wk[_slices(t_lo, t_hi)]
            for b in range(xS.shape[0]):
                out[b] += wT * translated_convolution(psi, orc.R, xS[b], s_lo, s_hi, t_lo, t_hi)
        else:
            wS = wk[_slices(s_lo, s_hi)]
            for b in range(xS.shape[0]):
                out[b] += translated_convolution(phi, orc.R, wS * xS[b], s_lo, s_hi, t_lo, t_hi)
    return out
