"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module holds none of the product-convolution arithmetic.  It only makes
the things a *user* of the method supplies:

* the box Omega and a leaf-cell grid (regular, or the quadtree rule used for
  the adaptive 1024^2 workload),
* the operator A being approximated, as a closed-form kernel A[y, x] (the
  paper's L0 "apply A" access: Eq. varphi_p, Section 1),
* impulse-response windows phi_k[z] = (A delta_{p_k})[z + p_k] for sample
  points the caller passes in (Eq. varphi_p_section2),
* right-hand sides x ~ iid N(0, 1).

Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014), used counter-style: output i of
stream s is mix(seed + (i + 1) * 0x9E3779B97F4A7C15).  Normals use the
Box-Muller transform.  Seeds are ``workload_index * 1000 + stream``.

All values are generated in FP64; right-hand sides are rounded to FP32 once so
that the oracle (which promotes that FP32 vector back to FP64) and the GPU see
bit-identical inputs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, List, Sequence, Tuple

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, n: int) -> np.ndarray:
    """Outputs start..start+n-1 of the SplitMix64 stream with the given seed."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


class Stream:
    """Sequential view of one counter-based SplitMix64 stream."""

    def __init__(self, seed: int):
        self.seed = int(seed)
        self.pos = 0

    def uniform(self, n: int) -> np.ndarray:
        """n doubles in [0, 1): top 53 bits of each output times 2^-53."""
        z = splitmix64(self.seed, self.pos, n)
        self.pos += n
        return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)

    def normal(self, n: int) -> np.ndarray:
        """n iid N(0,1) doubles by Box-Muller on consecutive uniform pairs."""
        m = (n + 1) // 2
        u = self.uniform(2 * m)
        u1 = 1.0 - u[0::2]  # (0, 1]
        u2 = u[1::2]
        rad = np.sqrt(-2.0 * np.log(u1))
        out = np.empty(2 * m)
        out[0::2] = rad * np.cos(2.0 * math.pi * u2)
        out[1::2] = rad * np.sin(2.0 * math.pi * u2)
        return out[:n]


def rhs(seed: int, nrhs: int, shape: Sequence[int]) -> np.ndarray:
    """Right-hand sides x[b] ~ iid N(0,1), rounded to FP32, layout [B][n1][n2](...)."""
    n = int(np.prod(shape))
    return Stream(seed).normal(nrhs * n).astype(np.float32).reshape((nrhs,) + tuple(shape))


# --------------------------------------------------------------------------
# Grids: leaf cells are closed integer boxes [lo, hi] that tile Omega and share
# facets (Section 2.2).  A grid is an int array [num_cells][2][d].
# --------------------------------------------------------------------------

def regular_points_1d(length: int, n: int) -> np.ndarray:
    """n sample coordinates on [0, length-1], both ends included: floor(i(L-1)/(n-1) + 1/2)."""
    return np.array([int(math.floor(i * (length - 1) / (n - 1) + 0.5)) for i in range(n)], dtype=np.int64)


def regular_grid(shape: Sequence[int], npts: Sequence[int]) -> np.ndarray:
    """Leaf cells of a regular sample grid with npts[i] points per axis (npts[i]-1 cells)."""
    axes = [regular_points_1d(L, n) for L, n in zip(shape, npts)]
    d = len(shape)
    cells = []
    for idx in np.ndindex(*[n - 1 for n in npts]):
        lo = [axes[a][idx[a]] for a in range(d)]
        hi = [axes[a][idx[a] + 1] for a in range(d)]
        cells.append([lo, hi])
    return np.array(cells, dtype=np.int32).reshape(-1, 2, d)


def _split_box(lo, hi, axis):
    mid = (lo[axis] + hi[axis]) // 2
    a_hi = list(hi)
    a_hi[axis] = mid
    b_lo = list(lo)
    b_lo[axis] = mid
    return (list(lo), a_hi), (b_lo, list(hi))


def quadtree_grid(shape: Sequence[int], min_level: int, max_level: int,
                  refine: Callable[[List[int], List[int]], bool]) -> np.ndarray:
    """2D quadtree leaves: uniform to min_level, then cells where refine(lo, hi) is
    true are split in both axes (at floor((lo+hi)/2)) until max_level."""
    root = ([0, 0], [shape[0] - 1, shape[1] - 1])
    leaves = []

    def rec(lo, hi, level):
        if level < min_level or (level < max_level and refine(lo, hi)):
            c0, c1 = _split_box(lo, hi, 0)
            for c in (c0, c1):
                d0, d1 = _split_box(c[0], c[1], 1)
                rec(d0[0], d0[1], level + 1)
                rec(d1[0], d1[1], level + 1)
        else:
            leaves.append([lo, hi])

    rec(root[0], root[1], 0)
    return np.array(leaves, dtype=np.int32).reshape(-1, 2, 2)


# --------------------------------------------------------------------------
# Smooth random parameter fields (sum of 4 seeded low-frequency sinusoids).
# --------------------------------------------------------------------------

@dataclass
class SmoothField:
    """s(x) = 1/2 (1 + sum_i a_i sin(2 pi k_i.x / L + ph_i) / sum_i a_i) in [0, 1],
    mapped linearly to [lo, hi]."""
    shape: Tuple[int, ...]
    lo: float
    hi: float
    seed: int
    a: np.ndarray = field(init=False)
    k: np.ndarray = field(init=False)
    ph: np.ndarray = field(init=False)

    def __post_init__(self):
        st = Stream(self.seed)
        d = len(self.shape)
        self.a = 0.5 + 0.5 * st.uniform(4)
        ks = []
        while len(ks) < 4:
            kk = np.floor(st.uniform(d) * 7.0).astype(np.int64) - 3
            if np.any(kk != 0):
                ks.append(kk)
        self.k = np.array(ks, dtype=np.float64)
        self.ph = 2.0 * math.pi * st.uniform(4)

    def __call__(self, x: np.ndarray) -> np.ndarray:
        """x: [..., d] coordinates (float) -> field values [...]."""
        x = np.asarray(x, dtype=np.float64)
        L = np.asarray(self.shape, dtype=np.float64)
        s = np.zeros(x.shape[:-1])
        for i in range(4):
            s = s + self.a[i] * np.sin(2.0 * math.pi * np.sum(self.k[i] * x / L, axis=-1) + self.ph[i])
        s = 0.5 * (1.0 + s / np.sum(self.a))
        return self.lo + (self.hi - self.lo) * s


# --------------------------------------------------------------------------
# Operators A (closed-form kernels).  A[y, x] = K(y - x; params(x)) for
# |y - x|_2 <= R, else 0.  Parameters are evaluated at the source x.
# --------------------------------------------------------------------------

class Kernel:
    """Base: subclasses implement value(z, x) for offsets z=[..., d], sources x=[..., d]."""
    radius: int

    def value(self, z: np.ndarray, x: np.ndarray) -> np.ndarray:  # pragma: no cover
        raise NotImplementedError

    def entry(self, y: np.ndarray, x: np.ndarray) -> np.ndarray:
        """A[y, x] with truncation |y - x|_2 <= R (closed)."""
        y = np.asarray(y, dtype=np.float64)
        x = np.asarray(x, dtype=np.float64)
        z = y - x
        v = self.value(z, x)
        return np.where(np.sum(z * z, axis=-1) <= float(self.radius) ** 2, v, 0.0)


class GaussianIso(Kernel):
    """exp(-|z|^2 / (2 s(x)^2)) / (2 pi s(x)^2)  (2D), s given as a callable."""

    def __init__(self, sigma: Callable, radius: int):
        self.sigma = sigma
        self.radius = radius

    def value(self, z, x):
        s = self.sigma(x)
        return np.exp(-np.sum(z * z, axis=-1) / (2.0 * s * s)) / (2.0 * math.pi * s * s)


class GaussianAniso2D(Kernel):
    """Rotated anisotropic Gaussian exp(-z^T S^-1 z / 2) / (2 pi s1 s2),
    S = Rot(t) diag(s1^2, s2^2) Rot(t)^T, all three evaluated at the source."""

    def __init__(self, s1: Callable, s2: Callable, theta: Callable, radius: int):
        self.s1, self.s2, self.theta = s1, s2, theta
        self.radius = radius

    def value(self, z, x):
        a, b, t = self.s1(x), self.s2(x), self.theta(x)
        c, s = np.cos(t), np.sin(t)
        u = c * z[..., 0] + s * z[..., 1]
        v = -s * z[..., 0] + c * z[..., 1]
        return np.exp(-0.5 * (u * u / (a * a) + v * v / (b * b))) / (2.0 * math.pi * a * b)


class GaussianAxis3D(Kernel):
    """Axis-aligned 3D Gaussian exp(-sum z_i^2/(2 s_i^2)) / ((2 pi)^{3/2} s1 s2 s3)."""

    def __init__(self, s1: Callable, s2: Callable, s3: Callable, radius: int):
        self.s = (s1, s2, s3)
        self.radius = radius

    def value(self, z, x):
        sig = [f(x) for f in self.s]
        q = sum(z[..., i] ** 2 / (sig[i] ** 2) for i in range(3))
        return np.exp(-0.5 * q) / ((2.0 * math.pi) ** 1.5 * sig[0] * sig[1] * sig[2])


class HeavyTailed(Kernel):
    """(1 + |z|^2 / s(x)^2)^(-3/2), unnormalised."""

    def __init__(self, sigma: Callable, radius: int):
        self.sigma = sigma
        self.radius = radius

    def value(self, z, x):
        s = self.sigma(x)
        return (1.0 + np.sum(z * z, axis=-1) / (s * s)) ** -1.5


class Skewed(Kernel):
    """Off-centre Gaussian exp(-|z - mu(x)|^2 / (2 s^2)): not symmetric under
    z -> -z, so a flipped convolution index cannot go unnoticed."""

    def __init__(self, mu: Sequence[float], sigma: Callable, radius: int):
        self.mu = np.asarray(mu, dtype=np.float64)
        self.sigma = sigma
        self.radius = radius

    def value(self, z, x):
        s = self.sigma(x)
        dz = z - self.mu
        return np.exp(-np.sum(dz * dz, axis=-1) / (2.0 * s * s))


def impulse_windows(shape: Sequence[int], points: np.ndarray, kernel: Kernel) -> np.ndarray:
    """phi_k[z] = A[z + p_k, p_k] on the window z in [-R, R]^d, zero where
    z + p_k lies outside Omega.  Returns FP64 [r][(2R+1)^d], z + R in C order."""
    points = np.asarray(points, dtype=np.int64)
    r, d = points.shape
    R = kernel.radius
    w = 2 * R + 1
    offs = np.stack(np.meshgrid(*[np.arange(-R, R + 1)] * d, indexing="ij"), axis=-1).reshape(-1, d)
    out = np.zeros((r, w ** d))
    shp = np.asarray(shape)
    chunk = max(1, 4_000_000 // (w ** d))
    for c0 in range(0, r, chunk):
        p = points[c0:c0 + chunk]                         # [c, d]
        y = p[:, None, :] + offs[None, :, :]              # [c, w^d, d]
        inside = np.all((y >= 0) & (y < shp), axis=-1)
        xx = np.broadcast_to(p[:, None, :], y.shape)
        v = kernel.entry(y, xx)
        out[c0:c0 + chunk] = np.where(inside, v, 0.0)
    return out


def dense_operator(shape: Sequence[int], kernel: Kernel) -> np.ndarray:
    """Dense A[y, x] on a tiny box (row y, column x, C-order flattening)."""
    pts = np.stack(np.meshgrid(*[np.arange(n) for n in shape], indexing="ij"), axis=-1).reshape(-1, len(shape))
    Y = pts[:, None, :]
    X = pts[None, :, :]
    return kernel.entry(np.broadcast_to(Y, (len(pts), len(pts), len(shape))),
                        np.broadcast_to(X, (len(pts), len(pts), len(shape))))


def impulse_windows_from_matrix(shape: Sequence[int], points: np.ndarray, R: int, A: np.ndarray) -> np.ndarray:
    """phi_k[z] = (A delta_{p_k})[z + p_k] read from a dense operator (column p_k),
    on the window [-R, R]^d, zero where z + p_k lies outside Omega."""
    points = np.asarray(points, dtype=np.int64)
    r, d = points.shape
    shp = np.asarray(shape)
    strides = np.array([int(np.prod(shape[a + 1:])) for a in range(d)])
    offs = np.stack(np.meshgrid(*[np.arange(-R, R + 1)] * d, indexing="ij"), axis=-1).reshape(-1, d)
    out = np.zeros((r, len(offs)))
    for k in range(r):
        col = A[:, int(points[k] @ strides)]
        y = offs + points[k]
        inside = np.all((y >= 0) & (y < shp), axis=-1)
        yi = np.clip(y, 0, shp - 1) @ strides
        out[k] = np.where(inside, col[yi], 0.0)
    return out
