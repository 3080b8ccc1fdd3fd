"""The synthetic workloads, by name and size.

Each builder returns a :class:`Workload`: box shape, leaf-cell grid, operator
kernel, truncation radius, right-hand-side count and seeds.  Nothing here
computes sample points, weights, extensions or convolutions.

Workloads (seeds are ``index * 1000 + stream``):

* ``fp64_64``   - 64x64, regular 4x4 sample grid, isotropic Gaussian blur with
  sigma(x) = 2 + sin(2 pi x1/64) cos(2 pi x2/64), R = 12, 1 RHS, FP64 path.
* ``fp32_512``  - 512x512, regular 16x16 grid, rotated anisotropic Gaussian,
  sigma1, sigma2 in [2, 8] and theta in [0, pi) as smooth random fields,
  R = 24, 64 RHS, FP32 path, 128^2 patch FFTs.
* ``adaptive_1024`` - 1024x1024 quadtree (levels 2..7) refined where
  |grad sigma| * cell width > 0.05 (max over a 5x5 sampling of the cell),
  heavy-tailed kernel (1 + |z|^2/sigma^2)^(-3/2) with sigma = 2 + 6
  logistic((|x - c| - 170)/4), c = (511.5, 511.5), R = 64.  This smooth ring
  stands in for the piecewise-constant blur of Section 5.1.
* ``fp32_128c`` - 3D 128^3, regular 8x8x8 grid, axis-aligned Gaussian with
  sigma_i in [1.5, 5] smooth random fields, R = 12, 32 RHS, 64^3 patch FFTs.
"""
from __future__ import annotations

import math
from dataclasses import dataclass
from typing import Optional, Tuple

import numpy as np

from . import (GaussianAniso2D, GaussianAxis3D, GaussianIso, HeavyTailed, Kernel,
               SmoothField, quadtree_grid, regular_grid)


@dataclass
class Workload:
    name: str
    index: int
    shape: Tuple[int, ...]
    cells: np.ndarray          # [num_cells][2][d] int32 closed leaf boxes
    kernel: Kernel
    radius: int
    nrhs: int
    fft: int                   # padded FFT extent per axis used by the CUDA path
    precision: str             # "fp64" | "fp32"
    rhs_seed: int

    @property
    def ndim(self) -> int:
        return len(self.shape)

    @property
    def n(self) -> int:
        return int(np.prod(self.shape))


def fp64_64() -> Workload:
    L = 64

    def sigma(x):
        return 2.0 + np.sin(2 * math.pi * x[..., 0] / L) * np.cos(2 * math.pi * x[..., 1] / L)

    return Workload("fp64_64", 1, (L, L), regular_grid((L, L), (4, 4)),
                    GaussianIso(sigma, 12), 12, 1, 64, "fp64", 1000 + 0)


def fp32_512(nrhs: int = 64) -> Workload:
    L = 512
    shape = (L, L)
    s1 = SmoothField(shape, 2.0, 8.0, 2000 + 1)
    s2 = SmoothField(shape, 2.0, 8.0, 2000 + 2)
    th = SmoothField(shape, 0.0, math.pi, 2000 + 3)
    return Workload("fp32_512", 2, shape, regular_grid(shape, (16, 16)),
                    GaussianAniso2D(s1, s2, th, 24), 24, nrhs, 128, "fp32", 2000 + 0)


def adaptive_sigma(x, centre=(511.5, 511.5), rho=170.0, omega=4.0):
    d = np.sqrt((x[..., 0] - centre[0]) ** 2 + (x[..., 1] - centre[1]) ** 2)
    return 2.0 + 6.0 / (1.0 + np.exp(-(d - rho) / omega))


def adaptive_grad_sigma(x, centre=(511.5, 511.5), rho=170.0, omega=4.0):
    d = np.sqrt((x[..., 0] - centre[0]) ** 2 + (x[..., 1] - centre[1]) ** 2)
    s = 1.0 / (1.0 + np.exp(-(d - rho) / omega))
    return 6.0 * s * (1.0 - s) / omega


def adaptive_1024(nrhs: int = 32, shape: Tuple[int, int] = (1024, 1024)) -> Workload:
    def refine(lo, hi):
        g = np.stack(np.meshgrid(np.linspace(lo[0], hi[0], 5), np.linspace(lo[1], hi[1], 5),
                                 indexing="ij"), axis=-1)
        width = max(hi[0] - lo[0], hi[1] - lo[1])
        return bool(np.max(adaptive_grad_sigma(g)) * width > 0.05)

    cells = quadtree_grid(shape, 2, 7, refine)
    return Workload("adaptive_1024", 3, shape, cells, HeavyTailed(adaptive_sigma, 64), 64,
                    nrhs, 256, "fp32", 3000 + 0)


def fp32_128c(nrhs: int = 32) -> Workload:
    L = 128
    shape = (L, L, L)
    s = [SmoothField(shape, 1.5, 5.0, 4000 + 1 + i) for i in range(3)]
    return Workload("fp32_128c", 4, shape, regular_grid(shape, (8, 8, 8)),
                    GaussianAxis3D(s[0], s[1], s[2], 12), 12, nrhs, 64, "fp32", 4000 + 0)


BY_NAME = {
    "fp64_64": fp64_64,
    "fp32_512": fp32_512,
    "adaptive_1024": adaptive_1024,
    "fp32_128c": fp32_128c,
}


def get(name: str, **kw) -> Workload:
    return BY_NAME[name](**kw)
