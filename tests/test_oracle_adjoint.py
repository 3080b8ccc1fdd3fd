"""Oracle adjoint apply (Eq. adjoint_random_z) against what the paper and the
mathematics fix.

* it is the adjoint of the pinned forward apply: <A~ x, y> = <x, A~* y> on
  regular, adaptive (hanging-node) and 3D grids, and the dense matrix of
  A~* is the transpose of the dense A~ (entries, Eq. conv_matrix_entries);
* a translation-invariant (deliberately asymmetric) operator: A~* is the
  restricted correlation with the kernel, checked against scipy.signal;
* the weight multiplies after the correlation (w_k . (flip(phi) * f), not
  flip(phi) * (w_k . f)), and planted mistakes (unflipped kernel, weight on
  the wrong side, dropped extension) fail these pins.
"""
import numpy as np
import pytest
from scipy import signal

import workloads
from oracle import Grid, PCOracle
from oracle.dense import dense_pc

from test_oracle_geometry import ADAPTIVE_CELLS, ADAPTIVE_SHAPE

CASES = [
    ("1d", (23,), workloads.regular_grid((23,), (4,))),
    ("2d", (14, 17), workloads.regular_grid((14, 17), (3, 4))),
    ("2d-adaptive", ADAPTIVE_SHAPE, np.array(ADAPTIVE_CELLS)),
    ("3d", (7, 8, 6), workloads.regular_grid((7, 8, 6), (3, 3, 2))),
]


def _varying(shape):
    L = float(max(shape))
    return lambda x: 1.2 + 0.6 * np.sin(2 * np.pi * x[..., 0] / L) * np.cos(np.pi * x[..., -1] / L)


def _skew(d, R, sigma):
    return workloads.Skewed([0.7, -0.4, 0.3][:d], sigma, R)


def _oracle(shape, cells, kernel, extend=True):
    g = Grid(shape, cells)
    return PCOracle(shape, cells, workloads.impulse_windows(shape, g.points, kernel), kernel.radius, extend=extend)


@pytest.mark.parametrize("name,shape,cells", CASES)
def test_adjoint_identity(name, shape, cells):
    orc = _oracle(shape, cells, _skew(len(shape), 3, _varying(shape)))
    N = int(np.prod(shape))
    rng = np.random.default_rng(7)
    x, y = rng.standard_normal((2, N)), rng.standard_normal((2, N))
    ax = orc.apply(x).reshape(2, N)
    aty = orc.apply_adjoint(y).reshape(2, N)
    lhs, rhs = np.sum(ax * y, axis=1), np.sum(x * aty, axis=1)
    scale = np.linalg.norm(ax, axis=1) * np.linalg.norm(y, axis=1)
    assert np.all(np.abs(lhs - rhs) <= 1e-13 * scale), (lhs, rhs)


@pytest.mark.parametrize("name,shape,cells", CASES[:3])
def test_adjoint_matrix_is_the_transpose(name, shape, cells):
    orc = _oracle(shape, cells, _skew(len(shape), 3, _varying(shape)))
    N = int(np.prod(shape))
    D = dense_pc(orc)                       # entries of A~ from Eq. conv_matrix_entries
    At = orc.apply_adjoint(np.eye(N)).reshape(N, N).T   # column j = A~* e_j
    assert np.max(np.abs(At - D.T)) < 1e-13 * np.abs(D).max()
    # sampled outputs equal the full apply bit for bit
    f = np.random.default_rng(8).standard_normal((3, N))
    full = orc.apply_adjoint(f).reshape(3, N)
    pts = np.random.default_rng(9).choice(N, 11, replace=False)
    assert np.array_equal(orc.apply_adjoint(f, points=pts), full[:, pts])
    assert np.array_equal(orc.apply_adjoint(f, nthreads=1).reshape(3, N), full)


def _restricted_correlation(f, psi, R):
    """Textbook: (psi correlated with f)[x] = sum_z psi[z] f[x + z], f zero outside Omega."""
    full = signal.correlate(f, psi, mode="full", method="direct")
    sl = tuple(slice(R, R + n) for n in f.shape)
    return full[sl]


@pytest.mark.parametrize("name,shape,cells", CASES)
def test_translation_invariant_adjoint_is_correlation(name, shape, cells):
    R = 3
    d = len(shape)
    kern = _skew(d, R, lambda x: 1.1 + 0.0 * x[..., 0])
    orc = _oracle(shape, cells, kern)
    psi = workloads.impulse_windows((2 * R + 1,) * d, np.array([[R] * d]), kern).reshape((2 * R + 1,) * d)
    f = np.random.default_rng(10).standard_normal(shape)
    y = orc.apply_adjoint(f[None])[0]
    ref = _restricted_correlation(f, psi, R)
    assert np.max(np.abs(y - ref)) < 1e-13 * np.abs(ref).max()


def test_planted_adjoint_mistakes_are_caught():
    shape, cells = (14, 17), workloads.regular_grid((14, 17), (3, 4))
    R = 3
    orc = _oracle(shape, cells, _skew(2, R, _varying(shape)))
    N = int(np.prod(shape))
    rng = np.random.default_rng(11)
    x, y = rng.standard_normal((1, N)), rng.standard_normal((1, N))
    ax = orc.apply(x).ravel()
    good = float(np.dot(ax, y.ravel()))
    scale = np.linalg.norm(ax) * np.linalg.norm(y)

    def gap(aty):
        return abs(good - float(np.dot(x.ravel(), np.asarray(aty).ravel()))) / scale

    assert gap(orc.apply_adjoint(y)) < 1e-13
    flipped = PCOracle(shape, cells, orc.phi, R)
    flipped.phiE = orc.phiE.reshape(-1, 7, 7)[:, ::-1, ::-1].reshape(orc.grid.r, -1).copy()
    # unflipped kernel: w_k . (phi_k * f), a convolution instead of a correlation
    assert gap(flipped.apply_adjoint(y)) > 1e-3
    # weight on the wrong side: flip(phi_k) * (w_k . f), which is the forward
    # sum with the flipped kernel
    assert gap(flipped.apply(y)) > 1e-3
    # dropped extension (a different operator, so not the adjoint of A~)
    assert gap(_oracle(shape, cells, _skew(2, R, _varying(shape)), extend=False).apply_adjoint(y)) > 1e-3
    # and A~ is not symmetric here, so the forward apply is no stand-in
    assert gap(orc.apply(y)) > 1e-3
