"""Oracle randomized error estimator (Section 2.6) against what the
mathematics fixes.

* with the deterministic probe matrix Z = sqrt(N) I (q = N), the estimator is
  exact: eta_C = e_C = ||(A~ - A)[Omega, C]||_F, with A~ from the entry
  formula and A the dense operator (independent constructions);
* eta_C = 0 for every cell when every point is a sample point (A~ = A);
* with Gaussian probes the squared estimator is unbiased (Eq. saa_XZ): over
  many probes it approaches e_C^2;
* planted mistakes (a missing 1/q, cells taken as half-open boxes) are caught.
"""
import numpy as np

import workloads
from oracle import Grid, PCOracle
from oracle.dense import dense_pc
from oracle.estimator import cell_point_indices, eta, eta_from_adjoints, true_cell_errors


def _setup(shape=(13, 11), n=(3, 3), R=3):
    cells = workloads.regular_grid(shape, n)
    L = float(max(shape))
    kern = workloads.Skewed([0.6, -0.3], lambda x: 1.0 + 0.5 * np.sin(2 * np.pi * x[..., 0] / L), R)
    g = Grid(shape, cells)
    orc = PCOracle(shape, cells, workloads.impulse_windows(shape, g.points, kern), R)
    A = workloads.dense_operator(shape, kern)
    return orc, A


def test_identity_probes_give_the_exact_cell_errors():
    orc, A = _setup()
    N = A.shape[0]
    Z = np.sqrt(N) * np.eye(N)
    Y = Z @ A   # row i = (A* zeta_i)^T, zeta_i = sqrt(N) e_i
    e = true_cell_errors(orc.grid, dense_pc(orc), A)
    got = eta(orc, Z, Y)
    assert np.all(e > 1e-6)
    assert np.max(np.abs(got - e)) < 1e-12 * e.max()


def test_zero_when_every_point_is_sampled():
    shape = (6, 5)
    cells = np.array([[[i, j], [i + 1, j + 1]] for i in range(5) for j in range(4)])
    kern = workloads.Skewed([0.6, -0.3], lambda x: 1.0 + 0.2 * x[..., 0], 2)
    g = Grid(shape, cells)
    orc = PCOracle(shape, cells, workloads.impulse_windows(shape, g.points, kern), 2)
    A = workloads.dense_operator(shape, kern)
    Z = np.random.default_rng(1).standard_normal((5, 30))
    assert np.max(eta(orc, Z, Z @ A)) < 1e-12 * np.abs(Z @ A).max()


def test_gaussian_probes_are_unbiased():
    orc, A = _setup()
    N = A.shape[0]
    e = true_cell_errors(orc.grid, dense_pc(orc), A)
    Z = np.random.default_rng(2).standard_normal((4000, N))
    got = eta(orc, Z, Z @ A)
    # E[eta_C^2] = e_C^2; with 4000 probes the relative spread of eta^2 is a few %
    assert np.all(np.abs(got ** 2 / e ** 2 - 1.0) < 0.15), got ** 2 / e ** 2


def test_planted_estimator_mistakes_are_caught():
    orc, A = _setup()
    N = A.shape[0]
    Z = np.sqrt(N) * np.eye(N)
    Y = Z @ A
    e = true_cell_errors(orc.grid, dense_pc(orc), A)
    Yt = orc.apply_adjoint(Z).reshape(N, N)
    # missing 1/q
    d = Yt - Y
    no_q = np.array([np.sqrt(np.sum(d[:, cell_point_indices(orc.grid, c)] ** 2)) for c in range(len(orc.grid.cells))])
    assert np.max(np.abs(no_q - e)) > 0.5 * e.max()
    # cells as half-open boxes (shared facets dropped)
    half = []
    for c in range(len(orc.grid.cells)):
        lo, hi = orc.grid.cells[c]
        idx = np.ravel_multi_index(np.meshgrid(*[np.arange(a, b) for a, b in zip(lo, hi)], indexing="ij"),
                                   orc.grid.shape).ravel()
        half.append(np.sqrt(np.sum(d[:, idx] ** 2) / N))
    assert np.max(np.abs(np.array(half) - e)) > 1e-3 * e.max()
    # and the forward operator in place of the adjoint
    fwd = eta_from_adjoints(orc.grid, orc.apply(Z), Y)
    assert np.max(np.abs(fwd - e)) > 1e-3 * e.max()
