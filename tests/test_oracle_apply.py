"""Oracle apply against what the paper and the mathematics fix.

* hand-worked 1D matrix (tests/golden/hand_1d_5pt.txt),
* entry formula (Eq. conv_matrix_entries) vs direct summation,
* exactness at sample points: A~ e_{p_k} = A e_{p_k},
* a translation-invariant operator (restricted convolution) is reproduced
  exactly, boundaries included, checked against scipy.signal's convolution,
  while extension by zero leaves an O(1) boundary artifact (Fig. 1d_conv),
* A~ = A when every point is a sample point,
* Proposition 4.3 (W_k partition of unity on Omega x Omega, supp W_k in
  mu_k^E, A~ = sum_k W_k phi_k), Proposition 4.4 and Theorem 4.5,
* planted mistakes (a flipped index, a transposed operand, a dropped
  extension) are caught by these pins.
"""
import numpy as np
import pytest
from scipy import signal

import workloads
from oracle import Grid, PCOracle
from oracle.dense import dense_F, dense_pc, dense_W

from test_oracle_geometry import ADAPTIVE_CELLS, ADAPTIVE_SHAPE


def _const(v):
    return lambda x: v + 0.0 * x[..., 0]


def _varying(shape):
    L = float(max(shape))
    return lambda x: 1.2 + 0.6 * np.sin(2 * np.pi * x[..., 0] / L) * np.cos(np.pi * x[..., -1] / L)


def _oracle(shape, cells, kernel, extend=True):
    g = Grid(shape, cells)
    phi = workloads.impulse_windows(shape, g.points, kernel)
    return PCOracle(shape, cells, phi, kernel.radius, extend=extend)


CASES = [
    ("1d", (23,), workloads.regular_grid((23,), (4,))),
    ("2d", (14, 17), workloads.regular_grid((14, 17), (3, 4))),
    ("2d-adaptive", ADAPTIVE_SHAPE, np.array(ADAPTIVE_CELLS)),
    ("3d", (7, 8, 6), workloads.regular_grid((7, 8, 6), (3, 3, 2))),
]


def _skew(d, R, sigma):
    mu = [0.7, -0.4, 0.3][:d]
    return workloads.Skewed(mu, sigma, R)


# ------------------------------------------------------------------ golden

def test_hand_worked_1d_matrix(golden):
    g5 = golden("hand_1d_5pt.txt")
    A, At = g5["A"], g5["Atilde"]
    cells = np.array([[[0], [2]], [[2], [4]]])
    g = Grid((5,), cells)
    phi = workloads.impulse_windows_from_matrix((5,), g.points, 1, A)
    orc = PCOracle((5,), cells, phi, 1)
    # the weights come out of a Laplace solve, so allow rounding
    assert np.max(np.abs(dense_pc(orc) - At)) < 1e-13
    assert np.max(np.abs(orc.apply(np.eye(5)).T - At)) < 1e-13


# ------------------------------------------------------------------ entries vs direct sum

@pytest.mark.parametrize("name,shape,cells", CASES)
def test_entry_formula_matches_direct_sum(name, shape, cells):
    orc = _oracle(shape, cells, _skew(len(shape), 3, _varying(shape)))
    N = int(np.prod(shape))
    D = dense_pc(orc)
    f = np.random.default_rng(1).standard_normal((3, N))
    y = orc.apply(f).reshape(3, N)
    assert np.max(np.abs(y - f @ D.T)) < 1e-13 * max(1.0, np.abs(y).max())
    # sampled outputs equal the full apply bit for bit; thread count is irrelevant
    pts = np.random.default_rng(2).choice(N, 17, replace=False)
    assert np.array_equal(orc.apply(f, points=pts), y[:, pts])
    assert np.array_equal(orc.apply(f, nthreads=1).reshape(3, N), y)


# ------------------------------------------------------------------ exact at sample points

@pytest.mark.parametrize("name,shape,cells", CASES)
def test_exact_at_sample_points(name, shape, cells):
    kern = _skew(len(shape), 3, _varying(shape))
    orc = _oracle(shape, cells, kern)
    A = workloads.dense_operator(shape, kern)
    N = int(np.prod(shape))
    strides = np.array([int(np.prod(shape[a + 1:])) for a in range(len(shape))])
    for k in range(orc.grid.r):
        e = np.zeros(N)
        e[int(orc.grid.points[k] @ strides)] = 1.0
        col = orc.apply(e[None]).ravel()
        assert np.max(np.abs(col - A[:, int(orc.grid.points[k] @ strides)])) < 1e-15


# ------------------------------------------------------------------ translation invariance

def _restricted_convolution(f, psi, R):
    """Textbook: extend f by zero, convolve with psi on [-R,R]^d, restrict to Omega."""
    full = signal.convolve(f, psi, mode="full", method="direct")
    sl = tuple(slice(R, R + n) for n in f.shape)
    return full[sl]


@pytest.mark.parametrize("name,shape,cells", CASES)
def test_translation_invariant_operator_is_reproduced(name, shape, cells):
    R = 3
    d = len(shape)
    kern = _skew(d, R, _const(1.1))
    orc = _oracle(shape, cells, kern)
    psi = workloads.impulse_windows((2 * R + 1,) * d, np.array([[R] * d]), kern).reshape((2 * R + 1,) * d)
    f = np.random.default_rng(4).standard_normal(shape)
    y = orc.apply(f[None])[0]
    ref = _restricted_convolution(f, psi, R)
    assert np.max(np.abs(y - ref)) < 1e-13 * np.abs(ref).max()
    # same operator with zero extension: boundary artifacts (Fig. 1d_conv)
    y0 = _oracle(shape, cells, kern, extend=False).apply(f[None])[0]
    assert np.max(np.abs(y0 - ref)) > 1e-2 * np.abs(ref).max()


def test_figure_1d_conv_setup_two_end_points():
    """1D: a convolution operator on [1, N], two sample points at the ends."""
    N, R = 40, 6
    kern1d = workloads.Skewed([0.0], _const(2.0), R)
    cells = np.array([[[0], [N - 1]]])
    A = workloads.dense_operator((N,), kern1d)
    orc = _oracle((N,), cells, kern1d)
    assert np.max(np.abs(dense_pc(orc) - A)) < 1e-13
    orc0 = _oracle((N,), cells, kern1d, extend=False)
    assert np.max(np.abs(dense_pc(orc0) - A)) > 0.1 * np.abs(A).max()


def test_all_points_sampled_gives_A():
    shape = (6, 7)
    cells = [[[i, j], [i + 1, j + 1]] for i in range(5) for j in range(6)]
    kern = workloads.GaussianAniso2D(_const(1.3), _varying(shape), _varying(shape), 3)
    orc = _oracle(shape, np.array(cells), kern)
    A = workloads.dense_operator(shape, kern)
    assert orc.grid.r == 42
    assert np.max(np.abs(dense_pc(orc) - A)) < 1e-14


# ------------------------------------------------------------------ Section 4

THEORY_CASES = [
    ("2d", (9, 11), workloads.regular_grid((9, 11), (3, 3))),
    ("2d-adaptive", (13, 9), np.array([[[0, 0], [4, 8]], [[4, 0], [8, 4]], [[4, 4], [8, 8]],
                                         [[8, 0], [12, 8]]])),
    ("1d", (17,), workloads.regular_grid((17,), (4,))),
]


@pytest.mark.parametrize("name,shape,cells", THEORY_CASES)
def test_proposition_4_3_4_4_theorem_4_5(name, shape, cells):
    R = 3
    sig = lambda x: 0.9 + 0.5 * np.sin(0.7 * x[..., 0]) + 0.3 * np.cos(0.5 * x[..., -1])  # noqa: E731
    kern = _skew(len(shape), R, sig)
    orc = _oracle(shape, cells, kern)
    g = orc.grid
    A = workloads.dense_operator(shape, kern)
    At = dense_pc(orc)
    W = dense_W(orc)
    Fk, F, mu = dense_F(g, A)
    # 4.3(2): partition of unity on Omega x Omega
    assert np.max(np.abs(W.sum(axis=0) - 1.0)) < 1e-14
    # 4.3(3): supp W_k in mu_k^E
    assert np.all(W[~mu] == 0.0)
    # 4.3(1): A~[y,x] = sum_k W_k[y,x] phi_k[y-x]; phi_k[y-x] = A[y-x+p_k, p_k] on mu_k^E
    phik = Fk + np.where(mu, A[None], 0.0)
    assert np.max(np.abs(At - np.sum(W * phik, axis=0))) < 1e-14
    # 4.4: A~ - A = sum_k W_k F_k
    assert np.max(np.abs((At - A) - np.sum(W * Fk, axis=0))) < 1e-14
    # 4.5: pointwise and Frobenius bounds
    assert np.all(np.abs(At - A) <= F + 1e-14)
    assert np.linalg.norm(At - A) <= np.linalg.norm(F) + 1e-14
    assert np.linalg.norm(At - A) > 0  # varying kernel: a non-trivial case


# ------------------------------------------------------------------ planted mistakes

def test_planted_mistakes_are_caught():
    """Each plausible slip changes the oracle enough for a pin above to fail."""
    shape, cells = (14, 17), workloads.regular_grid((14, 17), (3, 4))
    R = 3
    kern = _skew(2, R, _const(1.1))
    orc = _oracle(shape, cells, kern)
    psi = workloads.impulse_windows((7, 7), np.array([[R, R]]), kern).reshape(7, 7)
    f = np.random.default_rng(4).standard_normal(shape)
    ref = _restricted_convolution(f, psi, R)
    scale = np.abs(ref).max()
    assert np.max(np.abs(orc.apply(f[None])[0] - ref)) < 1e-13 * scale
    # flipped convolution index: phi^E[x - y] instead of phi^E[y - x]
    flipped = PCOracle(shape, cells, orc.phi, R)
    flipped.phiE = orc.phiE.reshape(-1, 7, 7)[:, ::-1, ::-1].reshape(orc.grid.r, -1).copy()
    assert np.max(np.abs(flipped.apply(f[None])[0] - ref)) > 1e-2 * scale
    # transposed operand: f^T fed on a square box
    sq_shape, sq_cells = (15, 15), workloads.regular_grid((15, 15), (3, 4))
    sq = _oracle(sq_shape, sq_cells, kern)
    g = np.random.default_rng(5).standard_normal(sq_shape)
    ref_sq = _restricted_convolution(g, psi, R)
    assert np.max(np.abs(sq.apply(g.T[None])[0] - ref_sq)) > 1e-2 * np.abs(ref_sq).max()
    # dropped extension
    assert np.max(np.abs(_oracle(shape, cells, kern, extend=False).apply(f[None])[0] - ref)) > 1e-2 * scale
    # weights that miss one hat (not a partition of unity) break exactness
    bad = PCOracle(shape, cells, orc.phi, R, weights=[w * (0.5 if k == 3 else 1.0) for k, w in enumerate(orc.W)])
    assert np.max(np.abs(bad.apply(f[None])[0] - ref)) > 1e-3 * scale
