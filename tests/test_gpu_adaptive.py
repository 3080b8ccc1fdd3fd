"""Adaptive construction (Algorithm 1) on the library against the oracle's
independent implementation, and a qualitative reproduction of the blur
experiment of Section 5.1 on a synthetic ring.

With FP64 operators the library's estimates agree with the oracle's to
about 1e-12, so both sides take the same refinement decisions (which cell,
which direction) and must end with the identical leaf cells."""
import numpy as np
import pytest

import workloads
from oracle import Grid, PCOracle
from oracle.adaptive import construct as oracle_construct

from gpu_common import context

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    context()


def _aniso(shape):
    L = float(shape[0])
    return workloads.GaussianAniso2D(lambda x: 1.0 + 1.5 * x[..., 0] / L, lambda x: 1.2 + 0.8 * x[..., 1] / L,
                                     lambda x: 0.3 + 0 * x[..., 0], 5)


def _canon(cells):
    return sorted(tuple(int(v) for v in np.asarray(c).ravel()) for c in cells)


@pytest.mark.parametrize("batch", [1, 3])
def test_same_refinement_as_the_oracle_fp64(batch):
    from paper_1805_06018_gb300 import adaptive
    shape = (40, 36)
    kern = _aniso(shape)
    A = workloads.dense_operator(shape, kern)
    Z = np.random.default_rng(21).standard_normal((6, int(np.prod(shape))))
    Y = Z @ A
    impulse = lambda pts: workloads.impulse_windows(shape, pts, kern)  # noqa: E731
    tau = 0.03
    cells_o, hist_o = oracle_construct(shape, impulse, 5, Z, Y, tau=tau, max_passes=40, batch=batch)
    zt = torch.from_numpy(Z.reshape((6,) + shape)).cuda()
    yt = torch.from_numpy(Y.reshape((6,) + shape)).cuda()
    op, cells_l, hist_l = adaptive.construct(context(), shape, impulse, 5, zt, yt, tau=tau, precision="fp64",
                                             max_passes=40, batch=batch)
    assert _canon(cells_l) == _canon(cells_o)
    assert len(hist_l) == len(hist_o) > 2
    for (rl, el), (ro, eo) in zip(hist_l, hist_o):
        assert rl == ro and abs(el - eo) <= 1e-9 * eo
    assert hist_l[-1][1] <= tau


def test_ring_blur_refines_near_the_ring():
    """Section 5.1, qualitatively: the blur width jumps across a circle; the
    construction refines along the circle, stops at tau, and the true
    relative error (dense matrices) is of the estimated size."""
    from paper_1805_06018_gb300 import adaptive
    shape = (64, 64)
    c, rho, omega = 31.5, 18.0, 1.5

    def sigma(x):
        d = np.sqrt((x[..., 0] - c) ** 2 + (x[..., 1] - c) ** 2)
        return 1.0 + 2.0 / (1.0 + np.exp(-(d - rho) / omega))

    kern = workloads.HeavyTailed(sigma, 8)
    A = workloads.dense_operator(shape, kern)
    q = 6
    Z = workloads.rhs(31, q, shape).reshape(q, -1).astype(np.float64)
    Y = (Z @ A).astype(np.float32)
    impulse = lambda pts: workloads.impulse_windows(shape, pts, kern)  # noqa: E731
    tau = 0.05
    op, cells, hist = adaptive.construct(context(), shape, impulse, 8, torch.from_numpy(Z.astype(np.float32).reshape(
        (q,) + shape)).cuda(), torch.from_numpy(Y.reshape((q,) + shape)).cuda(), tau=tau, precision="fp32",
        max_passes=40, batch=4)
    assert hist[-1][1] <= tau < hist[0][1]
    # leaves crossing the ring are smaller than the others
    area = np.array([np.prod(cc[1] - cc[0] + 1) for cc in cells])
    corners = [[(cc[0][0], cc[0][1]), (cc[0][0], cc[1][1]), (cc[1][0], cc[0][1]), (cc[1][0], cc[1][1])] for cc in cells]
    dist = [np.array([np.hypot(a - c, b - c) for a, b in cs]) for cs in corners]
    crossing = np.array([dd.min() <= rho + 2 * omega and dd.max() >= rho - 2 * omega for dd in dist])
    assert crossing.any() and (~crossing).any()
    assert area[crossing].mean() < area[~crossing].mean()
    # true relative Frobenius error of the result: every entry of A~ from
    # pc_entries (Eq. conv_matrix_entries) against the dense operator
    N = int(np.prod(shape))
    rows = torch.arange(N, device="cuda").repeat_interleave(N)
    cols = torch.arange(N, device="cuda").repeat(N)
    At = op.entries(rows, cols).cpu().numpy().reshape(N, N)
    true_err = np.linalg.norm(At - A) / np.linalg.norm(A)
    assert true_err < 3 * tau
    # spot-check those entries against the oracle's direct sum on the same leaves
    g = Grid(shape, cells)
    orc = PCOracle(shape, cells, workloads.impulse_windows(shape, g.points, kern), 8)
    pick = np.random.default_rng(32).choice(N, 5, replace=False)
    for x in pick:
        e = np.zeros(N)
        e[x] = 1.0
        col = orc.apply(e[None]).ravel()
        assert np.max(np.abs(At[:, x] - col)) <= 1e-6 * np.abs(col).max()


def test_3d_construction():
    """Algorithm 1 in 3D (hanging nodes from the second split on), FP32: every
    split follows the axis of change, the estimate reaches tau, and the final
    leaves' estimates agree with the oracle's on the same leaves."""
    from paper_1805_06018_gb300 import adaptive
    from oracle.estimator import eta_from_adjoints
    shape = (11, 12, 17)
    L = 17.0
    kern = workloads.GaussianAxis3D(lambda x: 1.0 + 0 * x[..., 0], lambda x: 1.0 + 0 * x[..., 0],
                                    lambda x: 0.8 + 1.6 * x[..., 2] / L, 3)
    A = workloads.dense_operator(shape, kern)
    q = 4
    Z = workloads.rhs(33, q, shape).reshape(q, -1).astype(np.float64)
    Y = (Z @ A).astype(np.float32)
    impulse = lambda pts: workloads.impulse_windows(shape, pts, kern)  # noqa: E731
    op, cells, hist = adaptive.construct(context(), shape, impulse, 3,
                                         torch.from_numpy(Z.astype(np.float32).reshape((q,) + shape)).cuda(),
                                         torch.from_numpy(Y.reshape((q,) + shape)).cuda(), tau=0.06,
                                         precision="fp32", max_passes=12, batch=2)
    assert hist[-1][1] <= 0.06 < hist[0][1] and len(cells) > 8
    for lo, hi in cells:
        assert (lo[0], hi[0]) in ((0, 5), (5, 10)) and (lo[1], hi[1]) in ((0, 5), (5, 11))
    g = Grid(shape, cells)
    orc = PCOracle(shape, cells, workloads.impulse_windows(shape, g.points, kern), 3)
    ref = eta_from_adjoints(g, orc.apply_adjoint(Z.reshape((q,) + shape)), Y.astype(np.float64).reshape(q, -1))
    eta = op.estimate_cell_errors(torch.from_numpy(Z.astype(np.float32).reshape((q,) + shape)).cuda(),
                                  torch.from_numpy(Y.reshape((q,) + shape)).cuda(), len(cells))
    assert np.max(np.abs(eta - ref)) <= 1e-4 * ref.max()
