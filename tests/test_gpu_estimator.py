"""Randomized error estimator (Section 2.6, Eq. randomized_estimator_ec)
through the C ABI against the oracle.

The GPU forms Y~ = A~* Z with its adjoint apply and reduces every cell in
FP64.  For the same Z and Y the oracle's eta differs only through Y~:
|eta_gpu[C] - eta_orc[C]| <= ||Y~_gpu[C, .] - Y~_orc[C, .]|| / sqrt(q) (reverse
triangle inequality), which is the bound the FP32 tests assert per cell; the
FP64 path must reproduce the exact cell errors of the identity probes to
1e-9."""
import numpy as np
import pytest

import workloads
from workloads import configs
from oracle import Grid
from oracle.dense import dense_pc
from oracle.estimator import cell_point_indices, eta_from_adjoints, true_cell_errors

from gpu_common import context, make_pair

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    context()


def _dev(a, prec):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda",
                                                        dtype=torch.float64 if prec == "fp64" else torch.float32)


def _kernel(shape, R):
    L = float(max(shape))
    return workloads.Skewed([0.6, -0.3], lambda x: 1.0 + 0.5 * np.sin(2 * np.pi * x[..., 0] / L), R)


def test_identity_probes_give_exact_cell_errors_fp64():
    shape = (13, 11)
    cells = workloads.regular_grid(shape, (3, 3))
    kern = _kernel(shape, 3)
    op, orc = make_pair(shape, cells, kern, "fp64")
    A = workloads.dense_operator(shape, kern)
    N = A.shape[0]
    Z = np.sqrt(N) * np.eye(N)
    Y = Z @ A
    e = true_cell_errors(orc.grid, dense_pc(orc), A)
    eta = op.estimate_cell_errors(_dev(Z, "fp64"), _dev(Y, "fp64"), len(cells))
    torch.cuda.synchronize()
    op.check()
    assert np.max(np.abs(eta - e)) <= 1e-9 * e.max(), (eta, e)


def _assert_within_adjoint_bound(op, orc, Z, Y, eta):
    q = Z.shape[0]
    yt_gpu = op.apply_adjoint(_dev(Z, op.precision)).cpu().numpy().reshape(q, -1).astype(np.float64)
    yt_orc = orc.apply_adjoint(Z).reshape(q, -1)
    ref = eta_from_adjoints(orc.grid, yt_orc, Y)
    for c in range(len(orc.grid.cells)):
        idx = cell_point_indices(orc.grid, c)
        bound = np.linalg.norm(yt_gpu[:, idx] - yt_orc[:, idx]) / np.sqrt(q)
        assert abs(eta[c] - ref[c]) <= bound * (1 + 1e-6) + 1e-12 * ref.max(), (c, eta[c], ref[c], bound)
    return ref


def test_gaussian_probes_fp32_true_adjoint():
    """A 64 x 56 box, q = 8 Gaussian probes, Y = A* Z from the dense operator."""
    shape = (64, 56)
    cells = workloads.regular_grid(shape, (4, 4))
    kern = _kernel(shape, 6)
    op, orc = make_pair(shape, cells, kern, "fp32")
    A = workloads.dense_operator(shape, kern)
    Z = workloads.rhs(81, 8, shape).reshape(8, -1).astype(np.float64)   # FP32-rounded N(0,1)
    Y = (Z @ A).astype(np.float32).astype(np.float64)
    eta = op.estimate_cell_errors(_dev(Z, "fp32"), _dev(Y, "fp32"), len(cells))
    op.check()
    ref = _assert_within_adjoint_bound(op, orc, Z, Y, eta)
    assert np.all(ref > 0)
    # bitwise reproducible
    assert np.array_equal(eta, op.estimate_cell_errors(_dev(Z, "fp32"), _dev(Y, "fp32"), len(cells)))


def test_workload_512_cells():
    """The 512^2 benchmark operator (256 cells of ~35^2 points), q = 4."""
    wl = configs.fp32_512()
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "fp32")
    Z = workloads.rhs(82, 4, wl.shape).reshape(4, -1).astype(np.float64)
    Y = workloads.rhs(83, 4, wl.shape).reshape(4, -1).astype(np.float64)
    eta = op.estimate_cell_errors(_dev(Z, "fp32"), _dev(Y, "fp32"), len(wl.cells))
    op.check()
    assert eta.shape == (len(wl.cells),)
    _assert_within_adjoint_bound(op, orc, Z, Y, eta)


def test_estimator_3d_fp32():
    """3D cells (closed boxes, facet voxels in every cell holding them): the
    per-cell bound against the oracle on true A* Z."""
    shape = (14, 12, 10)
    cells = workloads.regular_grid(shape, (3, 3, 2))
    kern = workloads.Skewed([0.7, -0.4, 0.3], lambda x: 1.1 + 0.4 * np.sin(x[..., 0] / 5.0), 3)
    op, orc = make_pair(shape, cells, kern, "fp32")
    A = workloads.dense_operator(shape, kern)
    Z = workloads.rhs(85, 6, shape).reshape(6, -1).astype(np.float64)
    Y = (Z @ A).astype(np.float32).astype(np.float64)
    eta = op.estimate_cell_errors(_dev(Z, "fp32"), _dev(Y, "fp32"), len(cells))
    op.check()
    ref = _assert_within_adjoint_bound(op, orc, Z, Y, eta)
    assert np.all(ref > 0)


def test_estimator_bf16x3():
    """BF16x3 operators estimate through the tensor-core adjoint: the per-cell
    estimates equal the FP32 operator's to the BF16x3 bound."""
    shape = (24, 20, 18)
    cells = workloads.regular_grid(shape, (2, 2, 2))
    kern = workloads.GaussianAxis3D(lambda x: 1.5 + 0 * x[..., 0], lambda x: 1.2 + 0 * x[..., 0],
                                    lambda x: 1.0 + 0 * x[..., 0], 4)
    op16, _ = make_pair(shape, cells, kern, "bf16x3")
    op32, _ = make_pair(shape, cells, kern, "fp32")
    A = workloads.dense_operator(shape, kern)
    Z = workloads.rhs(84, 6, shape).reshape(6, -1).astype(np.float64)
    Y = (Z @ A).astype(np.float32).astype(np.float64)
    eta16 = op16.estimate_cell_errors(_dev(Z, "fp32"), _dev(Y, "fp32"), len(cells))
    op16.check()
    eta32 = op32.estimate_cell_errors(_dev(Z, "fp32"), _dev(Y, "fp32"), len(cells))
    op32.check()
    # |eta16[C] - eta32[C]| <= ||(Y~16 - Y~32)[C, .]|| / sqrt(q) (reverse
    # triangle inequality), and each Y~ is within 1e-4 of A~* Z per column
    yt = np.linalg.norm(Z @ A)
    assert np.all(np.abs(np.asarray(eta16) - np.asarray(eta32)) <= 2e-4 * yt / np.sqrt(6)), (eta16, eta32)
