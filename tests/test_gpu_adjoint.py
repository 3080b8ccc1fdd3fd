"""Adjoint apply (Eq. adjoint_random_z) through the C ABI against the FP64
oracle's adjoint on the same seeded inputs.  Tolerances as for the forward
apply: relative l2 per right-hand side 1e-10 (FP64 path), 1e-5 (FP32)."""
import numpy as np
import pytest

import workloads
from workloads import configs

from gpu_common import context, make_pair, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-10, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    context()


def run_adjoint(op, x_np):
    dt = torch.float64 if op.precision == "fp64" else torch.float32
    x = torch.from_numpy(np.ascontiguousarray(x_np)).to(device="cuda", dtype=dt)
    y = op.apply_adjoint(x)
    torch.cuda.synchronize()
    op.check()
    return y.cpu().numpy()


def run_forward(op, x_np):
    dt = torch.float64 if op.precision == "fp64" else torch.float32
    x = torch.from_numpy(np.ascontiguousarray(x_np)).to(device="cuda", dtype=dt)
    y = op.apply(x)
    torch.cuda.synchronize()
    op.check()
    return y.cpu().numpy()


def _aniso(shape, R):
    L = float(max(shape))
    return workloads.GaussianAniso2D(lambda x: 2.0 + 1.2 * np.sin(2 * np.pi * x[..., 0] / L),
                                     lambda x: 1.5 + 0.5 * np.cos(2 * np.pi * x[..., 1] / L),
                                     lambda x: 0.7 + 0.3 * x[..., 0] / L, R)


def test_adjoint_fp32_ragged_full():
    """Tiles of different extents, output boxes cut by the boundary, an odd
    batch (the last pair carries one right-hand side)."""
    shape = (97, 83)
    cells = workloads.regular_grid(shape, (5, 4))
    op, orc = make_pair(shape, cells, _aniso(shape, 9), "fp32")
    x = workloads.rhs(71, 3, shape)
    err = rel_l2(run_adjoint(op, x), orc.apply_adjoint(x))
    assert np.all(err <= TOL["fp32"]), err


def test_adjoint_fp64_workload_64():
    wl = configs.fp64_64()
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "fp64")
    x = workloads.rhs(wl.rhs_seed, 2, wl.shape).astype(np.float64)
    err = rel_l2(run_adjoint(op, x), orc.apply_adjoint(x))
    assert np.all(err <= TOL["fp64"]), err


def test_adjoint_identity_fp64():
    """<A~ x, y> = <x, A~* y> with both sides computed on the GPU."""
    wl = configs.fp64_64()
    op, _ = make_pair(wl.shape, wl.cells, wl.kernel, "fp64")
    rng = np.random.default_rng(72)
    x, y = rng.standard_normal((2,) + wl.shape), rng.standard_normal((2,) + wl.shape)
    ax, aty = run_forward(op, x), run_adjoint(op, y)
    lhs = np.sum((ax * y).reshape(2, -1), axis=1)
    rhs = np.sum((x * aty).reshape(2, -1), axis=1)
    scale = np.linalg.norm(ax.reshape(2, -1), axis=1) * np.linalg.norm(y.reshape(2, -1), axis=1)
    assert np.all(np.abs(lhs - rhs) <= 1e-12 * scale), (lhs, rhs)


def test_adjoint_hanging_nodes_and_split_windows():
    """A quadtree grid with hanging nodes and a kernel window cut into
    sub-windows (R = 50 at P = 128): every sub-window item adds into the same
    input box, which the colouring keeps ordered."""
    shape = (160, 144)
    cells = workloads.quadtree_grid(shape, 2, 4, lambda lo, hi: lo[0] < 70 and lo[1] < 60 and hi[0] - lo[0] > 20)
    kern = workloads.HeavyTailed(lambda x: 3.0 + 1.0 * np.sin(x[..., 0] / 30.0), 50)
    op, orc = make_pair(shape, cells, kern, "fp32")
    assert op.info()["num_tiles"] > orc.grid.r
    x = workloads.rhs(73, 2, shape)
    y = run_adjoint(op, x).reshape(2, -1)
    assert np.array_equal(y, run_adjoint(op, x).reshape(2, -1))   # fixed summation order
    pts = np.random.default_rng(74).choice(int(np.prod(shape)), 600, replace=False)
    ref = orc.apply_adjoint(x, points=pts)
    err = np.linalg.norm(y[:, pts] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.all(err <= TOL["fp32"]), err


def test_adjoint_workload_512_sampled():
    """The 512^2 benchmark operator at its full batch of 64 right-hand sides:
    every output of 2 right-hand sides and 512 seeded pixels of all 64."""
    wl = configs.fp32_512()
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "fp32")
    x = workloads.rhs(wl.rhs_seed, 64, wl.shape)
    y = run_adjoint(op, x).reshape(64, -1)
    pts = np.random.default_rng(75).choice(wl.n, 512, replace=False)
    ref = orc.apply_adjoint(x, points=pts)
    err = np.linalg.norm(y[:, pts] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.all(err <= TOL["fp32"]), err
    full = orc.apply_adjoint(x[[5, 38]]).reshape(2, -1)
    assert np.all(rel_l2(y[[5, 38]], full) <= TOL["fp32"])


def _skew3(shape, R):
    L = float(max(shape))
    return workloads.Skewed([0.7, -0.4, 0.3], lambda x: 1.1 + 0.4 * np.sin(2 * np.pi * x[..., 0] / L), R)


def test_adjoint_3d_fp32_ragged():
    """3D (P = 64): ragged tiles, output boxes cut by the boundary, an
    asymmetric kernel (an unflipped correlation would fail), an odd batch;
    bitwise reproducible."""
    shape = (37, 29, 33)
    op, orc = make_pair(shape, workloads.regular_grid(shape, (3, 3, 4)), _skew3(shape, 5), "fp32")
    x = workloads.rhs(76, 3, shape)
    y = run_adjoint(op, x)
    assert np.all(rel_l2(y, orc.apply_adjoint(x)) <= TOL["fp32"])
    assert np.array_equal(y, run_adjoint(op, x))


def test_adjoint_3d_identity():
    """<A~ x, y> = <x, A~* y> for 3D operators, both sides on the GPU (FP32)."""
    shape = (30, 26, 22)
    op, _ = make_pair(shape, workloads.regular_grid(shape, (3, 3, 3)), _skew3(shape, 4), "fp32")
    x, y = workloads.rhs(77, 2, shape), workloads.rhs(78, 2, shape)
    ax, aty = run_forward(op, x).astype(np.float64), run_adjoint(op, y).astype(np.float64)
    lhs = np.sum((ax * y).reshape(2, -1), axis=1)
    rhs = np.sum((x * aty).reshape(2, -1), axis=1)
    scale = np.linalg.norm(ax.reshape(2, -1), axis=1) * np.linalg.norm(y.reshape(2, -1), axis=1)
    assert np.all(np.abs(lhs - rhs) <= 1e-5 * scale), (lhs, rhs)


def test_adjoint_3d_workload_128_sampled():
    """The 128^3 operator at its benchmark batch of 32: 256 seeded voxels of
    every right-hand side against the oracle."""
    wl = configs.fp32_128c()
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "fp32")
    x = workloads.rhs(wl.rhs_seed, 32, wl.shape)
    y = run_adjoint(op, x).reshape(32, -1)
    pts = np.random.default_rng(79).choice(wl.n, 256, replace=False)
    ref = orc.apply_adjoint(x, points=pts)
    err = np.linalg.norm(y[:, pts] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.all(err <= TOL["fp32"]), err


def test_adjoint_bf16x3_workload_128_sampled():
    """The 128^3 operator in BF16x3 at its batch of 32, through the tensor-core
    adjoint (two chunks of the split path): 256 seeded voxels of every
    right-hand side against the oracle, within the BF16x3 bound."""
    wl = configs.fp32_128c()
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "bf16x3")
    x = workloads.rhs(wl.rhs_seed, 32, wl.shape)
    y = run_adjoint(op, x).reshape(32, -1)
    pts = np.random.default_rng(80).choice(wl.n, 256, replace=False)
    ref = orc.apply_adjoint(x, points=pts)
    err = np.linalg.norm(y[:, pts] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.all(err <= 1e-4), err


def test_adjoint_bf16x3():
    """BF16x3 operators: the first-axis correlation as split-BF16 tensor-core
    GEMMs (GEMM 1 over all first-axis planes of the output box, those outside
    Omega read as zero, the conjugate spectrum, GEMM 2 keeping the input-box
    planes).  Against the oracle's adjoint within the BF16x3 bound (1e-4 per
    right-hand side, the forward's; see test_gpu_tensor.py), against the FP32
    operator's adjoint, and the duality <A~ x, y> = <x, A~* y> to the same
    bound; odd batch, ragged tiles, output boxes cut by the boundary."""
    shape = (45, 29, 38)
    cells = workloads.regular_grid(shape, (4, 2, 3))
    kern = workloads.GaussianAxis3D(lambda x: 2.0 + 0.5 * np.cos(x[..., 1] / 6.0), lambda x: 1.5 + 0 * x[..., 0],
                                    lambda x: 1.2 + 0.2 * np.sin(x[..., 2] / 4.0), 9)
    op16, orc = make_pair(shape, cells, kern, "bf16x3")
    op32, _ = make_pair(shape, cells, kern, "fp32")
    x = workloads.rhs(76, 5, shape)
    z16 = run_adjoint(op16, x)
    ref = orc.apply_adjoint(x)
    err = rel_l2(z16, ref)
    assert np.all(err <= 1e-4), err
    assert np.all(rel_l2(z16, run_adjoint(op32, x)) <= 1e-4)
    # duality against the BF16x3 forward apply
    y = workloads.rhs(77, 5, shape)
    ax = run_forward(op16, x).reshape(5, -1).astype(np.float64)
    aty = run_adjoint(op16, y).reshape(5, -1).astype(np.float64)
    lhs = np.sum(ax * y.reshape(5, -1), axis=1)
    rhs_ = np.sum(x.reshape(5, -1) * aty, axis=1)
    scale = np.linalg.norm(ax, axis=1) * np.linalg.norm(y.reshape(5, -1), axis=1)
    assert np.all(np.abs(lhs - rhs_) <= 2e-4 * scale), (lhs, rhs_)
    # bitwise reproducible
    assert np.array_equal(run_adjoint(op16, x), z16)
