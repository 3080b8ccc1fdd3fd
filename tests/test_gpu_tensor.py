"""Tensor-core (BF16x3) 3D path through the C ABI against the FP64 oracle.

The first-axis DFTs of every 64^3 patch run as tcgen05 GEMMs with split BF16
operands (a = a_hi + a_lo, products a_lo b_hi + a_hi b_lo + a_hi b_hi in FP32).
Each split operand carries a relative error of at most 2^-18 and the dropped
a_lo b_lo term is at most 2^-18 of |a b|, so a product is good to about
3 * 2^-18 = 1.1e-5; the stated bound for the whole apply is a relative l2
error of 1e-4 per right-hand side."""
import numpy as np
import pytest

import workloads
from workloads import configs

from gpu_common import context, make_pair, rel_l2, run

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL_BF16X3 = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    context()


def _small_kernel():
    s = lambda x: 1.2 + 0.3 * np.sin(x[..., 0] / 7.0)  # noqa: E731
    return workloads.GaussianAxis3D(s, lambda x: 1.6 + 0 * x[..., 0], lambda x: 1.0 + 0.2 * np.cos(x[..., 2] / 5.0), 5)


def test_bf16x3_3d_small_full():
    shape = (40, 36, 30)
    cells = workloads.regular_grid(shape, (3, 3, 3))
    op, orc = make_pair(shape, cells, _small_kernel(), "bf16x3")
    assert op.info()["precision"] == 2
    x = workloads.rhs(61, 3, shape)
    y = run(op, x)
    err = rel_l2(y, orc.apply(x))
    assert np.all(err <= TOL_BF16X3), err
    # the stages were timed on the caller's stream
    assert all(op.stage_ms(s) > 0 for s in range(3))
    assert op.launches() == 4   # zero-fill + one chunk of three kernels


def test_bf16x3_3d_ragged_odd_batch():
    """Odd batch (the last pair carries one right-hand side), tiles of
    different extents along every axis, a large kernel window (R = 9)."""
    shape = (45, 29, 38)
    cells = workloads.regular_grid(shape, (4, 2, 3))
    kern = workloads.GaussianAxis3D(lambda x: 2.0 + 0.5 * np.cos(x[..., 1] / 6.0), lambda x: 1.5 + 0 * x[..., 0],
                                    lambda x: 1.2 + 0.2 * np.sin(x[..., 2] / 4.0), 9)
    op, orc = make_pair(shape, cells, kern, "bf16x3")
    x = workloads.rhs(63, 5, shape)
    err = rel_l2(run(op, x), orc.apply(x))
    assert np.all(err <= TOL_BF16X3), err


def test_bf16x3_3d_matches_fp32_path():
    """Same operator built in FP32 (all FFTs on CUDA cores) and BF16x3: the two
    differ by the tensor-core rounding only."""
    shape = (40, 36, 30)
    cells = workloads.regular_grid(shape, (3, 3, 3))
    kern = _small_kernel()
    op32, orc = make_pair(shape, cells, kern, "fp32")
    op16, _ = make_pair(shape, cells, kern, "bf16x3")
    x = workloads.rhs(64, 4, shape)
    y32, y16 = run(op32, x), run(op16, x)
    ref = orc.apply(x)
    e32, e16 = rel_l2(y32, ref), rel_l2(y16, ref)
    assert np.all(e32 <= 1e-5), e32
    assert np.all(e16 <= TOL_BF16X3), e16
    assert np.all(rel_l2(y16, y32) <= TOL_BF16X3)


def test_bf16x3_3d_chunks_deterministic():
    """A batch with more work items than one chunk (27 tiles x 152 pairs = 4104
    > 4096) runs as two chunks; every right-hand side is bit-identical to the
    same right-hand side applied in a small batch (the overlap-add order does
    not depend on the chunking), and a sample matches the oracle."""
    shape = (40, 36, 30)
    cells = workloads.regular_grid(shape, (3, 3, 3))
    op, orc = make_pair(shape, cells, _small_kernel(), "bf16x3")
    assert op.info()["num_tiles"] == 27
    x = workloads.rhs(65, 304, shape)
    y_big = run(op, x)
    assert op.launches() == 1 + 3 * 2
    y_small = run(op, x[:6])
    assert np.array_equal(y_big[:6], y_small)
    y_tail = run(op, x[-4:])
    assert np.array_equal(y_big[-4:], y_tail)
    err = rel_l2(y_big[[0, 151, 303]], orc.apply(x[[0, 151, 303]]))
    assert np.all(err <= TOL_BF16X3), err


def test_bf16x3_3d_workload_128_sampled():
    """The 128^3 workload (8x8x8 regular grid, anisotropic 3D Gaussian, R = 12)
    at its full batch of 32 right-hand sides: 1024 seeded voxels of every
    right-hand side against the oracle."""
    wl = configs.fp32_128c(32)
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "bf16x3")
    x = workloads.rhs(wl.rhs_seed, 32, wl.shape)
    y = run(op, x).reshape(32, -1)
    pts = np.random.default_rng(12).choice(wl.n, 1024, replace=False)
    ref = orc.apply(x, points=pts)
    err = np.linalg.norm(y[:, pts] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.all(err <= TOL_BF16X3), err


def test_bf16x3_unsupported_forms():
    import paper_1805_06018_gb300 as pcg
    from paper_1805_06018_gb300.binding import PC_ERR_NOT_READY, PC_ERR_UNSUPPORTED
    shape = (48, 40)
    cells = workloads.regular_grid(shape, (3, 3))
    kern = workloads.GaussianIso(lambda x: 2.0 + 0 * x[..., 0], 6)
    phi = workloads.impulse_windows(shape, pcg.pc_sample_points(shape, cells), kern)
    for prec in ("bf16x3", "tf32x3"):
        with pytest.raises(pcg.PCError) as ei:
            pcg.Operator(context(), shape, cells, 6, phi, precision=prec)
        assert ei.value.status == PC_ERR_UNSUPPORTED
    op = pcg.Operator(context(), shape, cells, 6, phi, precision="fp32")
    run(op, workloads.rhs(66, 1, shape))
    with pytest.raises(pcg.PCError) as ei:
        op.stage_ms(0)
    assert ei.value.status == PC_ERR_NOT_READY
