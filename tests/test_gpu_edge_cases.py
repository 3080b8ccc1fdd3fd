"""Degenerate and extreme cases of the method through the C ABI, forward and
adjoint, against the FP64 oracle (relative l2 per right-hand side: 1e-10 for
FP64 operators, 1e-5 for FP32):

* the smallest box (2 x 2, one cell, R = 1) and its 3D counterpart;
* a kernel window wider than the box (R = 7 on 5 x 3);
* every grid point a sample point (cells of width 1), where the method
  reproduces A exactly (Section 2: phi_k^E = phi_k at each point), checked
  against the dense operator;
* thin boxes (2 x 300, 300 x 2);
* a large odd batch (131 right-hand sides, 66 pairs)."""
import numpy as np
import pytest

import workloads

from gpu_common import context, make_pair, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-10, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    context()


def _kernel(d, R):
    return workloads.Skewed([0.6, -0.3, 0.2][:d], lambda x: 1.0 + 0.3 * np.sin(x[..., 0] / 3.0), R)


def _both(op, orc, x, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    xd = torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dt)
    y = op.apply(xd)
    z = op.apply_adjoint(xd)
    torch.cuda.synchronize()
    op.check()
    x64 = np.asarray(x, dtype=np.float64)
    assert np.all(rel_l2(y.double().cpu().numpy(), orc.apply(x64)) <= TOL[prec])
    assert np.all(rel_l2(z.double().cpu().numpy(), orc.apply_adjoint(x64)) <= TOL[prec])
    return y, z


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape,npts,R", [
    ((2, 2), (2, 2), 1),        # the smallest box: one cell, four points
    ((5, 3), (2, 2), 7),        # the kernel window is wider than the box
    ((2, 300), (2, 7), 4),      # thin boxes
    ((300, 2), (9, 2), 4),
])
def test_degenerate_2d_boxes(prec, shape, npts, R):
    op, orc = make_pair(shape, workloads.regular_grid(shape, npts), _kernel(2, R), prec)
    _both(op, orc, workloads.rhs(120, 3, shape), prec)


@pytest.mark.parametrize("shape,npts,R", [((2, 2, 2), (2, 2, 2), 1), ((3, 9, 2), (2, 3, 2), 3)])
def test_degenerate_3d_boxes(shape, npts, R):
    op, orc = make_pair(shape, workloads.regular_grid(shape, npts), _kernel(3, R), "fp32")
    _both(op, orc, workloads.rhs(121, 3, shape), "fp32")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_every_point_a_sample_point_reproduces_A(prec):
    shape = (9, 7)
    kern = _kernel(2, 3)
    op, orc = make_pair(shape, workloads.regular_grid(shape, shape), kern, prec)
    A = workloads.dense_operator(shape, kern)
    x = workloads.rhs(122, 2, shape)
    y, z = _both(op, orc, x, prec)
    x64 = x.reshape(2, -1).astype(np.float64)
    assert np.all(rel_l2(y.double().cpu().numpy(), x64 @ A.T) <= TOL[prec])
    assert np.all(rel_l2(z.double().cpu().numpy(), x64 @ A) <= TOL[prec])


def test_large_odd_batch():
    shape = (40, 36)
    op, orc = make_pair(shape, workloads.regular_grid(shape, (4, 3)), _kernel(2, 5), "fp32")
    x = workloads.rhs(123, 131, shape)
    y, _ = _both(op, orc, x, "fp32")
    # the last (half-used) pair and a middle one match single applies
    for b in (0, 77, 130):
        one = op.apply(torch.from_numpy(x[b:b + 1]).cuda())
        assert np.allclose(one.cpu().numpy(), y[b:b + 1].cpu().numpy(), rtol=0, atol=1e-5 * float(one.abs().max()))
