"""Entry points on a non-blocking stream (torch.cuda.Stream), straight after
the setup that feeds them: an operator's build, the first apply of a batch
size (which grows the ordering flags), the plain path's first call (which
uploads its tables), a block plan and the incremental estimator.  The
library's synchronous setup copies and clears run on the legacy default
stream, which a non-blocking stream is not ordered after, so each is
finished before work on the caller's stream can read it.  Every result must
equal the default-stream result bitwise."""
import numpy as np
import pytest

import workloads

from gpu_common import context

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPE = (56, 48)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    context()


def _operator(prec):
    import paper_1805_06018_gb300 as pcg
    cells = workloads.regular_grid(SHAPE, (4, 4))
    kern = workloads.Skewed([0.5, -0.25], lambda x: 1.0 + 0.3 * np.cos(x[..., 0] / 5.0), 5)
    pts = pcg.pc_sample_points(SHAPE, cells)
    return pcg.Operator(context(), SHAPE, cells, 5, workloads.impulse_windows(SHAPE, pts, kern), precision=prec), cells


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_applies_on_a_side_stream_right_after_setup(prec):
    import paper_1805_06018_gb300 as pcg
    dt = torch.float64 if prec == "fp64" else torch.float32
    x = torch.from_numpy(workloads.rhs(140, 7, SHAPE)).to(dt).cuda()
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        op, cells = _operator(prec)
        y = op.apply(x, stream=side)                    # first apply of 7: flags grow
        z = op.apply_adjoint(x, stream=side)
        yp = op.apply_plain(x, stream=side) if prec == "fp32" else None   # plain tables upload
        plan = pcg.BlockPlan(op, (8, 8), (31, 27), (20, 16), (47, 39))
        xs = x[:, 20:48, 16:40].contiguous()
        yb = plan.apply(xs, stream=side)
    side.synchronize()
    op.check()
    plan.check()
    ref_op, _ = _operator(prec)
    assert torch.equal(y, ref_op.apply(x))
    assert torch.equal(z, ref_op.apply_adjoint(x))
    if yp is not None:
        assert torch.equal(yp, ref_op.apply_plain(x))
    ref_plan = pcg.BlockPlan(ref_op, (8, 8), (31, 27), (20, 16), (47, 39))
    assert torch.equal(yb, ref_plan.apply(xs))
    torch.cuda.synchronize()


def test_estimator_update_on_a_side_stream():
    import paper_1805_06018_gb300 as pcg
    Z = torch.from_numpy(workloads.rhs(141, 4, SHAPE)).cuda()
    Y = torch.from_numpy(workloads.rhs(142, 4, SHAPE)).cuda()
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        op, cells = _operator("fp32")
        est = pcg.Estimator(context(), SHAPE, Z, Y, "fp32")
        eta, rec = est.update(op, len(cells), stream=side)
    ref_est = pcg.Estimator(context(), SHAPE, Z, Y, "fp32")
    ref, _ = ref_est.update(op, len(cells))
    assert rec == op.info()["r"] and np.array_equal(eta, ref)
    est.close()
    ref_est.close()
