"""Operators whose patches take their own launch shape (pc_tuning.per_patch):
the small patches of a locally refined quadtree get 128^2 FFTs (with split
kernel windows at the largest radius), the large ones 256^2.  Each shape is a part with its own
schedule and spectra, applied by its own launch after the zero-fill.  The
result must match the FP64 oracle, be bitwise reproducible, be bitwise
the same through the host-buffer apply, the server and the allocation-free
apply, and the adjoint must match the oracle's adjoint."""
import time

import numpy as np
import pytest

import workloads

from gpu_common import context, make_pair, rel_l2, run

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPE = (160, 150)


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    context()


def _cells():
    return workloads.quadtree_grid(SHAPE, 1, 4, lambda lo, hi: lo[0] < 50 and lo[1] < 50)


def _kernel(R):
    return workloads.HeavyTailed(lambda x: 2.0 + 2.0 * (x[..., 0] / 160.0), R)


@pytest.mark.parametrize("prec,R", [("fp32", 30), ("fp32", 50), ("fp64", 20)])
def test_per_patch_operator_matches_oracle(prec, R):
    op, orc = make_pair(SHAPE, _cells(), _kernel(R), prec, per_patch=True)
    info = op.info()
    if prec == "fp32":
        assert info["num_parts"] == (2 if R == 30 else 3), info
    x = workloads.rhs(81, 5, SHAPE)
    xin = x.astype(np.float64) if prec == "fp64" else x
    y = run(op, xin)
    tol = 1e-10 if prec == "fp64" else 1e-5
    assert np.all(rel_l2(y, orc.apply(x)) <= tol)
    assert np.array_equal(run(op, xin), y)   # fixed summation order
    dt = torch.float64 if prec == "fp64" else torch.float32
    ya = op.apply_adjoint(torch.from_numpy(xin).to(device="cuda", dtype=dt))
    torch.cuda.synchronize()
    op.check()
    assert np.all(rel_l2(ya.cpu().numpy(), orc.apply_adjoint(x)) <= tol)


def test_per_patch_operator_through_every_apply_path():
    import paper_1805_06018_gb300 as pcg
    op, _ = make_pair(SHAPE, _cells(), _kernel(30), "fp32", per_patch=True)
    assert op.info()["num_parts"] >= 2
    B, N = 6, op.N
    xh = torch.from_numpy(workloads.rhs(82, B, SHAPE)).pin_memory()
    ref = op.apply(xh.cuda())
    torch.cuda.synchronize()
    op.check()
    # host buffers (the chunked pipeline)
    assert torch.equal(op.apply_host(xh, chunk=2), ref.cpu())
    # allocation-free apply
    y = torch.full_like(ref, float("nan"))
    op.pc_apply_batched_noalloc(B, xh.cuda().data_ptr(), N, y.data_ptr(), N, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    context().noalloc_check()
    assert torch.equal(y, ref)
    # served alone on a slot
    srv = pcg.Server(context(), budget_bytes=4 << 30, streams=2)
    x = xh.cuda()
    yo = torch.full_like(x, float("nan"))
    t = srv.submit(op, x, yo)
    t0 = time.time()
    while srv.poll(t) is None:
        assert time.time() - t0 < 60
        time.sleep(0.001)
    srv.close()
    assert torch.equal(yo, ref)
    # the paths that keep one launch shape refuse it
    with pytest.raises(pcg.PCError) as e:
        pcg.BlockPlan(op, (0, 0), (40, 40), (0, 0), (40, 40))
    assert e.value.status == pcg.binding.PC_ERR_UNSUPPORTED
    with pytest.raises(pcg.PCError) as e:
        op.apply_plain(x)
    assert e.value.status == pcg.binding.PC_ERR_UNSUPPORTED
