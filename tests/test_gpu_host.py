"""Host-buffer apply (pc_apply_host): the batch streams through the device in
chunks of an even number of right-hand sides, so its result must be bitwise
that of the device apply of the whole batch, whatever the chunking; and it
must match the FP64 oracle at the device apply's tolerance."""
import numpy as np
import pytest

import workloads

from gpu_common import context, make_pair, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    context()


def _kernel(shape, R):
    L = float(max(shape))
    return workloads.Skewed([0.5, -0.2], lambda x: 1.0 + 0.4 * np.cos(2 * np.pi * x[..., 1] / L), R)


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("adjoint", [False, True])
@pytest.mark.parametrize("nrhs,chunk", [(9, 0), (9, 2), (9, 3), (8, 8), (1, 0), (13, 4)])
def test_host_apply_is_bitwise_the_device_apply(prec, adjoint, nrhs, chunk):
    shape = (48, 44)
    op, orc = make_pair(shape, workloads.regular_grid(shape, (4, 4)), _kernel(shape, 6), prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    xh = torch.from_numpy(workloads.rhs(70 + nrhs, nrhs, shape)).to(dt).pin_memory()
    yh = op.apply_host(xh, adjoint=adjoint, chunk=chunk)
    op.check()
    xd = xh.cuda()
    yd = op.apply_adjoint(xd) if adjoint else op.apply(xd)
    torch.cuda.synchronize()
    assert torch.equal(yh, yd.cpu())
    if nrhs == 9 and chunk == 0:
        x64 = xh.double().numpy()
        ref = orc.apply_adjoint(x64) if adjoint else orc.apply(x64)
        assert np.max(rel_l2(yh.double().numpy(), ref)) <= (1e-10 if prec == "fp64" else 1e-5)


def test_host_apply_strided_and_pageable():
    """ldx, ldy > N and plain (pageable) host memory."""
    shape = (40, 36)
    op, _ = make_pair(shape, workloads.regular_grid(shape, (3, 3)), _kernel(shape, 5), "fp32")
    N = op.N
    B = 5
    xs = np.zeros((B, N + 7), dtype=np.float32)
    xs[:, :N] = workloads.rhs(77, B, shape).reshape(B, N)
    ys = np.full((B, N + 3), 7.0, dtype=np.float32)
    op.pc_apply_host(B, xs.ctypes.data, N + 7, ys.ctypes.data, N + 3, False, 2,
                     torch.cuda.current_stream().cuda_stream)
    torch.cuda.current_stream().synchronize()
    op.check()
    ref = op.apply(torch.from_numpy(np.ascontiguousarray(xs[:, :N])).cuda()).cpu().numpy()
    assert np.array_equal(ys[:, :N], ref)
    assert np.all(ys[:, N:] == 7.0)   # the gaps between vectors are left alone


def test_host_apply_3d():
    shape = (24, 20, 18)
    kern = workloads.GaussianAxis3D(lambda x: 1.5 + 0 * x[..., 0], lambda x: 1.2 + 0 * x[..., 0],
                                    lambda x: 1.0 + 0 * x[..., 0], 4)
    op, orc = make_pair(shape, workloads.regular_grid(shape, (3, 3, 2)), kern, "fp32")
    xh = torch.from_numpy(workloads.rhs(78, 5, shape)).pin_memory()
    yh = op.apply_host(xh, chunk=2)
    op.check()
    assert np.max(rel_l2(yh.numpy(), orc.apply(xh.double().numpy()))) <= 1e-5
    assert torch.equal(yh, op.apply(xh.cuda()).cpu())


def test_host_apply_bad_arguments():
    import paper_1805_06018_gb300 as pcg
    from paper_1805_06018_gb300.binding import PC_ERR_ARG
    shape = (40, 36)
    op, _ = make_pair(shape, workloads.regular_grid(shape, (3, 3)), _kernel(shape, 5), "fp32")
    x = np.zeros((2, op.N), dtype=np.float32)
    for args in [(2, x.ctypes.data, op.N - 1, x.ctypes.data, op.N, False, 0),
                 (2, x.ctypes.data, op.N, x.ctypes.data, op.N, False, 0),       # x and y overlap
                 (2, x.ctypes.data, op.N, 0, op.N, False, 0),
                 (-1, x.ctypes.data, op.N, x.ctypes.data, op.N, False, 0)]:
        with pytest.raises(pcg.PCError) as ei:
            op.pc_apply_host(*args, 0)
        assert ei.value.status == PC_ERR_ARG


@pytest.mark.parametrize("adjoint", [False, True])
def test_host_apply_with_blocking_launches_takes_the_chunked_pipeline(monkeypatch, adjoint):
    """Where launches block the calling thread (CUDA_LAUNCH_BLOCKING), the
    segmented launch could not be fed its chunks; 2D operators then take the
    chunked pipeline (one zero and one patch launch per chunk) with the same
    bitwise result, as they do on request (PC_HOST_PIPELINE=chunked).  CUDA
    itself reads CUDA_LAUNCH_BLOCKING only when it starts, so here it steers
    the library alone."""
    shape = (48, 44)
    op, _ = make_pair(shape, workloads.regular_grid(shape, (4, 4)), _kernel(shape, 6), "fp32")
    xh = torch.from_numpy(workloads.rhs(79, 9, shape)).pin_memory()
    seg = op.apply_host(xh, adjoint=adjoint, chunk=2)
    assert op.launches() == 2
    monkeypatch.setenv("CUDA_LAUNCH_BLOCKING", "0")
    assert torch.equal(op.apply_host(xh, adjoint=adjoint, chunk=2), seg)
    assert op.launches() == 2
    monkeypatch.setenv("CUDA_LAUNCH_BLOCKING", "1")
    chunked = op.apply_host(xh, adjoint=adjoint, chunk=2)
    op.check()
    assert op.launches() == 2 * 5
    assert torch.equal(chunked, seg)
    monkeypatch.delenv("CUDA_LAUNCH_BLOCKING")
    monkeypatch.setenv("PC_HOST_PIPELINE", "chunked")
    assert torch.equal(op.apply_host(xh, adjoint=adjoint, chunk=2), seg)
    assert op.launches() == 2 * 5
    yd = op.apply_adjoint(xh.cuda()) if adjoint else op.apply(xh.cuda())
    assert torch.equal(chunked, yd.cpu())
