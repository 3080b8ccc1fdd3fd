"""pc_apply_batched_noalloc, the entry point for callers that cannot allocate
device memory while they apply the operator (its scratch is a static device
array inside libpc), against pc_apply_batched on the same inputs, through the
C ABI.  The two run the same kernel on the same schedule, so their results
must be bitwise equal.  This file is collected last on purpose."""
import numpy as np
import pytest

import workloads
from workloads import configs

from gpu_common import context, make_pair

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    context()


def _stream():
    return torch.cuda.current_stream().cuda_stream


def test_noalloc_allocates_nothing_and_matches_batched_apply():
    """On a fresh operator: one warm-up call (nrhs = 0, the set-up), then a
    batch larger than any the operator has seen (80 RHS, 40 pairs): neither
    the operator's device bytes nor the device's free memory change, and the
    result is bitwise that of pc_apply_batched, twice in a row."""
    wl = configs.fp32_512(1)
    op, _ = make_pair(wl.shape, wl.cells, wl.kernel, "fp32")
    B, N = 80, wl.n
    x = torch.from_numpy(workloads.rhs(21, B, wl.shape)).cuda()
    y = torch.full_like(x, float("nan"))
    op.pc_apply_batched_noalloc(0, 0, N, 0, N, _stream())
    # the test's own buffers, and torch's fill and copy kernels (loaded on
    # first use, which takes device memory), before the measurement starts
    outs = [torch.empty_like(y) for _ in range(2)]
    for o in outs:
        o.copy_(y)
    y.fill_(float("nan"))
    torch.cuda.synchronize()
    dev_bytes = op.info()["device_bytes"]
    free0 = torch.cuda.mem_get_info()[0]
    for o in outs:
        y.fill_(float("nan"))
        op.pc_apply_batched_noalloc(B, x.data_ptr(), N, y.data_ptr(), N, _stream())
        torch.cuda.synchronize()
        context().noalloc_check()
        o.copy_(y)
    torch.cuda.synchronize()
    assert op.info()["device_bytes"] == dev_bytes
    assert torch.cuda.mem_get_info()[0] == free0
    ref = torch.empty_like(x)
    op.pc_apply_batched(B, x.data_ptr(), N, ref.data_ptr(), N, _stream())
    torch.cuda.synchronize()
    op.check()
    for o in outs:
        assert torch.equal(o, ref)


def test_noalloc_alternating_operators():
    """The one array serves every operator: calls alternate between the 512^2
    operator and the FP64 64^2 one (different tile counts and batches), so
    flags left by one call must be cleared by the next; each result is
    bitwise its own operator's pc_apply_batched."""
    ops = []
    for wl, prec, B in ((configs.fp32_512(1), "fp32", 7), (configs.fp64_64(), "fp64", 3)):
        op, _ = make_pair(wl.shape, wl.cells, wl.kernel, prec)
        dt = torch.float64 if prec == "fp64" else torch.float32
        x = torch.from_numpy(workloads.rhs(40 + B, B, wl.shape)).to(device="cuda", dtype=dt)
        ref = torch.empty_like(x)
        op.pc_apply_batched(B, x.data_ptr(), wl.n, ref.data_ptr(), wl.n, _stream())
        ops.append((op, x, ref, B, wl.n))
    torch.cuda.synchronize()
    for _ in range(2):
        for op, x, ref, B, N in ops:
            y = torch.full_like(x, float("nan"))
            op.pc_apply_batched_noalloc(B, x.data_ptr(), N, y.data_ptr(), N, _stream())
            torch.cuda.synchronize()
            context().noalloc_check()
            assert torch.equal(y, ref)


def test_noalloc_refuses_3d_operators():
    import paper_1805_06018_gb300 as pcg
    shape = (20, 18, 16)
    op, _ = make_pair(shape, workloads.regular_grid(shape, (2, 2, 2)),
                      workloads.GaussianAxis3D(*(lambda x: 1.2 + 0 * x[..., 0],) * 3, 3), "fp32")
    x = torch.zeros(op.N, device="cuda")
    y = torch.zeros(op.N, device="cuda")
    with pytest.raises(pcg.PCError) as e:
        op.pc_apply_batched_noalloc(1, x.data_ptr(), op.N, y.data_ptr(), op.N, _stream())
    assert e.value.status == pcg.binding.PC_ERR_UNSUPPORTED


def test_noalloc_rejects_batches_beyond_its_scratch():
    import paper_1805_06018_gb300 as pcg
    wl = configs.fp32_512(1)
    op, _ = make_pair(wl.shape, wl.cells, wl.kernel, "fp32")
    tiles = op.info()["num_tiles"]
    nrhs = 2 * (262128 // tiles + 1)
    x = torch.zeros(4, device="cuda")
    with pytest.raises(pcg.PCError) as e:
        # nothing is launched: the size check comes first, so x and y are never read
        op.pc_apply_batched_noalloc(nrhs, x.data_ptr(), wl.n, x.data_ptr() + 8 * wl.n * nrhs, wl.n, _stream())
    assert e.value.status == pcg.binding.PC_ERR_ARG
    assert "static scratch" in str(e.value)
