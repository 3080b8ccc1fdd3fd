"""Failure detection of the device-side waits (bounded, sticky), tested
without a GPU fault: the segmented host apply is run with the host holding
back the ready word of every segment after the first (PC_TEST_WITHHOLD_READY),
so the kernel's wait for it runs out.  The call must come back with
PC_ERR_TIMEOUT within about one wait limit (a 10 ms limit set through
pc_tuning.wait_limit_us), the other CTAs must give up at once instead of
each waiting out its own limit, and the context must then run a correct
apply."""
import os
import time

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


@pytest.fixture
def _segmented_host_path(monkeypatch):
    # the segmented launch (not the chunked fallback) is the path under test
    monkeypatch.delenv("PC_HOST_PIPELINE", raising=False)
    if os.environ.get("CUDA_LAUNCH_BLOCKING", "0") not in ("", "0"):
        pytest.skip("launches block the calling thread: the host apply takes the chunked pipeline")


def test_withheld_ready_word_times_out_then_context_recovers(_segmented_host_path, monkeypatch):
    import paper_1805_06018_gb300 as pcg
    wl = configs.fp32_512(16)
    op, _ = make_pair(wl.shape, wl.cells, wl.kernel, "fp32", wait_limit_us=10000)
    xh = torch.from_numpy(workloads.rhs(91, 16, wl.shape)).pin_memory()
    ref = op.apply(xh.cuda())
    torch.cuda.synchronize()
    op.check()
    # warm-up of the host path's own resources (copy streams, staging, flags)
    y0 = op.apply_host(xh, chunk=4)
    assert torch.equal(y0, ref.cpu())

    monkeypatch.setenv("PC_TEST_WITHHOLD_READY", "1")
    t0 = time.perf_counter()
    with pytest.raises(pcg.PCError) as e:
        op.apply_host(xh, chunk=4)
    elapsed = time.perf_counter() - t0
    assert e.value.status == pcg.binding.PC_ERR_TIMEOUT, str(e.value)
    # one 10 ms limit, not one per CTA (152 CTAs x 10 ms = 1.5 s) nor the 2 s default
    assert elapsed < 1.0, elapsed
    monkeypatch.delenv("PC_TEST_WITHHOLD_READY")

    # the status word was cleared; the context and the operator work again
    op.check()
    y1 = op.apply_host(xh, chunk=4)
    op.check()
    assert torch.equal(y1, ref.cpu())
    y2 = op.apply(xh.cuda())
    torch.cuda.synchronize()
    op.check()
    assert torch.equal(y2, ref)


def test_wait_limit_does_not_disturb_a_normal_apply():
    """A 1 ms limit is far above any legitimate wait of a small apply."""
    wl = configs.fp32_512(6)
    op, _ = make_pair(wl.shape, wl.cells, wl.kernel, "fp32", wait_limit_us=1000)
    ref_op, _ = make_pair(wl.shape, wl.cells, wl.kernel, "fp32")
    x = torch.from_numpy(workloads.rhs(92, 6, wl.shape)).cuda()
    for _ in range(3):
        y = op.apply(x)
        yr = ref_op.apply(x)
        torch.cuda.synchronize()
        op.check()
        assert torch.equal(y, yr)
