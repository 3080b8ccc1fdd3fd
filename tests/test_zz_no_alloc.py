"""pc_apply_batched_noalloc, the entry point for callers that cannot allocate
device memory while they apply the operator (its scratch is a static device
array inside libpc), against pc_apply_batched on the same inputs, called
twice in a row through the C ABI.  This file is collected last on purpose."""
import numpy as np
import pytest

import workloads
from workloads import configs

from gpu_common import context, make_pair, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-5   # FP32 relative l2 per right-hand side, as in the parity tests


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    context()


def test_noalloc_matches_batched_apply_twice():
    wl = configs.fp32_512(5)
    op, _ = make_pair(wl.shape, wl.cells, wl.kernel, "fp32")
    x = torch.from_numpy(workloads.rhs(21, 5, wl.shape)).cuda()
    N = wl.n
    s = torch.cuda.current_stream().cuda_stream
    ref = torch.empty_like(x)
    op.pc_apply_batched(5, x.data_ptr(), N, ref.data_ptr(), N, s)
    torch.cuda.synchronize()
    op.check()
    ref_np = ref.cpu().numpy()
    for _ in range(2):
        y = torch.full_like(x, float("nan"))
        op.pc_apply_batched_noalloc(5, x.data_ptr(), N, y.data_ptr(), N, s)
        torch.cuda.synchronize()
        err = rel_l2(y.cpu().numpy(), ref_np)
        assert np.all(err <= TOL), err


def test_noalloc_rejects_batches_beyond_its_scratch():
    import paper_1805_06018_gb300 as pcg
    wl = configs.fp32_512(1)
    op, _ = make_pair(wl.shape, wl.cells, wl.kernel, "fp32")
    tiles = op.info()["num_tiles"]
    nrhs = 2 * (262128 // tiles + 1)
    x = torch.zeros(4, device="cuda")
    with pytest.raises(pcg.PCError) as e:
        # nothing is launched: the size check comes first, so x and y are never read
        op.pc_apply_batched_noalloc(nrhs, x.data_ptr(), wl.n, x.data_ptr() + 8 * wl.n * nrhs, wl.n,
                                    torch.cuda.current_stream().cuda_stream)
    assert e.value.status == pcg.binding.PC_ERR_ARG
    assert "static scratch" in str(e.value)
