"""The hand-worked examples of tests/golden/ through the C ABI on the GPU:
the library's apply and entries reproduce values derived on paper, not only
the oracle's."""
import numpy as np
import pytest

from conftest import load_golden_sections
from gpu_common import context

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    context()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_hand_worked_column_of_the_approximation(prec, tol):
    """tests/golden/extension_2d_3x3.txt: A~ e_(1,1) on a 3 x 3 box with its
    four corners as sample points, R = 1 (Sections 2.4, 2.5, Eq.
    conv_matrix_entries)."""
    import paper_1805_06018_gb300 as pcg
    from test_oracle_geometry import _hand_extension_inputs
    want = load_golden_sections("extension_2d_3x3.txt")["Atilde_col_1_1"]
    shape, cells, phi = _hand_extension_inputs()
    op = pcg.Operator(context(), shape, cells, 1, phi, precision=prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    e = torch.zeros((1,) + shape, dtype=dt, device="cuda")
    e[0, 1, 1] = 1.0
    y = op.apply(e)
    torch.cuda.synchronize()
    op.check()
    assert np.max(np.abs(y[0].double().cpu().numpy() - want)) <= tol * np.abs(want).max()
    # the same column from the O(1) entry formula
    rows = torch.arange(9, dtype=torch.int64, device="cuda")
    cols = torch.full((9,), 4, dtype=torch.int64, device="cuda")
    ent = op.entries(rows, cols)
    torch.cuda.synchronize()
    assert np.max(np.abs(ent.cpu().numpy().reshape(3, 3) - want)) <= tol * np.abs(want).max()
