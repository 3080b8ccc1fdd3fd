"""O(1) matrix entries (Section 3.1, Eq. conv_matrix_entries) through the C
ABI against the oracle's dense matrix built from the same entry formula (the
oracle's dense matrix is itself pinned to the direct-sum apply)."""
import numpy as np
import pytest

import workloads
from oracle.dense import dense_pc

from gpu_common import context, make_pair
from test_oracle_geometry import ADAPTIVE_CELLS, ADAPTIVE_SHAPE

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    context()


def _kernel(d, R):
    return workloads.Skewed([0.6, -0.3, 0.2][:d], lambda x: 1.0 + 0.3 * np.sin(x[..., 0] / 4.0), R)


def _all_entries(op, N):
    rows = torch.arange(N, device="cuda").repeat_interleave(N)
    cols = torch.arange(N, device="cuda").repeat(N)
    out = op.entries(rows, cols)
    torch.cuda.synchronize()
    return out.cpu().numpy().reshape(N, N)


@pytest.mark.parametrize("name,shape,cells,prec,tol", [
    ("2d-regular-fp64", (13, 11), workloads.regular_grid((13, 11), (3, 3)), "fp64", 1e-13),
    ("2d-adaptive-fp64", ADAPTIVE_SHAPE, np.array(ADAPTIVE_CELLS), "fp64", 1e-13),
    ("2d-regular-fp32", (14, 17), workloads.regular_grid((14, 17), (3, 4)), "fp32", 1e-6),
    ("3d-regular-fp32", (7, 8, 6), workloads.regular_grid((7, 8, 6), (3, 3, 2)), "fp32", 1e-6),
])
def test_all_entries_match_the_entry_formula(name, shape, cells, prec, tol):
    op, orc = make_pair(shape, cells, _kernel(len(shape), 3), prec)
    N = int(np.prod(shape))
    got = _all_entries(op, N)
    ref = dense_pc(orc)
    assert np.max(np.abs(got - ref)) <= tol * np.abs(ref).max()


def test_sampled_entries_of_the_512_operator_and_bad_indices():
    from workloads import configs
    wl = configs.fp32_512(1)
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "fp32")
    rng = np.random.default_rng(5)
    x = rng.integers(0, wl.n, 300)
    # targets within the kernel window of each source, plus some far away
    off = rng.integers(-24, 25, (300, 2))
    xi, xj = np.unravel_index(x, wl.shape)
    y = np.ravel_multi_index((np.clip(xi + off[:, 0], 0, 511), np.clip(xj + off[:, 1], 0, 511)), wl.shape)
    y[::10] = rng.integers(0, wl.n, 30)
    got = op.entries(torch.from_numpy(y), torch.from_numpy(x)).cpu().numpy()
    # oracle: the column A~ e_x by direct summation, read at y
    for i in range(0, 300, 15):
        e = np.zeros(wl.n)
        e[x[i]] = 1.0
        col = orc.apply(e[None], points=np.array([y[i]]))[0, 0]
        assert abs(got[i] - col) <= 1e-6 * max(1e-3, abs(col)), (i, got[i], col)
    bad = op.entries(torch.tensor([0, -1, wl.n]), torch.tensor([wl.n + 5, 0, 3])).cpu().numpy()
    assert np.all(np.isnan(bad))


def test_entries_after_estimator_and_clean_teardown():
    """Every entry point on one operator, in turn: the estimator's scratch must
    not disturb the entry tables, and destroying the operator must free
    everything without a CUDA error."""
    shape = (13, 11)
    cells = workloads.regular_grid(shape, (3, 3))
    op, orc = make_pair(shape, cells, _kernel(2, 3), "fp64")
    N = int(np.prod(shape))
    ref = dense_pc(orc)
    z = torch.from_numpy(workloads.rhs(86, 3, shape).astype(np.float64)).cuda()
    for q in (1, 3):    # the second call grows the estimator scratch
        op.estimate_cell_errors(z[:q], z[:q], len(cells))
        got = _all_entries(op, N)
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.abs(ref).max()
    op.close()
    torch.cuda.synchronize()
    torch.zeros(4, device="cuda").sum().item()
