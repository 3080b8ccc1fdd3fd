"""Incremental estimator (Algorithm 1's update of Y~ = A~* Z) through the C
ABI.

* From an empty cache it recomputes every sample point and equals
  pc_estimate_cell_errors up to summation order (FP64: 1e-12 relative).
* After a refinement it recomputes only points that are new or have a new
  neighbour (the oracle's grids decide which), and still equals the full
  estimator of the refined operator.
* FP32: within 1e-5 of ||Y~[C]|| / sqrt(q) of the full estimator per cell.
* The adaptive construction gives the same leaves and estimates with and
  without it, and recomputes fewer points per pass than it has."""
import numpy as np
import pytest

import workloads
from oracle import Grid
from oracle.adaptive import initial_cells, subdivide

from gpu_common import context

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    context()


SHAPE = (40, 36)


def _kernel():
    return workloads.Skewed([0.6, -0.3], lambda x: 1.0 + 0.4 * np.sin(x[..., 0] / 6.0), 4)


def _op(cells, prec, R=4):
    import paper_1805_06018_gb300 as pcg
    pts = pcg.pc_sample_points(SHAPE, cells)
    return pcg.Operator(context(), SHAPE, cells, R, workloads.impulse_windows(SHAPE, pts, _kernel()),
                        precision=prec), pts


def _probes(prec, q=5):
    dt = torch.float64 if prec == "fp64" else torch.float32
    Z = torch.from_numpy(workloads.rhs(90, q, SHAPE)).to(dt).cuda()
    Y = torch.from_numpy(workloads.rhs(91, q, SHAPE)).to(dt).cuda()
    return Z, Y


def _affected(cells_a, cells_b):
    """Points of the refined grid that are new or have a new neighbour."""
    ga, gb = Grid(SHAPE, cells_a), Grid(SHAPE, cells_b)
    ia = {tuple(p): k for k, p in enumerate(ga.points)}
    out = 0
    for k, p in enumerate(gb.points):
        ka = ia.get(tuple(p))
        if ka is None or set(map(tuple, gb.points[gb.nbrs[k]])) != set(map(tuple, ga.points[ga.nbrs[ka]])):
            out += 1
    return out


def test_fresh_update_equals_the_full_estimator_fp64():
    import paper_1805_06018_gb300 as pcg
    cells = workloads.regular_grid(SHAPE, (4, 3))
    op, pts = _op(cells, "fp64")
    Z, Y = _probes("fp64")
    est = pcg.Estimator(context(), SHAPE, Z, Y, "fp64")
    eta, rec = est.update(op, len(cells))
    assert rec == len(pts)
    ref = op.estimate_cell_errors(Z, Y, len(cells))
    assert np.max(np.abs(eta - ref) / ref) <= 1e-12
    eta2, rec2 = est.update(op, len(cells))     # nothing changed: nothing recomputed, same bits
    assert rec2 == 0 and np.array_equal(eta2, eta)
    est.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_refinement_recomputes_only_affected_points(prec):
    import paper_1805_06018_gb300 as pcg
    cells_a = subdivide(subdivide(initial_cells(SHAPE), 0, 0), 2, 1)
    cells_b = subdivide(cells_a, 3, 1)
    cells_c = subdivide(cells_b, 0, 0)
    Z, Y = _probes(prec)
    est = pcg.Estimator(context(), SHAPE, Z, Y, prec)
    op_a, _ = _op(cells_a, prec)
    est.update(op_a, len(cells_a))
    for before, after in [(cells_a, cells_b), (cells_b, cells_c)]:
        op, pts = _op(after, prec)
        eta, rec = est.update(op, len(after))
        assert 0 < rec <= _affected(before, after) < len(pts)
        ref = op.estimate_cell_errors(Z, Y, len(after))
        if prec == "fp64":
            assert np.max(np.abs(eta - ref) / ref) <= 1e-12
        else:
            yt = op.apply_adjoint(Z).double().cpu().numpy().reshape(len(Z), *SHAPE)
            g = Grid(SHAPE, after)
            for c, (lo, hi) in enumerate(g.cells):
                sl = (slice(None),) + tuple(slice(int(a), int(b) + 1) for a, b in zip(lo, hi))
                scale = np.linalg.norm(yt[sl]) / np.sqrt(len(Z))
                assert abs(eta[c] - ref[c]) <= 1e-5 * scale + 1e-30
    est.close()


def test_adaptive_construction_with_and_without_the_update():
    from paper_1805_06018_gb300 import adaptive
    kern = _kernel()
    A = workloads.dense_operator(SHAPE, kern)
    Zn = np.random.default_rng(92).standard_normal((6, int(np.prod(SHAPE))))
    Yn = Zn @ A
    Z = torch.from_numpy(Zn.reshape((6,) + SHAPE)).cuda()
    Y = torch.from_numpy(Yn.reshape((6,) + SHAPE)).cuda()
    impulse = lambda pts: workloads.impulse_windows(SHAPE, pts, kern)  # noqa: E731
    st_inc, st_full = {}, {}
    _, cells_i, hist_i = adaptive.construct(context(), SHAPE, impulse, 4, Z, Y, tau=0.02, precision="fp64",
                                            max_passes=30, stats=st_inc)
    _, cells_f, hist_f = adaptive.construct(context(), SHAPE, impulse, 4, Z, Y, tau=0.02, precision="fp64",
                                            max_passes=30, incremental=False, stats=st_full)
    canon = lambda cs: sorted(tuple(int(v) for v in np.asarray(c).ravel()) for c in cs)  # noqa: E731
    assert canon(cells_i) == canon(cells_f)
    assert len(hist_i) == len(hist_f) > 3
    for (ri, ei), (rf, ef) in zip(hist_i, hist_f):
        assert ri == rf and abs(ei - ef) <= 1e-10 * ef
    rec, full = st_inc["recomputed"], st_full["recomputed"]
    assert rec[0] == full[0]
    assert all(a < b for a, b in zip(rec[1:], full[1:]))
    assert sum(rec) < 0.6 * sum(full)
