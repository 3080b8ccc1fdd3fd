"""Oracle adaptive construction (Algorithm 1) against what the method fixes.

* a translation-invariant operator is reproduced exactly (Section 2), so the
  estimator is zero at the first pass and nothing is refined;
* anisotropic refinement (Section 2.7): when the impulse responses change
  only along one axis, every split is along that axis;
* the loop stops once eta_Omega <= tau, and refining drives the true error
  (dense matrices, tiny box) down with the estimate;
* a planted mistake (splitting in the direction of least change) breaks the
  anisotropy pin.
"""
import numpy as np
import pytest

import workloads
from oracle import adaptive, Grid, harmonic_weights
from oracle.adaptive import construct, split_direction
from oracle.dense import dense_pc
from oracle.apply import PCOracle


def _impulse(shape, kern):
    return lambda pts: workloads.impulse_windows(shape, pts, kern)


def _probes(shape, A, q=6, seed=3):
    Z = np.random.default_rng(seed).standard_normal((q, int(np.prod(shape))))
    return Z, Z @ A


def test_translation_invariant_needs_no_refinement():
    shape = (30, 26)
    kern = workloads.Skewed([0.5, -0.2], lambda x: 1.3 + 0 * x[..., 0], 4)
    A = workloads.dense_operator(shape, kern)
    Z, Y = _probes(shape, A)
    cells, hist = construct(shape, _impulse(shape, kern), 4, Z, Y, tau=1e-8)
    assert len(hist) == 1 and hist[0][1] < 1e-10
    assert len(cells) == 4


def test_refinement_follows_the_axis_of_change():
    shape = (48, 40)
    L = 48.0
    kern = workloads.GaussianIso(lambda x: 0.7 + 3.0 * x[..., 0] / L, 6)   # varies along axis 0 only
    A = workloads.dense_operator(shape, kern)
    Z, Y = _probes(shape, A)
    cells, hist = construct(shape, _impulse(shape, kern), 6, Z, Y, tau=1e-3, max_passes=8)
    assert len(hist) == 8
    # the four first cells were split along axis 0 only: every leaf still
    # spans one of the two axis-1 halves of the first split
    m1 = (shape[1] - 1) // 2
    spans = {(int(c[0][1]), int(c[1][1])) for c in cells}
    assert spans == {(0, m1), (m1, shape[1] - 1)}


def test_loop_stops_at_tau_and_the_true_error_drops():
    shape = (40, 36)
    L = 40.0
    kern = workloads.GaussianAniso2D(lambda x: 1.0 + 1.5 * x[..., 0] / L, lambda x: 1.2 + 0.8 * x[..., 1] / L,
                                     lambda x: 0.3 + 0 * x[..., 0], 5)
    A = workloads.dense_operator(shape, kern)
    Z, Y = _probes(shape, A, q=8)
    tau = 0.02
    cells, hist = construct(shape, _impulse(shape, kern), 5, Z, Y, tau=tau, max_passes=60, batch=2)
    assert hist[-1][1] <= tau < hist[0][1]
    g = Grid(shape, cells)
    orc = PCOracle(shape, cells, workloads.impulse_windows(shape, g.points, kern), 5)
    true_final = np.linalg.norm(dense_pc(orc) - A) / np.linalg.norm(A)
    g0 = Grid(shape, adaptive.initial_cells(shape))
    orc0 = PCOracle(shape, g0.cells, workloads.impulse_windows(shape, g0.points, kern), 5)
    true_first = np.linalg.norm(dense_pc(orc0) - A) / np.linalg.norm(A)
    assert true_final < 0.5 * true_first
    # the estimate tracks the true relative Frobenius error within a small factor
    assert 0.2 < hist[-1][1] / true_final < 5.0


def test_planted_direction_mistake_is_caught(monkeypatch):
    """The anisotropy pin fails when the split direction is chosen wrongly
    (here: the direction of least change)."""
    shape = (48, 40)
    kern = workloads.GaussianIso(lambda x: 0.7 + 3.0 * x[..., 0] / 48.0, 6)
    g = Grid(shape, adaptive.initial_cells(shape))
    orc = PCOracle(shape, g.cells, workloads.impulse_windows(shape, g.points, kern), 6)
    assert all(split_direction(g, orc.phiE, 6, c) == 0 for c in range(4))
    real = adaptive.split_directions

    def least_change(grid, phiE, R, c):
        order = real(grid, phiE, R, c)
        return order[1:] + order[:1]

    monkeypatch.setattr(adaptive, "split_directions", least_change)
    A = workloads.dense_operator(shape, kern)
    Z, Y = _probes(shape, A)
    cells, _ = construct(shape, _impulse(shape, kern), 6, Z, Y, tau=1e-3, max_passes=8)
    m1 = (shape[1] - 1) // 2
    assert {(int(c[0][1]), int(c[1][1])) for c in cells} != {(0, m1), (m1, shape[1] - 1)}


def test_update_reuses_exactly_the_unaffected_correlations():
    """Section 2.8: after a refinement only the correlations of sample points
    that are new or have a new neighbour change.  Pinned on the oracle: every
    other point keeps bbox(U_k) and phi_k^E exactly, so its correlation
    flip(phi_k^E) * z on bbox(U_k) is reusable; and an update that reuses them
    and recomputes only the others reproduces A~* Z of the refined operator."""
    from oracle.adaptive import initial_cells, subdivide
    shape = (40, 36)
    kern = workloads.Skewed([0.6, -0.3], lambda x: 1.0 + 0.4 * np.sin(x[..., 0] / 6.0), 4)
    impulse = _impulse(shape, kern)
    cells_a = subdivide(subdivide(initial_cells(shape), 0, 0), 2, 1)
    cells_b = subdivide(cells_a, 3, 1)
    ga, gb = Grid(shape, cells_a), Grid(shape, cells_b)
    oa = PCOracle(shape, cells_a, impulse(ga.points), 4)
    ob = PCOracle(shape, cells_b, impulse(gb.points), 4)
    ia = {tuple(p): k for k, p in enumerate(ga.points)}
    z = np.random.default_rng(5).standard_normal((2,) + shape)

    def corr(orc, k):
        # flip(phi_k^E) * z restricted to bbox(U_k), unweighted
        w = [np.zeros_like(W) for W in orc.W]
        lo, hi = orc.grid.bbox_lo[k], orc.grid.bbox_hi[k]
        w[k] = np.ones(orc.grid.bbox_shape(k))
        one = PCOracle(shape, orc.grid.cells, orc.phi, orc.R, weights=w)
        one.phiE = orc.phiE
        return one.apply_adjoint(z)[(slice(None),) + tuple(slice(a, b + 1) for a, b in zip(lo, hi))]

    affected = 0
    yt = np.zeros((2,) + shape)
    for k, p in enumerate(gb.points):
        ka = ia.get(tuple(p))
        new_nbr = ka is None or set(map(tuple, gb.points[gb.nbrs[k]])) != set(map(tuple, ga.points[ga.nbrs[ka]]))
        if not new_nbr:
            assert np.array_equal(ob.phiE[k], oa.phiE[ka])
            assert np.array_equal(gb.bbox_lo[k], ga.bbox_lo[ka]) and np.array_equal(gb.bbox_hi[k], ga.bbox_hi[ka])
            c = corr(oa, ka)
        else:
            affected += 1
            c = corr(ob, k)
        lo, hi = gb.bbox_lo[k], gb.bbox_hi[k]
        yt[(slice(None),) + tuple(slice(a, b + 1) for a, b in zip(lo, hi))] += ob.W[k] * c
    assert 0 < affected < gb.r
    ref = ob.apply_adjoint(z)
    assert np.max(np.abs(yt - ref)) <= 1e-12 * np.abs(ref).max()


def test_3d_refinement_follows_the_axis_of_change():
    """3D (hanging nodes appear from the second split on): when the impulse
    responses change along one axis only, every split is along that axis, and
    the estimate falls to tau."""
    shape = (11, 12, 17)
    L = 17.0
    kern = workloads.GaussianAxis3D(lambda x: 1.0 + 0 * x[..., 0], lambda x: 1.0 + 0 * x[..., 0],
                                    lambda x: 0.8 + 1.6 * x[..., 2] / L, 3)
    A = workloads.dense_operator(shape, kern)
    Z, Y = _probes(shape, A, q=4)
    cells, hist = construct(shape, _impulse(shape, kern), 3, Z, Y, tau=0.06, max_passes=12, batch=2)
    assert hist[-1][1] <= 0.06 < hist[0][1]
    for lo, hi in cells:
        # leaves differ from the first subdivision only along axis 2
        for a in (0, 1):
            assert (lo[a], hi[a]) in (((0, 5), (5, 10)) if a == 0 else ((0, 5), (5, 11)))
    assert len(cells) > 8


def _crosswise_grid(second_axis):
    """Octants of 9^3; the octant at the origin split along axis 1, then its
    neighbour across x0 = 4 split along `second_axis`."""
    from oracle.adaptive import initial_cells, subdivide
    shape = (9, 9, 9)
    cells = initial_cells(shape)
    left = next(j for j, c in enumerate(cells) if tuple(c[0]) == (0, 0, 0))
    cells = subdivide(cells, left, 1)
    right = next(j for j, c in enumerate(cells) if tuple(c[0]) == (4, 0, 0))
    return shape, subdivide(cells, right, second_axis)


def test_crosswise_broken_facet_has_no_value_at_the_crossing():
    """Section 2.4 builds w_k on the pieces of broken facets down to their
    corners.  When the two sides of a facet are split along different axes
    (here y on one side, z on the other), the pieces meet at (4, 2, 2), which
    is no cell's corner: the recursion has no value there, and the oracle's
    weights refuse the grid.  Splitting both sides along the same axis leaves
    hanging nodes only, and is fine."""
    from oracle.adaptive import pieces_have_sample_corners
    shape, cells = _crosswise_grid(2)
    assert not pieces_have_sample_corners(shape, cells)
    assert (4, 2, 2) not in {tuple(int(v) for v in p) for p in Grid(shape, cells).points}
    with pytest.raises(ValueError):
        harmonic_weights(Grid(shape, cells))
    shape, cells = _crosswise_grid(1)
    assert pieces_have_sample_corners(shape, cells)
    harmonic_weights(Grid(shape, cells))


def test_3d_construction_skips_crosswise_splits():
    """A 3D kernel that changes along y on one side of x0 = 6 and along z on
    the other: Section 2.7 asks for crosswise splits across that plane.  Each
    is skipped for the cell's next direction, the construction goes on, every
    pass's grid is one Section 2.4 defines weights on, and the estimate
    falls."""
    shape = (13, 13, 13)
    L = 13.0
    kern = workloads.GaussianAxis3D(lambda x: 1.0 + 0 * x[..., 0],
                                    lambda x: 0.8 + 1.6 * (x[..., 0] < 6) * x[..., 1] / L,
                                    lambda x: 0.8 + 1.6 * (x[..., 0] >= 6) * x[..., 2] / L, 3)
    A = workloads.dense_operator(shape, kern)
    Z, Y = _probes(shape, A, q=4)
    stats = {}
    cells, hist = construct(shape, _impulse(shape, kern), 3, Z, Y, tau=0.02, max_passes=6, batch=2, stats=stats)
    assert stats.get("skipped_splits", 0) >= 1 and stats.get("fallbacks", 0) >= 1
    assert hist[-1][1] < 0.6 * hist[0][1]
    harmonic_weights(Grid(shape, cells))
