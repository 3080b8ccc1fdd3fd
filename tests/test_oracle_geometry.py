"""Oracle grid, weights and extension against what the paper fixes
(Sections 2.2, 2.4, 2.5; Lemmas 4.1 and 4.2)."""
import itertools

import numpy as np
import pytest

import workloads
from oracle import Grid, harmonic_weights
from oracle.extension import domain_indicator, extend_impulse_responses, extension_weights
from oracle.grid import box_corners, box_midpoint
from oracle.weights import dirichlet_laplace, weight_on_omega

# a 2D grid with hanging nodes: one coarse leaf next to refined ones, and a
# coarse leaf whose edge carries two hanging nodes
ADAPTIVE_CELLS = [
    [[0, 0], [8, 8]], [[8, 0], [12, 4]], [[12, 0], [16, 4]], [[8, 4], [16, 8]],
    [[0, 8], [4, 12]], [[4, 8], [8, 12]], [[0, 12], [8, 16]], [[8, 8], [16, 16]],
    [[16, 0], [20, 16]],
]
ADAPTIVE_SHAPE = (21, 17)


def _grids():
    return [
        ((10, 13), workloads.regular_grid((10, 13), (3, 4))),
        ((9,), workloads.regular_grid((9,), (4,))),
        (ADAPTIVE_SHAPE, np.array(ADAPTIVE_CELLS)),
        ((7, 8, 9), workloads.regular_grid((7, 8, 9), (3, 3, 4))),
    ]


# ---------------------------------------------------------------- Lemma 4.1

def _box(lo, hi):
    return set(itertools.product(*[range(a, b + 1) for a, b in zip(lo, hi)]))


@pytest.mark.parametrize("seed", range(20))
def test_lemma_4_1_box_sums(seed):
    """S + T = S + corners(T) when S is at least as large as T (Lemma 4.1)."""
    rng = np.random.default_rng(seed)
    d = 1 + seed % 2
    tlo = rng.integers(-3, 3, d)
    text = rng.integers(0, 4, d)
    slo = rng.integers(-3, 3, d)
    sext = text + rng.integers(0, 3, d)
    S = _box(slo, slo + sext)
    T = _box(tlo, tlo + text)
    full = {tuple(a + b for a, b in zip(s, t)) for s in S for t in T}
    corn = {tuple(a + b for a, b in zip(s, t)) for s in S for t in box_corners(tlo, tlo + text)}
    assert full == corn


def test_midpoint_rounds_down_on_ties():
    assert box_midpoint([0, 0], [1023, 10]) == (511, 5)


# ---------------------------------------------------------------- grid (2.2)

@pytest.mark.parametrize("shape,cells", _grids())
def test_grid_structure(shape, cells):
    g = Grid(shape, cells)
    # points are exactly the leaf corners, lexicographically ordered
    corners = set()
    for lo, hi in g.cells:
        corners.update(box_corners(lo, hi))
    assert [tuple(p) for p in g.points] == sorted(corners)
    cover = np.zeros(shape, dtype=bool)
    for k in range(g.r):
        assert k in g.nbrs[k]
        for j in g.nbrs[k]:
            assert k in g.nbrs[j]
        cover |= g.U_mask_full(k)
        assert g.U_mask_full(k)[tuple(g.points[k])]
    assert cover.all()


def test_hanging_node_belongs_to_coarse_leaf():
    g = Grid(ADAPTIVE_SHAPE, ADAPTIVE_CELLS)
    k = g.index[(8, 4)]  # hanging on the edge x0 = 8 of leaf [0,8]x[0,8]
    cs = [tuple(map(tuple, g.cells[c])) for c in g.cells_of[k]]
    assert ((0, 0), (8, 8)) in cs
    # both hanging nodes on the edge x1 = 0..16 of leaf [16,20]x[0,16]
    for p in [(16, 4), (16, 8)]:
        cs = [tuple(map(tuple, g.cells[c])) for c in g.cells_of[g.index[p]]]
        assert ((16, 0), (20, 16)) in cs


# ---------------------------------------------------------------- weights (2.4)

@pytest.mark.parametrize("shape,cells", _grids())
def test_weights_partition_of_unity_and_delta(shape, cells):
    g = Grid(shape, cells)
    W = harmonic_weights(g)
    S = np.zeros(shape)
    for k in range(g.r):
        wk = weight_on_omega(g, W, k)
        S += wk
        for j in range(g.r):
            assert wk[tuple(g.points[j])] == (1.0 if j == k else 0.0)
        assert np.all(wk[~g.U_mask_full(k)] == 0.0)      # supp w_k in U_k
        assert wk.min() >= -1e-15 and wk.max() <= 1 + 1e-15  # maximum principle
    assert np.max(np.abs(S - 1.0)) < 1e-13


def _hat_1d(axis_pts, i, n):
    """Textbook piecewise-linear nodal basis function i on 0..n-1."""
    x = np.arange(n, dtype=np.float64)
    return np.interp(x, axis_pts, np.eye(len(axis_pts))[i])


@pytest.mark.parametrize("shape,npts", [((10, 13), (3, 4)), ((64, 64), (4, 4)), ((7, 8, 9), (3, 3, 4)),
                                        ((20, 19, 18), (3, 4, 3))])
def test_weights_are_multilinear_hats_on_conforming_cells(shape, npts):
    g = Grid(shape, workloads.regular_grid(shape, npts))
    W = harmonic_weights(g)
    axes = [workloads.regular_points_1d(L, n) for L, n in zip(shape, npts)]
    for k in range(g.r):
        idx = [int(np.nonzero(axes[a] == g.points[k][a])[0][0]) for a in range(len(shape))]
        hat = _hat_1d(axes[0], idx[0], shape[0])
        for a in range(1, len(shape)):
            hat = np.multiply.outer(hat, _hat_1d(axes[a], idx[a], shape[a]))
        assert np.max(np.abs(weight_on_omega(g, W, k) - hat)) < 1e-14


def test_weights_discrete_harmonic_with_hanging_nodes():
    """Graph-Laplacian residual vanishes inside each leaf; edge data is linear
    between consecutive sample points (Section 2.4)."""
    g = Grid(ADAPTIVE_SHAPE, ADAPTIVE_CELLS)
    W = harmonic_weights(g)
    pts = {tuple(p) for p in g.points}
    for k in range(g.r):
        wk = weight_on_omega(g, W, k)
        for lo, hi in g.cells:
            V = wk[lo[0]:hi[0] + 1, lo[1]:hi[1] + 1]
            if V.shape[0] > 2 and V.shape[1] > 2:
                res = 4 * V[1:-1, 1:-1] - V[:-2, 1:-1] - V[2:, 1:-1] - V[1:-1, :-2] - V[1:-1, 2:]
                assert np.max(np.abs(res)) < 1e-14
            # every edge: linear between consecutive sample points
            for a in range(2):
                for side in (lo[a], hi[a]):
                    b = 1 - a
                    line = [(side, t) if a == 0 else (t, side) for t in range(lo[b], hi[b] + 1)]
                    vals = np.array([wk[p] for p in line])
                    nodes = [i for i, p in enumerate(line) if p in pts]
                    for i0, i1 in zip(nodes[:-1], nodes[1:]):
                        lin = np.linspace(vals[i0], vals[i1], i1 - i0 + 1)
                        assert np.max(np.abs(vals[i0:i1 + 1] - lin)) < 1e-14


def test_hanging_node_weight_is_not_bilinear():
    """With a hanging node the harmonic weight differs from any bilinear hat:
    the coarse leaf sees a kinked edge."""
    g = Grid(ADAPTIVE_SHAPE, ADAPTIVE_CELLS)
    W = harmonic_weights(g)
    k = g.index[(8, 4)]
    wk = weight_on_omega(g, W, k)
    V = wk[0:9, 0:9]
    assert V[8, 4] == 1.0 and V[4, 4] > 0
    # a bilinear function with these edge values would be linear on x0 = 8 too
    assert abs(V[8, 2] - 0.5) < 1e-14 and abs(V[8, 6] - 0.5) < 1e-14


def test_sine_solver_against_dense_solve():
    rng = np.random.default_rng(3)
    for shp in [(5, 7), (4, 3, 6), (9,)]:
        V = rng.standard_normal(shp)
        U = dirichlet_laplace(V)
        inner = tuple(slice(1, -1) for _ in shp)
        m = tuple(s - 2 for s in shp)
        n = int(np.prod(m))
        # assemble the graph Laplacian independently
        L = np.zeros((n, n))
        b = np.zeros(n)
        idx = np.arange(n).reshape(m)
        for pos in itertools.product(*[range(s) for s in m]):
            i = idx[pos]
            L[i, i] = 2 * len(shp)
            for a in range(len(shp)):
                for dlt in (-1, 1):
                    q = list(pos)
                    q[a] += dlt
                    if 0 <= q[a] < m[a]:
                        L[i, idx[tuple(q)]] -= 1
                    else:
                        qq = [c + 1 for c in q]
                        b[i] += V[tuple(qq)]
        sol = np.linalg.solve(L, b).reshape(m)
        assert np.max(np.abs(U[inner] - sol)) < 1e-13
        # boundary untouched
        mask = np.ones(shp, bool)
        mask[inner] = False
        assert np.array_equal(U[mask], V[mask])


# 3D leaves with hanging nodes (broken facets, Section 2.4)
BROKEN_3D = [
    # a coarse leaf beside two finer ones: its facet x0 = 4 is broken at z = 2
    ((9, 5, 5), [[[0, 0, 0], [4, 4, 4]], [[4, 0, 0], [8, 4, 2]], [[4, 0, 2], [8, 4, 4]]]),
    # octants of 13^3, one octant split again into octants: hanging nodes on
    # facets (centres of broken facets) and on edges
    ((13, 13, 13), None),
]


def _octants(lo, hi):
    mid = [(a + b) // 2 for a, b in zip(lo, hi)]
    out = []
    for side in itertools.product((0, 1), repeat=3):
        out.append([[lo[a] if s == 0 else mid[a] for a, s in enumerate(side)],
                    [mid[a] if s == 0 else hi[a] for a, s in enumerate(side)]])
    return out


def _broken_grid(i):
    shape, cells = BROKEN_3D[i]
    if cells is None:
        cells = _octants([0, 0, 0], [12, 12, 12])
        fine = cells.pop(0)
        cells += _octants(fine[0], fine[1])
    return shape, cells


@pytest.mark.parametrize("i", [0, 1])
def test_3d_hanging_nodes_partition_delta_support_maximum(i):
    shape, cells = _broken_grid(i)
    g = Grid(shape, cells)
    W = harmonic_weights(g)       # also asserts that the leaves agree on shared facets
    S = np.zeros(shape)
    for k in range(g.r):
        wk = weight_on_omega(g, W, k)
        S += wk
        for j in range(g.r):
            assert wk[tuple(g.points[j])] == (1.0 if j == k else 0.0)
        assert np.all(wk[~g.U_mask_full(k)] == 0.0)
        assert wk.min() >= -1e-15 and wk.max() <= 1 + 1e-15
    assert np.max(np.abs(S - 1.0)) < 1e-13


def _residual(V):
    """Graph-Laplacian residual at the interior nodes of an array of any dimension."""
    m = V.ndim
    inner = tuple(slice(1, -1) for _ in range(m))
    res = 2 * m * V[inner]
    for a in range(m):
        lo = [slice(1, -1)] * m
        hi = [slice(1, -1)] * m
        lo[a] = slice(0, -2)
        hi[a] = slice(2, None)
        res = res - V[tuple(lo)] - V[tuple(hi)]
    return res


@pytest.mark.parametrize("i", [0, 1])
def test_3d_hanging_nodes_harmonic_on_every_piece(i):
    """The weight is discrete-harmonic inside every leaf and on every facet
    piece (the constituent boxes of broken facets), and linear on every edge
    between consecutive sample points."""
    from oracle.weights import facet_pieces
    shape, cells = _broken_grid(i)
    g = Grid(shape, cells)
    W = harmonic_weights(g)
    pts = {tuple(p) for p in g.points}
    nbroken = 0
    for k in range(g.r):
        wk = weight_on_omega(g, W, k)
        for c, (lo, hi) in enumerate(g.cells):
            V = wk[tuple(slice(a, b + 1) for a, b in zip(lo, hi))]
            if min(V.shape) > 2:
                assert np.max(np.abs(_residual(V))) < 1e-13
            for a in range(3):
                for side in (0, 1):
                    pieces = facet_pieces(g, c, a, side)
                    nbroken += len(pieces) > 1
                    for plo, phi in pieces:
                        F = wk[tuple(slice(x, y + 1) for x, y in zip(plo, phi))].squeeze(axis=a)
                        if min(F.shape) > 2:
                            assert np.max(np.abs(_residual(F))) < 1e-13
                        # its four edges: linear between consecutive sample points
                        for b in [x for x in range(3) if x != a]:
                            for e in (plo[b], phi[b]):
                                elo, ehi = plo.copy(), phi.copy()
                                elo[b] = ehi[b] = e
                                free = [x for x in range(3) if elo[x] != ehi[x]][0]
                                line = []
                                for t in range(elo[free], ehi[free] + 1):
                                    q = list(elo)
                                    q[free] = t
                                    line.append(tuple(q))
                                vals = np.array([wk[q] for q in line])
                                nodes = [j for j, q in enumerate(line) if q in pts]
                                for j0, j1 in zip(nodes[:-1], nodes[1:]):
                                    lin = np.linspace(vals[j0], vals[j1], j1 - j0 + 1)
                                    assert np.max(np.abs(vals[j0:j1 + 1] - lin)) < 1e-14
    assert nbroken > 0


def test_3d_broken_facet_as_one_box_is_caught(monkeypatch):
    """Planted mistake: solving a broken facet as one box (ignoring the finer
    leaves across it) gives the two sides different facet values."""
    from oracle import weights as ow
    shape, cells = _broken_grid(0)
    g = Grid(shape, cells)

    def whole(grid, c, a, side):
        lo, hi = (np.array(v, dtype=np.int64) for v in grid.cells[c])
        flo, fhi = lo.copy(), hi.copy()
        flo[a] = fhi[a] = hi[a] if side else lo[a]
        return [(flo, fhi)]
    monkeypatch.setattr(ow, "facet_pieces", whole)
    with pytest.raises((AssertionError, ValueError)):
        ow.harmonic_weights(g)


# ---------------------------------------------------------------- extension (2.5)

@pytest.mark.parametrize("shape,cells", _grids())
@pytest.mark.parametrize("R", [2, 5])
def test_lemma_4_2_extension_weights(shape, cells, R):
    """sum_j v_k^(j)[z] = 1 iff z in Omega - U_k, else 0 (Lemma 4.2)."""
    g = Grid(shape, cells)
    V = extension_weights(g, R)
    from oracle.extension import window_offsets
    Z = window_offsets(g.d, R)
    for k in range(g.r):
        s = sum(V[k].values())
        Uk = np.argwhere(g.U_mask_full(k))
        # z in Omega - U_k  <=>  exists u in U_k with z + u in Omega
        inside = np.zeros(Z.shape[:-1], dtype=bool)
        for u in Uk:
            y = Z + u
            inside |= np.all((y >= 0) & (y < np.asarray(shape)), axis=-1)
        assert np.max(np.abs(s - inside.astype(float))) < 1e-15


def test_extension_keeps_own_values_and_averages_neighbours():
    g = Grid(ADAPTIVE_SHAPE, ADAPTIVE_CELLS)
    R = 3
    rng = np.random.default_rng(0)
    phi = rng.standard_normal((g.r, (2 * R + 1) ** 2))
    ind = [domain_indicator(g, g.points[k], R).ravel() for k in range(g.r)]
    phi = phi * np.array(ind)  # impulse responses vanish outside Omega - p_k
    E = extend_impulse_responses(g, phi, R)
    for k in range(g.r):
        assert np.array_equal(E[k][ind[k]], phi[k][ind[k]])
        for z in np.nonzero(~ind[k])[0]:
            js = [j for j in g.nbrs[k] if j != k and ind[j][z]]
            want = np.mean([phi[j][z] for j in js]) if js else 0.0
            assert abs(E[k][z] - want) < 1e-15


HANGING_5x3 = ((5, 3), [[[0, 0], [2, 2]], [[2, 0], [4, 1]], [[2, 1], [4, 2]]])


def test_hanging_node_weights_match_the_hand_worked_fixture(golden):
    """tests/golden/hanging_2d_5x3.txt: the weights of a 5 x 3 box with one
    hanging node, worked out by hand from Section 2.4 (linear edges split at
    sample points, the 5-point mean at the one interior point)."""
    fx = golden("hanging_2d_5x3.txt")
    shape, cells = HANGING_5x3
    g = Grid(shape, np.array(cells))
    W = harmonic_weights(g)
    assert [tuple(int(v) for v in p) for p in g.points] == [(0, 0), (0, 2), (2, 0), (2, 1), (2, 2), (4, 0), (4, 1),
                                                            (4, 2)]
    for k, p in enumerate(g.points):
        want = fx["w_%d_%d" % (int(p[0]), int(p[1]))]
        assert np.max(np.abs(weight_on_omega(g, W, k) - want)) < 1e-15


def _hand_extension_inputs():
    shape = (3, 3)
    cells = np.array([[[0, 0], [2, 2]]])
    a, b = np.meshgrid(np.arange(3), np.arange(3), indexing="ij")
    phi = np.stack([10.0 * (j + 1) + 3 * a + b for j in range(4)]).reshape(4, 9)
    return shape, cells, phi


def test_extension_matches_the_hand_worked_fixture(golden):
    """tests/golden/extension_2d_3x3.txt: phi_k^E on a 3 x 3 box with its four
    corners as sample points, worked out by hand from Section 2.5."""
    from oracle.extension import extend_impulse_responses
    fx = golden("extension_2d_3x3.txt")
    shape, cells, phi = _hand_extension_inputs()
    g = Grid(shape, cells)
    offs = np.stack(np.meshgrid(np.arange(-1, 2), np.arange(-1, 2), indexing="ij"), -1).reshape(-1, 2)
    mask = np.array([[np.all((p + z >= 0) & (p + z < 3)) for z in offs] for p in g.points], dtype=float)
    got = extend_impulse_responses(g, mask * phi, 1)
    for k in range(4):
        assert np.array_equal(got[k].reshape(3, 3), fx["phiE_%d" % k])


def test_hand_worked_column_of_the_approximation(golden):
    """The column x = (1,1) of A~ on the hand-worked 3 x 3 example, from the
    oracle's direct-sum apply of e_(1,1) and from its entry-formula matrix."""
    from oracle import PCOracle
    from oracle.dense import dense_pc
    fx = golden("extension_2d_3x3.txt")
    shape, cells, phi = _hand_extension_inputs()
    g = Grid(shape, cells)
    offs = np.stack(np.meshgrid(np.arange(-1, 2), np.arange(-1, 2), indexing="ij"), -1).reshape(-1, 2)
    mask = np.array([[np.all((p + z >= 0) & (p + z < 3)) for z in offs] for p in g.points], dtype=float)
    orc = PCOracle(shape, cells, mask * phi, 1)
    e = np.zeros((1, 3, 3))
    e[0, 1, 1] = 1.0
    assert np.max(np.abs(orc.apply(e)[0] - fx["Atilde_col_1_1"])) < 1e-13
    assert np.max(np.abs(dense_pc(orc)[:, 4].reshape(3, 3) - fx["Atilde_col_1_1"])) < 1e-13


HANGING_5x3x3 = ((5, 3, 3), [[[0, 0, 0], [2, 2, 2]], [[2, 0, 0], [4, 1, 2]], [[2, 1, 0], [4, 2, 2]]])


def test_3d_hanging_node_weight_matches_the_hand_worked_fixture(golden):
    """tests/golden/hanging_3d_5x3x3.txt: the weight of a hanging node on a
    broken facet, worked out by hand from Section 2.4 (edges, then the facet
    pieces and facets, then the interiors, each by its discrete Laplace
    mean)."""
    want = golden("hanging_3d_5x3x3.txt")["w_2_1_0"].reshape(5, 3, 3)
    shape, cells = HANGING_5x3x3
    g = Grid(shape, np.array(cells))
    W = harmonic_weights(g)
    k = [tuple(int(v) for v in p) for p in g.points].index((2, 1, 0))
    assert np.max(np.abs(weight_on_omega(g, W, k) - want)) < 1e-15
