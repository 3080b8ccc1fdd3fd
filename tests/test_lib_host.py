"""libpc host logic on the CPU: the library loads and exports every entry
point the header declares, and its sample points, neighbourhood boxes,
harmonic weights and extended impulse responses match the oracle's."""
import ctypes
import os
import re

import numpy as np
import pytest

import workloads
from workloads import configs
from oracle import Grid, harmonic_weights
from oracle.extension import extend_impulse_responses

from test_oracle_geometry import ADAPTIVE_CELLS, ADAPTIVE_SHAPE

pcb = pytest.importorskip("paper_1805_06018_gb300.binding")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built_library():
    from paper_1805_06018_gb300 import build
    build.build()
    return pcb.lib()


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names.update(re.findall(r"\b(pc_[a-z0-9_]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol():
    names = _declared()
    assert {"pc_build_spectra", "pc_apply", "pc_apply_batched", "pc_sample_points"} <= names
    L = ctypes.CDLL(pcb.LIB_PATH)
    for n in sorted(names):
        assert hasattr(L, n), n
    # and the binding wraps each of them
    assert names <= set(pcb._PROTOS), sorted(names - set(pcb._PROTOS))


GRIDS = [
    ((64, 64), workloads.regular_grid((64, 64), (4, 4))),
    ((512, 512), workloads.regular_grid((512, 512), (16, 16))),
    ((37, 23), workloads.regular_grid((37, 23), (5, 3))),
    (ADAPTIVE_SHAPE, np.array(ADAPTIVE_CELLS)),
    ((40, 30, 20), workloads.regular_grid((40, 30, 20), (3, 4, 2))),
]


@pytest.mark.parametrize("shape,cells", GRIDS)
def test_sample_points_and_boxes_match_oracle(shape, cells):
    g = Grid(shape, cells)
    pts = pcb.pc_sample_points(shape, cells)
    assert np.array_equal(pts, g.points)
    lo, hi = pcb.pc_neighbourhood_boxes(shape, cells)
    assert np.array_equal(lo, g.bbox_lo) and np.array_equal(hi, g.bbox_hi)


def test_adaptive_workload_points_match_oracle():
    wl = configs.adaptive_1024()
    g = Grid(wl.shape, wl.cells)
    assert np.array_equal(pcb.pc_sample_points(wl.shape, wl.cells), g.points)


@pytest.mark.parametrize("shape,cells", [GRIDS[0], GRIDS[2], GRIDS[4]])
def test_weights_match_oracle_on_conforming_grids(shape, cells):
    g = Grid(shape, cells)
    W = harmonic_weights(g)
    lw = pcb.pc_harmonic_weights(shape, cells)
    assert lw.size == sum(w.size for w in W)
    assert np.max(np.abs(lw - np.concatenate([w.ravel() for w in W]))) < 1e-14


@pytest.mark.parametrize("shape,cells,R", [(GRIDS[0][0], GRIDS[0][1], 12), (GRIDS[2][0], GRIDS[2][1], 5),
                                           (ADAPTIVE_SHAPE, np.array(ADAPTIVE_CELLS), 4),
                                           (GRIDS[4][0], GRIDS[4][1], 3)])
def test_extension_matches_oracle(shape, cells, R):
    g = Grid(shape, cells)
    rng = np.random.default_rng(11)
    phi = rng.standard_normal((g.r, (2 * R + 1) ** len(shape)))
    ref = extend_impulse_responses(g, workloads_mask(shape, g.points, R) * phi, R)
    got = pcb.pc_extend_impulse(shape, cells, R, phi)   # library ignores values outside Omega - p_k
    assert np.max(np.abs(got - ref)) < 1e-15 * max(1.0, np.abs(ref).max()) * 4


def workloads_mask(shape, points, R):
    d = len(shape)
    offs = np.stack(np.meshgrid(*[np.arange(-R, R + 1)] * d, indexing="ij"), -1).reshape(-1, d)
    y = points[:, None, :] + offs[None]
    return np.all((y >= 0) & (y < np.asarray(shape)), axis=-1).astype(float)


@pytest.mark.parametrize("cells,why", [
    ([[[0, 0], [5, 5]], [[4, 0], [9, 5]]], "overlap"),
    ([[[0, 0], [5, 5]]], "uncovered"),
    ([[[0, 0], [0, 5]], [[0, 0], [9, 5]]], "degenerate"),
    ([[[0, 0], [5, 5]], [[5, 0], [10, 5]]], "outside"),
])
def test_grid_validation(cells, why):
    with pytest.raises(pcb.PCError) as ei:
        pcb.pc_sample_points((10, 6), np.array(cells))
    assert ei.value.status == pcb.PC_ERR_GRID, why


@pytest.mark.parametrize("which", ["small", "adaptive_1024", "3d_broken_facet", "3d_octants"])
def test_weights_match_oracle_with_hanging_nodes(which):
    """The library solves 2D hanging-node leaves by bilinear + per-edge
    separation of variables, and 3D ones by facet pieces + a sine-basis
    interior solve written separately; the oracle by its recursive sine-basis
    solves.  Both are exact discrete harmonic extensions, so they agree to
    rounding."""
    from test_oracle_geometry import _broken_grid
    if which == "small":
        shape, cells = ADAPTIVE_SHAPE, np.array(ADAPTIVE_CELLS)
    elif which == "adaptive_1024":
        wl = configs.adaptive_1024()
        shape, cells = wl.shape, wl.cells
    else:
        shape, cells = _broken_grid(0 if which == "3d_broken_facet" else 1)
        cells = np.array(cells)
    g = Grid(shape, cells)
    W = harmonic_weights(g)
    lw = pcb.pc_harmonic_weights(shape, cells)
    ref = np.concatenate([w.ravel() for w in W])
    assert lw.size == ref.size
    assert np.max(np.abs(lw - ref)) < 1e-12


def test_header_is_plain_c_and_links():
    """include/pc.h compiles as pedantic C99, and a C program that takes the
    address of every declared entry point links against libpc.so (C linkage,
    no C++ name mangling)."""
    import shutil
    import subprocess
    import tempfile
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    names = sorted(_declared())
    src = "#include \"pc.h\"\n#include <stdio.h>\nint main(void) {\n"
    src += "".join("    printf(\"%%p\\n\", (void *)%s);\n" % n for n in names)
    src += "    return 0;\n}\n"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "abi.c")
        with open(c, "w") as fh:
            fh.write(src)
        libdir = os.path.dirname(pcb.LIB_PATH)
        cmd = [gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-I", os.path.join(root, "include"),
               c, "-o", os.path.join(d, "abi"), "-L", libdir, "-l:" + os.path.basename(pcb.LIB_PATH),
               "-Wl,-rpath," + libdir, "-Wl,--unresolved-symbols=ignore-in-shared-libs"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr


def _random_tree_3d(seed, shape=(17, 15, 13), splits=10):
    """Random one-axis splits of random leaves (the anisotropic refinement of
    Section 2.7), starting from the box split once per axis; splits that
    would break a facet crosswise (no weights defined, Section 2.4) are
    redrawn."""
    from oracle.adaptive import initial_cells, pieces_have_sample_corners, subdivide
    rng = np.random.default_rng(seed)
    cells = initial_cells(shape)
    for _ in range(splits):
        while True:
            c, a = int(rng.integers(len(cells))), int(rng.integers(3))
            if cells[c][1][a] - cells[c][0][a] > 2:
                nxt = subdivide(cells, c, a)
                if pieces_have_sample_corners(shape, nxt):
                    break
        cells = nxt
    return shape, cells


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_3d_weights_on_random_anisotropic_trees_match_oracle(seed):
    """One-axis splits break facets into T-junctions and put several hanging
    nodes on one edge; the library's weights (facet pieces, then a sine-basis
    interior solve) still equal the oracle's recursive solves, and form a
    partition of unity with the delta property."""
    shape, cells = _random_tree_3d(seed)
    g = Grid(shape, cells)
    W = harmonic_weights(g)       # asserts that the leaves agree on shared facets
    ref = np.concatenate([w.ravel() for w in W])
    lw = pcb.pc_harmonic_weights(shape, cells)
    assert lw.size == ref.size
    assert np.max(np.abs(lw - ref)) < 1e-12
    S = np.zeros(shape)
    for k in range(g.r):
        sl = tuple(slice(a, b + 1) for a, b in zip(g.bbox_lo[k], g.bbox_hi[k]))
        S[sl] += W[k]
    assert np.max(np.abs(S - 1.0)) < 1e-13


@pytest.mark.parametrize("seed", [0, 1, 2, 3, 4, 5])
def test_adaptive_split_admissibility_matches_oracle(seed):
    """The library's check that a split keeps every facet piece's corners at
    sample points (pc_split_is_admissible, written locally around the new
    leaves) agrees with the oracle's check of the whole grid, on every
    candidate split of random anisotropic 3D trees, crosswise ones included."""
    from oracle.adaptive import pieces_have_sample_corners, subdivide
    shape, cells = _random_tree_3d(seed, splits=6)
    arr = np.array(cells, dtype=np.int32)
    seen = {True: 0, False: 0}
    for c in range(len(cells)):
        for i in range(3):
            if cells[c][1][i] - cells[c][0][i] <= 2:
                continue
            got = pcb.pc_split_is_admissible(shape, arr, c, i)
            want = pieces_have_sample_corners(shape, subdivide(cells, c, i))
            assert got == want, (c, i)
            seen[got] += 1
    assert seen[True] > 0 and seen[False] > 0


def test_adaptive_crosswise_split_is_refused_by_both_sides():
    """The octant beside a leaf split along y: splitting it along z breaks
    their facet crosswise (refused by the library's check and by its
    weights), along y only leaves hanging nodes."""
    from oracle.adaptive import initial_cells, subdivide
    shape = (9, 9, 9)
    cells = initial_cells(shape)
    left = next(j for j, c in enumerate(cells) if tuple(c[0]) == (0, 0, 0))
    cells = subdivide(cells, left, 1)
    right = next(j for j, c in enumerate(cells) if tuple(c[0]) == (4, 0, 0))
    for axis, ok in [(2, False), (1, True)]:
        assert pcb.pc_split_is_admissible(shape, np.array(cells, dtype=np.int32), right, axis) == ok
        split = np.array(subdivide(cells, right, axis))
        if ok:
            pcb.pc_harmonic_weights(shape, split)
        else:
            with pytest.raises(pcb.PCError) as ei:
                pcb.pc_harmonic_weights(shape, split)
            assert ei.value.status == pcb.PC_ERR_GRID


@pytest.mark.parametrize("seed", [0, 1])
def test_adaptive_direction_order_matches_oracle(seed):
    """Section 2.7's directions, best first, from the library
    (pc_split_directions on its own extension) and from the oracle's
    extension, on every leaf of random 3D trees with a kernel that changes
    along all three axes."""
    import workloads
    from oracle import PCOracle
    from oracle.adaptive import split_directions
    shape, cells = _random_tree_3d(seed, splits=5)
    kern = workloads.GaussianAxis3D(lambda x: 1.0 + 0.05 * x[..., 0], lambda x: 1.2 + 0.04 * x[..., 1],
                                    lambda x: 0.9 + 0.06 * x[..., 2], 3)
    g = Grid(shape, cells)
    phi = workloads.impulse_windows(shape, g.points, kern)
    orc = PCOracle(shape, cells, phi, 3)
    arr = np.array(cells, dtype=np.int32)
    for c in range(len(cells)):
        got = pcb.pc_split_directions(shape, arr, 3, phi, c)
        assert got == split_directions(g, orc.phiE, 3, c)


class _OracleBackedOperator:
    """Stands in for the library operator inside the adaptive construction's
    host loop: the per-cell estimates come from the oracle, so the loop's
    choices (cells, directions, crosswise skips, batches) can be compared
    with the oracle's construction without a GPU."""

    def __init__(self, ctx, shape, cells, R, phi, precision="fp64", **tune):
        from oracle import PCOracle
        self.grid = Grid(shape, cells)
        self.orc = PCOracle(shape, cells, phi, R)

    def estimate_cell_errors(self, Z, Y, num_cells):
        from oracle.estimator import eta_from_adjoints
        z = Z.double().numpy()
        return eta_from_adjoints(self.grid, self.orc.apply_adjoint(z), Y.double().numpy().reshape(len(z), -1))

    def close(self):
        pass


@pytest.mark.parametrize("case", ["2d", "3d_crosswise"])
def test_adaptive_host_loop_matches_the_oracle_construction(monkeypatch, case):
    import torch
    import workloads
    from paper_1805_06018_gb300 import adaptive as lib_adaptive
    from oracle.adaptive import construct as oracle_construct
    if case == "2d":
        shape, R, batch, passes = (40, 36), 4, 2, 6
        kern = workloads.Skewed([0.6, -0.3], lambda x: 1.0 + 0.4 * np.sin(x[..., 0] / 6.0), R)
    else:
        shape, R, batch, passes = (13, 13, 13), 3, 2, 6
        kern = workloads.GaussianAxis3D(lambda x: 1.0 + 0 * x[..., 0],
                                        lambda x: 0.8 + 1.6 * (x[..., 0] < 6) * x[..., 1] / 13.0,
                                        lambda x: 0.8 + 1.6 * (x[..., 0] >= 6) * x[..., 2] / 13.0, R)
    A = workloads.dense_operator(shape, kern)
    q = 4
    Z = workloads.rhs(35, q, shape).reshape(q, -1).astype(np.float64)
    Y = Z @ A
    impulse = lambda pts: workloads.impulse_windows(shape, pts, kern)  # noqa: E731
    stats = {}
    ref_cells, ref_hist = oracle_construct(shape, impulse, R, Z, Y, tau=1e-6, max_passes=passes, batch=batch,
                                           stats=stats)
    monkeypatch.setattr(lib_adaptive, "Operator", _OracleBackedOperator)
    _, cells, hist = lib_adaptive.construct(None, shape, impulse, R, torch.from_numpy(Z.reshape((q,) + shape)),
                                            torch.from_numpy(Y.reshape((q,) + shape)), tau=1e-6,
                                            precision="fp64", max_passes=passes, batch=batch, incremental=False)
    assert np.array_equal(np.asarray(cells), np.asarray(ref_cells))
    assert [r for r, _ in hist] == [r for r, _ in ref_hist]
    assert np.allclose([e for _, e in hist], [e for _, e in ref_hist], rtol=1e-12, atol=0)
    if case == "3d_crosswise":
        assert stats.get("skipped_splits", 0) >= 1


def _mutations(cells, rng):
    """Invalid variants of a valid leaf list: a leaf grown into its
    neighbour, a leaf dropped, a degenerate leaf, a leaf past the box, a
    duplicated leaf."""
    cells = [np.array(c, dtype=np.int64) for c in cells]
    d = cells[0].shape[1]
    out = []
    c = int(rng.integers(len(cells)))
    a = int(rng.integers(d))
    grown = [x.copy() for x in cells]
    grown[c][1][a] += 1
    out.append(("overlap or outside", grown))
    out.append(("gap", [x for j, x in enumerate(cells) if j != c]))
    flat = [x.copy() for x in cells]
    flat[c][1][a] = flat[c][0][a]
    out.append(("degenerate", flat))
    shifted = [x.copy() for x in cells]
    shifted[c][0][a] -= 1
    out.append(("negative or overlap", shifted))
    out.append(("duplicate", cells + [cells[c].copy()]))
    return out


@pytest.mark.parametrize("seed", range(6))
def test_invalid_grids_are_refused_without_harm(seed):
    """Leaf lists that do not tile the box (overlaps, gaps, degenerate or
    out-of-box leaves, duplicates) are refused with PC_ERR_GRID by every host
    entry point that reads a grid; the oracle's grid refuses them too."""
    rng = np.random.default_rng(100 + seed)
    if seed % 2:
        shape, cells = _random_tree_3d(seed, splits=4)
    else:
        shape = (int(rng.integers(8, 40)), int(rng.integers(8, 40)))
        cells = workloads.regular_grid(shape, (int(rng.integers(2, 5)), int(rng.integers(2, 5))))
    for why, bad in _mutations(cells, rng):
        bad = np.array(bad, dtype=np.int64)
        for call in (lambda: pcb.pc_sample_points(shape, bad),
                     lambda: pcb.pc_neighbourhood_boxes(shape, bad),
                     lambda: pcb.pc_harmonic_weights(shape, bad)):
            with pytest.raises(pcb.PCError) as ei:
                call()
            assert ei.value.status == pcb.PC_ERR_GRID, why
        with pytest.raises(Exception):
            Grid(shape, bad)
    # and the valid grid still goes through
    assert np.array_equal(pcb.pc_sample_points(shape, np.array(cells)), Grid(shape, cells).points)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_extension_matches_oracle_on_random_3d_trees(seed):
    """phi_k^E (Section 2.5) on random anisotropic 3D trees, where sample
    points have uneven neighbour sets and the counting functions c_k vary."""
    shape, cells = _random_tree_3d(seed, splits=8)
    g = Grid(shape, cells)
    R = 4
    rng = np.random.default_rng(300 + seed)
    phi = rng.standard_normal((g.r, (2 * R + 1) ** 3))
    ref = extend_impulse_responses(g, workloads_mask(shape, g.points, R) * phi, R)
    got = pcb.pc_extend_impulse(shape, np.array(cells), R, phi)
    assert np.max(np.abs(got - ref)) < 4e-15 * max(1.0, np.abs(ref).max())


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_points_and_boxes_match_oracle_on_random_3d_trees(seed):
    shape, cells = _random_tree_3d(seed, splits=12)
    g = Grid(shape, cells)
    assert np.array_equal(pcb.pc_sample_points(shape, np.array(cells)), g.points)
    lo, hi = pcb.pc_neighbourhood_boxes(shape, np.array(cells))
    assert np.array_equal(lo, g.bbox_lo) and np.array_equal(hi, g.bbox_hi)


def _random_tree_2d(seed, shape=(41, 37), splits=25):
    from oracle.adaptive import initial_cells, subdivide
    rng = np.random.default_rng(seed)
    cells = initial_cells(shape)
    for _ in range(splits):
        while True:
            c, a = int(rng.integers(len(cells))), int(rng.integers(2))
            if cells[c][1][a] - cells[c][0][a] > 2:
                break
        cells = subdivide(cells, c, a)
    return shape, cells


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_2d_random_anisotropic_trees_match_oracle(seed):
    """Random one-axis splits in 2D: edges with several hanging nodes, leaves
    of very different sizes side by side.  Sample points, boxes, weights (to
    1e-12) and phi_k^E (to rounding) against the oracle."""
    shape, cells = _random_tree_2d(seed)
    g = Grid(shape, cells)
    arr = np.array(cells)
    assert np.array_equal(pcb.pc_sample_points(shape, arr), g.points)
    W = harmonic_weights(g)
    ref = np.concatenate([w.ravel() for w in W])
    assert np.max(np.abs(pcb.pc_harmonic_weights(shape, arr) - ref)) < 1e-12
    R = 6
    phi = np.random.default_rng(400 + seed).standard_normal((g.r, (2 * R + 1) ** 2))
    ext = extend_impulse_responses(g, workloads_mask(shape, g.points, R) * phi, R)
    assert np.max(np.abs(pcb.pc_extend_impulse(shape, arr, R, phi) - ext)) < 4e-15 * max(1.0, np.abs(ext).max())


def test_library_weights_match_the_hand_worked_fixture():
    """The library's weights on the hand-worked 5 x 3 box with one hanging
    node (tests/golden/hanging_2d_5x3.txt)."""
    from conftest import load_golden_sections
    from test_oracle_geometry import HANGING_5x3
    fx = load_golden_sections("hanging_2d_5x3.txt")
    shape, cells = HANGING_5x3
    arr = np.array(cells)
    pts = pcb.pc_sample_points(shape, arr)
    lo, hi = pcb.pc_neighbourhood_boxes(shape, arr)
    flat = pcb.pc_harmonic_weights(shape, arr)
    off = 0
    for k, p in enumerate(pts):
        ext = tuple(int(b - a + 1) for a, b in zip(lo[k], hi[k]))
        full = np.zeros(shape)
        full[lo[k][0]:hi[k][0] + 1, lo[k][1]:hi[k][1] + 1] = flat[off:off + int(np.prod(ext))].reshape(ext)
        off += int(np.prod(ext))
        assert np.max(np.abs(full - fx["w_%d_%d" % (int(p[0]), int(p[1]))])) < 1e-15
    assert off == flat.size


def test_library_extension_matches_the_hand_worked_fixture():
    """pc_extend_impulse on the hand-worked 3 x 3 example
    (tests/golden/extension_2d_3x3.txt); values outside Omega - p_k in the
    input are ignored by the library."""
    from conftest import load_golden_sections
    from test_oracle_geometry import _hand_extension_inputs
    fx = load_golden_sections("extension_2d_3x3.txt")
    shape, cells, phi = _hand_extension_inputs()
    got = pcb.pc_extend_impulse(shape, cells, 1, phi)
    for k in range(4):
        assert np.array_equal(got[k].reshape(3, 3), fx["phiE_%d" % k])


def test_library_3d_hanging_node_weight_matches_the_hand_worked_fixture():
    from conftest import load_golden_sections
    from test_oracle_geometry import HANGING_5x3x3
    want = load_golden_sections("hanging_3d_5x3x3.txt")["w_2_1_0"].reshape(5, 3, 3)
    shape, cells = HANGING_5x3x3
    arr = np.array(cells)
    pts = [tuple(int(v) for v in p) for p in pcb.pc_sample_points(shape, arr)]
    lo, hi = pcb.pc_neighbourhood_boxes(shape, arr)
    flat = pcb.pc_harmonic_weights(shape, arr)
    k = pts.index((2, 1, 0))
    sizes = [int(np.prod(h - l + 1)) for l, h in zip(lo, hi)]
    off = int(np.sum(sizes[:k]))
    ext = tuple(int(v) for v in hi[k] - lo[k] + 1)
    full = np.zeros(shape)
    full[tuple(slice(int(a), int(b) + 1) for a, b in zip(lo[k], hi[k]))] = flat[off:off + sizes[k]].reshape(ext)
    assert np.max(np.abs(full - want)) < 1e-15
