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
