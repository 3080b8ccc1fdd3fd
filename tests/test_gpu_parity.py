"""CUDA path (through the C ABI) against the FP64 oracle on the same seeded
inputs.  Tolerances are relative l2 per right-hand side: 1e-10 for the FP64
path, 1e-5 for FP32.  The results are unique (A~ is a fixed linear map), so
every output element is compared."""
import numpy as np
import pytest

import workloads
from workloads import configs

from gpu_common import context, make_pair, rel_l2, run

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-10, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    context()


def _const(v):
    return lambda x: v + 0.0 * x[..., 0]


def test_fp64_workload_64():
    wl = configs.fp64_64()
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "fp64")
    x = workloads.rhs(wl.rhs_seed, wl.nrhs, wl.shape)
    y = run(op, x.astype(np.float64))
    ref = orc.apply(x)
    assert np.all(rel_l2(y, ref) <= TOL["fp64"]), rel_l2(y, ref)


def test_fp64_exact_at_sample_points():
    wl = configs.fp64_64()
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "fp64")
    A_cols = []
    E = np.zeros((orc.grid.r,) + wl.shape)
    for k, p in enumerate(orc.grid.points):
        E[(k,) + tuple(p)] = 1.0
        A_cols.append(wl.kernel.entry(np.stack(np.meshgrid(*[np.arange(n) for n in wl.shape], indexing="ij"), -1),
                                      np.broadcast_to(p.astype(float), wl.shape + (2,))))
    y = run(op, E)
    for k in range(orc.grid.r):
        assert np.max(np.abs(y[k] - A_cols[k])) < 1e-12


@pytest.mark.parametrize("nrhs", [1, 3, 8])
def test_fp32_workload_512_small_batches(nrhs):
    wl = configs.fp32_512(nrhs)
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "fp32")
    x = workloads.rhs(wl.rhs_seed, nrhs, wl.shape)
    y = run(op, x)
    err = rel_l2(y, orc.apply(x))
    assert np.all(err <= TOL["fp32"]), err


def test_fp32_workload_512_full_batch_sampled():
    """The benchmark's own launch: 64 right-hand sides, 512x512; the oracle
    evaluates 4096 seeded pixels of every right-hand side."""
    wl = configs.fp32_512()
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "fp32")
    x = workloads.rhs(wl.rhs_seed, wl.nrhs, wl.shape)
    y = run(op, x).reshape(wl.nrhs, -1)
    pts = np.random.default_rng(5).choice(wl.n, 4096, replace=False)
    ref = orc.apply(x, points=pts)
    err = np.linalg.norm(y[:, pts] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.all(err <= TOL["fp32"]), err.max()
    # and two whole right-hand sides
    full = orc.apply(x[[0, 63]])
    assert np.all(rel_l2(y[[0, 63]], full) <= TOL["fp32"])


@pytest.mark.parametrize("shape,npts,R,tile,P", [
    ((97, 131), (4, 6), 9, 0, 0),        # ragged cells, one tile per patch
    ((97, 131), (4, 6), 9, 17, 0),       # forced multi-tile patches, ragged tails
    ((70, 45), (2, 2), 20, 0, 64),       # patches larger than one tile (T = 24)
    ((33, 200), (3, 9), 5, 7, 0),
])
def test_fp32_tiling_and_ragged_edges(shape, npts, R, tile, P):
    kern = workloads.Skewed([0.9, -1.7], lambda x: 1.5 + 0.5 * np.sin(x[..., 0] / 9.0), R)
    cells = workloads.regular_grid(shape, npts)
    op, orc = make_pair(shape, cells, kern, "fp32", tile=tile, fft_size=P)
    x = workloads.rhs(77, 5, shape)
    err = rel_l2(run(op, x), orc.apply(x))
    assert np.all(err <= TOL["fp32"]), err


def test_fp32_fft64_variant():
    wl = configs.fp32_512(4)
    kern = workloads.GaussianAniso2D(wl.kernel.s1, wl.kernel.s2, wl.kernel.theta, 12)
    op, orc = make_pair(wl.shape, wl.cells, kern, "fp32", fft_size=64)
    x = workloads.rhs(5, 4, wl.shape)
    err = rel_l2(run(op, x), orc.apply(x))
    assert np.all(err <= TOL["fp32"]), err


def test_translation_invariant_operator_on_gpu():
    """A restricted convolution is reproduced at every pixel, boundaries included."""
    shape, R = (150, 170), 11
    kern = workloads.Skewed([2.0, -1.0], _const(2.5), R)
    cells = workloads.regular_grid(shape, (5, 6))
    op, orc = make_pair(shape, cells, kern, "fp64")
    x = workloads.rhs(3, 2, shape).astype(np.float64)
    from scipy import signal
    psi = workloads.impulse_windows((2 * R + 1,) * 2, np.array([[R, R]]), kern).reshape(2 * R + 1, 2 * R + 1)
    y = run(op, x)
    for b in range(2):
        ref = signal.convolve(x[b], psi, mode="full", method="direct")[R:R + shape[0], R:R + shape[1]]
        assert np.max(np.abs(y[b] - ref)) < 1e-12 * np.abs(ref).max()


def test_bitwise_deterministic_and_strided():
    wl = configs.fp32_512(6)
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "fp32")
    x = workloads.rhs(9, 6, wl.shape)
    xt = torch.from_numpy(x).cuda()
    y1 = op.apply(xt)
    y2 = op.apply(xt)
    torch.cuda.synchronize()
    assert torch.equal(y1, y2)
    # strided batches: ldx, ldy > N
    N = wl.n
    xs = torch.zeros(6, N + 37, device="cuda")
    xs[:, :N] = xt.reshape(6, N)
    ys = torch.full((6, N + 11), 7.0, device="cuda")
    op.pc_apply_batched(6, xs.data_ptr(), N + 37, ys.data_ptr(), N + 11, torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert torch.equal(ys[:, :N], y1.reshape(6, N))
    assert torch.all(ys[:, N:] == 7.0)
    op.check()


def test_single_vector_entry_point():
    wl = configs.fp32_512(1)
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "fp32")
    x = torch.from_numpy(workloads.rhs(4, 1, wl.shape)).cuda()
    y = torch.empty_like(x)
    op.pc_apply(x.data_ptr(), y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert np.all(rel_l2(y.cpu().numpy(), orc.apply(x.cpu().numpy())) <= TOL["fp32"])


def test_plain_path_matches_oracle():
    wl = configs.fp32_512(3)
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "fp32")
    x = workloads.rhs(12, 3, wl.shape)
    err = rel_l2(run(op, x, plain=True), orc.apply(x))
    assert np.all(err <= TOL["fp32"]), err


@pytest.mark.parametrize("prec", ["fp32", "bf16x3"])
def test_plain_path_3d_matches_oracle(prec):
    """The plain per-vector path on a 3D operator (cuFFT 64^3 per tile), for
    both 3D precisions: their spectra are FP32, so the plain path meets the
    FP32 tolerance for either."""
    shape = (40, 36, 33)
    cells = workloads.regular_grid(shape, (3, 3, 3))
    kern = workloads.GaussianAxis3D(lambda x: 1.5 + 0.02 * x[..., 0], lambda x: 2.0 + 0 * x[..., 0],
                                    lambda x: 1.2 + 0.03 * x[..., 2], 6)
    op, orc = make_pair(shape, cells, kern, prec)
    x = workloads.rhs(13, 2, shape)
    err = rel_l2(run(op, x, plain=True), orc.apply(x))
    assert np.all(err <= TOL["fp32"]), err


def test_errors_are_returned():
    import paper_1805_06018_gb300 as pcg
    wl = configs.fp32_512(1)
    op, _ = make_pair(wl.shape, wl.cells, wl.kernel, "fp32")
    x = torch.zeros(2, wl.n, device="cuda")
    s = torch.cuda.current_stream().cuda_stream
    with pytest.raises(pcg.PCError) as e:
        op.pc_apply_batched(-1, x.data_ptr(), wl.n, x.data_ptr(), wl.n, s)
    assert e.value.status == 1
    with pytest.raises(pcg.PCError):
        op.pc_apply_batched(1, 0, wl.n, x.data_ptr(), wl.n, s)
    with pytest.raises(pcg.PCError):   # x and y overlap
        op.pc_apply_batched(1, x.data_ptr(), wl.n, x.data_ptr(), wl.n, s)
    with pytest.raises(pcg.PCError):   # ld smaller than N
        op.pc_apply_batched(1, x[0].data_ptr(), 5, x[1].data_ptr(), wl.n, s)
    op.pc_apply_batched(0, 0, 0, 0, 0, s)  # empty batch is a no-op
    op.check()


# ------------------------------------------------------------------ adaptive grids, large radii

from test_oracle_geometry import ADAPTIVE_CELLS, ADAPTIVE_SHAPE  # noqa: E402


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_hanging_nodes(precision):
    kern = workloads.Skewed([0.4, -0.8], lambda x: 1.0 + 0.4 * np.cos(x[..., 1] / 5.0), 3)
    op, orc = make_pair(ADAPTIVE_SHAPE, np.array(ADAPTIVE_CELLS), kern, precision)
    x = workloads.rhs(31, 3, ADAPTIVE_SHAPE)
    xin = x.astype(np.float64) if precision == "fp64" else x
    err = rel_l2(run(op, xin), orc.apply(x))
    assert np.all(err <= TOL[precision]), err


@pytest.mark.parametrize("precision,R", [("fp32", 64), ("fp64", 64), ("fp32", 58)])
def test_split_kernel_window(precision, R):
    """2R+1 wider than the FFT allows: the window is cut into sub-windows with
    their own spectra and the tiles shrink accordingly."""
    shape = (150, 161)
    cells = workloads.regular_grid(shape, (3, 3))
    kern = workloads.HeavyTailed(lambda x: 2.0 + 3.0 * (x[..., 0] / 150.0), R)
    op, orc = make_pair(shape, cells, kern, precision)
    info = op.info()
    assert info["num_tiles"] > orc.grid.r
    x = workloads.rhs(41, 2, shape)
    xin = x.astype(np.float64) if precision == "fp64" else x
    err = rel_l2(run(op, xin), orc.apply(x))
    assert np.all(err <= TOL[precision]), err


@pytest.mark.parametrize("tune", [{}, {"per_patch": True}])
def test_adaptive_workload_1024_sampled(tune):
    """The adaptive 1024^2 quadtree (r = 1579, hanging nodes, heavy-tailed
    kernel, R = 64), with one launch shape and with per-patch shapes (128^2
    with split windows and 256^2, the benchmark's): 4096 seeded pixels of
    every right-hand side of a 32-RHS batch."""
    wl = configs.adaptive_1024(32)
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "fp32", **tune)
    if tune:
        assert op.info()["num_parts"] == 2
    x = workloads.rhs(wl.rhs_seed, 32, wl.shape)
    y = run(op, x).reshape(32, -1)
    pts = np.random.default_rng(9).choice(wl.n, 4096, replace=False)
    ref = orc.apply(x, points=pts)
    err = np.linalg.norm(y[:, pts] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.all(err <= TOL["fp32"]), err


# ------------------------------------------------------------------ 3D patches (64^3 FFTs)

def test_3d_small_full():
    shape = (40, 36, 30)
    cells = workloads.regular_grid(shape, (3, 3, 3))
    s = lambda x: 1.2 + 0.3 * np.sin(x[..., 0] / 7.0)  # noqa: E731
    kern = workloads.GaussianAxis3D(s, lambda x: 1.6 + 0 * x[..., 0], lambda x: 1.0 + 0.2 * np.cos(x[..., 2] / 5.0), 5)
    op, orc = make_pair(shape, cells, kern, "fp32")
    x = workloads.rhs(61, 3, shape)
    err = rel_l2(run(op, x), orc.apply(x))
    assert np.all(err <= TOL["fp32"]), err


def test_3d_split_window():
    """R = 40 at P = 64: the 81^3 window is cut into sub-windows."""
    shape = (70, 66, 60)
    cells = workloads.regular_grid(shape, (2, 2, 2))
    kern = workloads.HeavyTailed(lambda x: 3.0 + 0 * x[..., 0], 40)
    op, orc = make_pair(shape, cells, kern, "fp32")
    assert op.info()["num_tiles"] > orc.grid.r
    x = workloads.rhs(62, 2, shape)
    y = run(op, x).reshape(2, -1)
    pts = np.random.default_rng(3).choice(int(np.prod(shape)), 512, replace=False)
    ref = orc.apply(x, points=pts)
    err = np.linalg.norm(y[:, pts] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.all(err <= TOL["fp32"]), err


def test_3d_workload_128_sampled():
    """128^3, regular 8x8x8 grid, anisotropic 3D Gaussian, R = 12: 4 right-hand
    sides, 2048 seeded voxels each (plus one full right-hand side)."""
    wl = configs.fp32_128c(4)
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "fp32")
    x = workloads.rhs(wl.rhs_seed, 4, wl.shape)
    y = run(op, x).reshape(4, -1)
    pts = np.random.default_rng(11).choice(wl.n, 2048, replace=False)
    ref = orc.apply(x, points=pts)
    err = np.linalg.norm(y[:, pts] - ref, axis=1) / np.linalg.norm(ref, axis=1)
    assert np.all(err <= TOL["fp32"]), err


def test_3d_hanging_nodes():
    """A 3D grid with broken facets (octants of 13^3, one octant split again):
    the library's facet-piece weights and the apply against the oracle."""
    from test_oracle_geometry import _broken_grid
    shape, cells = _broken_grid(1)
    kern = workloads.Skewed([0.7, -0.4, 0.3], lambda x: 1.1 + 0.3 * np.sin(x[..., 0] / 4.0), 3)
    op, orc = make_pair(shape, np.array(cells), kern, "fp32")
    x = workloads.rhs(124, 3, shape)
    err = rel_l2(run(op, x), orc.apply(x))
    assert np.all(err <= TOL["fp32"]), err
