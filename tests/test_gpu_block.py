"""Block apply (Section 3.3) through the C ABI against the FP64 oracle.

Relative l2 per right-hand side: 1e-10 (FP64 operators), 1e-5 (FP32), as for
the whole-box apply.  With S = T = Omega a plan keeps every tile unchanged,
so its result must be bitwise the whole-box apply's."""
import numpy as np
import pytest

import workloads
from workloads import configs
from oracle import block as ob

from gpu_common import context, make_pair, rel_l2
from test_oracle_geometry import ADAPTIVE_CELLS, ADAPTIVE_SHAPE

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = {"fp64": 1e-10, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    context()


def _kernel(shape, R):
    L = float(max(shape))
    return workloads.Skewed([0.6, -0.3], lambda x: 1.0 + 0.4 * np.sin(2 * np.pi * x[..., 0] / L), R)


def _dev(a, prec):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda",
                                                        dtype=torch.float64 if prec == "fp64" else torch.float32)


def _run_block(op, t_lo, t_hi, s_lo, s_hi, x, adjoint):
    from paper_1805_06018_gb300 import BlockPlan
    plan = BlockPlan(op, t_lo, t_hi, s_lo, s_hi, adjoint)
    y = plan.apply(_dev(x, op.precision))
    torch.cuda.synchronize()
    plan.check()
    return plan, y.cpu().numpy().astype(np.float64)


def _check(got, ref, prec):
    ref = ref.reshape(len(ref), -1)
    got = got.reshape(len(ref), -1)
    nz = np.linalg.norm(ref, axis=1) > 0
    if np.any(nz):
        assert np.max(rel_l2(got[nz], ref[nz])) <= TOL[prec]
    assert np.all(np.abs(got[~nz]) <= TOL[prec] * (np.abs(got).max() + 1e-300))


BOXES = [   # (t_lo, t_hi, s_lo, s_hi) on a 40 x 36 box
    ((0, 0), (39, 35), (0, 0), (39, 35)),          # the whole box
    ((5, 7), (20, 30), (10, 2), (33, 14)),         # overlapping, ragged
    ((0, 0), (9, 9), (12, 0), (20, 6)),            # beside, within reach
    ((30, 30), (39, 35), (0, 0), (5, 5)),          # beyond the kernel's reach: zero
    ((17, 17), (17, 17), (17, 17), (17, 17)),      # one pixel
    ((0, 3), (39, 3), (2, 0), (2, 35)),            # one column x one row
]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("adjoint", [False, True])
def test_blocks_regular_grid(prec, adjoint):
    shape = (40, 36)
    cells = workloads.regular_grid(shape, (4, 3))
    op, orc = make_pair(shape, cells, _kernel(shape, 5), prec)
    rng = np.random.default_rng(60)
    for t_lo, t_hi, s_lo, s_hi in BOXES:
        sS = tuple(b - a + 1 for a, b in zip(s_lo, s_hi))
        x = rng.standard_normal((3,) + sS).astype(np.float32).astype(np.float64)
        plan, got = _run_block(op, t_lo, t_hi, s_lo, s_hi, x, adjoint)
        ref = ob.apply_block_translated(orc, t_lo, t_hi, s_lo, s_hi, x, adjoint)
        _check(got, ref, prec)
        terms, tiles = plan.info()
        assert terms <= len(ob.block_terms(orc, t_lo, t_hi, s_lo, s_hi, adjoint))
        if t_lo == s_lo and t_hi == s_hi:
            assert terms == len(ob.block_terms(orc, t_lo, t_hi, s_lo, s_hi, adjoint))
        if not np.any(ref):
            assert tiles == 0
        plan.close()


@pytest.mark.parametrize("adjoint", [False, True])
def test_blocks_adaptive_grid_fp64(adjoint):
    shape, cells = ADAPTIVE_SHAPE, np.array(ADAPTIVE_CELLS)
    op, orc = make_pair(shape, cells, _kernel(shape, 4), "fp64")
    rng = np.random.default_rng(61)
    for _ in range(6):
        lo = [sorted(rng.integers(0, m, 2)) for m in shape]
        lo2 = [sorted(rng.integers(0, m, 2)) for m in shape]
        t_lo, t_hi = [a for a, _ in lo], [b for _, b in lo]
        s_lo, s_hi = [a for a, _ in lo2], [b for _, b in lo2]
        sS = tuple(int(b - a + 1) for a, b in zip(s_lo, s_hi))
        x = rng.standard_normal((2,) + sS)
        _, got = _run_block(op, t_lo, t_hi, s_lo, s_hi, x, adjoint)
        _check(got, ob.apply_block(orc, t_lo, t_hi, s_lo, s_hi, x, adjoint), "fp64")


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("adjoint", [False, True])
def test_whole_box_block_is_bitwise_the_apply(prec, adjoint):
    from paper_1805_06018_gb300 import BlockPlan
    shape = (40, 36)
    op, _ = make_pair(shape, workloads.regular_grid(shape, (4, 3)), _kernel(shape, 5), prec)
    x = _dev(workloads.rhs(62, 5, shape), prec)
    plan = BlockPlan(op, (0, 0), (39, 35), (0, 0), (39, 35), adjoint)
    yb = plan.apply(x)
    ya = op.apply_adjoint(x) if adjoint else op.apply(x)
    torch.cuda.synchronize()
    assert torch.equal(yb, ya)
    assert torch.equal(plan.apply(x), yb)      # and reproducible
    plan.close()


@pytest.mark.parametrize("adjoint", [False, True])
def test_blocks_of_the_512_operator(adjoint):
    """The 512^2 benchmark operator (R = 24, FFT size 128): a near-field block
    (adjacent 64 x 64 boxes), an overlapping block and a far-field block, 5
    right-hand sides (odd: one pair is half used)."""
    wl = configs.fp32_512()
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "fp32")
    cases = [((128, 128), (191, 191), (192, 128), (255, 191)),
             ((300, 40), (363, 103), (320, 60), (383, 123)),
             ((0, 0), (63, 63), (400, 400), (463, 463))]
    for t_lo, t_hi, s_lo, s_hi in cases:
        x = workloads.rhs(63, 5, (64, 64)).astype(np.float64)
        _, got = _run_block(op, t_lo, t_hi, s_lo, s_hi, x, adjoint)
        _check(got, ob.apply_block_translated(orc, t_lo, t_hi, s_lo, s_hi, x, adjoint), "fp32")


def test_bad_arguments():
    import paper_1805_06018_gb300 as pcg
    from paper_1805_06018_gb300 import BlockPlan
    from paper_1805_06018_gb300.binding import PC_ERR_ARG, PC_ERR_UNSUPPORTED
    shape = (40, 36)
    op, _ = make_pair(shape, workloads.regular_grid(shape, (4, 3)), _kernel(shape, 5), "fp32")
    for box in [((0, 0), (40, 35), (0, 0), (3, 3)), ((5, 5), (4, 9), (0, 0), (3, 3)),
                ((0, 0), (3, 3), (-1, 0), (3, 3))]:
        with pytest.raises(pcg.PCError) as ei:
            BlockPlan(op, *box)
        assert ei.value.status == PC_ERR_ARG
    plan = BlockPlan(op, (0, 0), (9, 9), (0, 0), (9, 9))
    x = torch.zeros(100, device="cuda")
    y = torch.zeros(100, device="cuda")
    with pytest.raises(pcg.PCError) as ei:
        plan.pc_block_apply(1, x.data_ptr(), 99, y.data_ptr(), 100, 0)
    assert ei.value.status == PC_ERR_ARG
    plan.pc_block_apply(0, x.data_ptr(), 100, y.data_ptr(), 100, 0)   # no-op
    plan.close()
    shape3 = (12, 10, 8)
    kern3 = workloads.GaussianAxis3D(lambda x: 1.2 + 0 * x[..., 0], lambda x: 1.0 + 0 * x[..., 0],
                                     lambda x: 1.0 + 0 * x[..., 0], 3)
    op3, _ = make_pair(shape3, workloads.regular_grid(shape3, (2, 2, 2)), kern3, "bf16x3")
    with pytest.raises(pcg.PCError) as ei:
        BlockPlan(op3, (0, 0, 0), (3, 3, 3), (0, 0, 0), (3, 3, 3))
    assert ei.value.status == PC_ERR_UNSUPPORTED


def _random_blocks(shape, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        t = [sorted(rng.integers(0, m, 2)) for m in shape]
        s = [sorted(rng.integers(0, m, 2)) for m in shape]
        out.append(([a for a, _ in t], [b for _, b in t], [a for a, _ in s], [b for _, b in s]))
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("adjoint", [False, True])
def test_many_blocks_in_one_launch_are_bitwise_the_single_blocks(prec, adjoint):
    from paper_1805_06018_gb300 import BlockPlan
    shape = (40, 36)
    op, orc = make_pair(shape, workloads.regular_grid(shape, (4, 3)), _kernel(shape, 5), prec)
    blocks = [tuple(map(list, b)) for b in BOXES] + _random_blocks(shape, 8, 64)
    plan = BlockPlan(op, *[[b[i] for b in blocks] for i in range(4)], adjoint)
    rng = np.random.default_rng(65)
    xs = [_dev(rng.standard_normal((3,) + tuple(sh)), prec) for sh in plan.s_shapes]
    ys = plan.apply_many(xs)
    torch.cuda.synchronize()
    plan.check()
    for (t_lo, t_hi, s_lo, s_hi), x, y in zip(blocks, xs, ys):
        one = BlockPlan(op, t_lo, t_hi, s_lo, s_hi, adjoint)
        assert torch.equal(one.apply(x), y)
        one.close()
    for (t_lo, t_hi, s_lo, s_hi), x, y in list(zip(blocks, xs, ys))[:4]:
        ref = ob.apply_block_translated(orc, t_lo, t_hi, s_lo, s_hi, x.double().cpu().numpy(), adjoint)
        _check(y.double().cpu().numpy(), ref, prec)
    plan.close()


def test_more_blocks_than_one_launch_holds():
    """70 blocks: two launch rounds of one plan."""
    from paper_1805_06018_gb300 import BlockPlan
    shape = (40, 36)
    op, _ = make_pair(shape, workloads.regular_grid(shape, (4, 3)), _kernel(shape, 5), "fp32")
    blocks = _random_blocks(shape, 70, 66)
    plan = BlockPlan(op, *[[b[i] for b in blocks] for i in range(4)])
    rng = np.random.default_rng(67)
    xs = [_dev(rng.standard_normal((2,) + tuple(sh)), "fp32") for sh in plan.s_shapes]
    ys = plan.apply_many(xs)
    ys2 = plan.apply_many(xs)   # descriptors reused across calls
    torch.cuda.synchronize()
    plan.check()
    for i in (0, 33, 63, 64, 69):
        one = BlockPlan(op, *blocks[i])
        assert torch.equal(one.apply(xs[i]), ys[i]) and torch.equal(ys[i], ys2[i])
        one.close()
    plan.close()


def test_many_blocks_reject_overlapping_outputs():
    import paper_1805_06018_gb300 as pcg
    from paper_1805_06018_gb300 import BlockPlan
    from paper_1805_06018_gb300.binding import PC_ERR_ARG
    shape = (40, 36)
    op, _ = make_pair(shape, workloads.regular_grid(shape, (4, 3)), _kernel(shape, 5), "fp32")
    plan = BlockPlan(op, [[0, 0], [10, 10]], [[9, 9], [19, 19]], [[0, 0], [10, 10]], [[9, 9], [19, 19]])
    x = torch.zeros(2, 100, device="cuda")
    y = torch.zeros(150, device="cuda")
    with pytest.raises(pcg.PCError) as ei:
        plan.pc_block_apply_many(1, [x[0].data_ptr(), x[1].data_ptr()], [100, 100],
                                 [y.data_ptr(), y[50:].data_ptr()], [100, 100], 0)
    assert ei.value.status == PC_ERR_ARG
    with pytest.raises(pcg.PCError):
        plan.pc_block_apply(1, x.data_ptr(), 100, y.data_ptr(), 100, 0)   # several blocks: apply_many only
    plan.close()


def _skew3(shape, R):
    return workloads.Skewed([0.7, -0.4, 0.3], lambda x: 1.1 + 0.4 * np.sin(x[..., 0] / 5.0), R)


BOXES3 = [   # (t_lo, t_hi, s_lo, s_hi) on a 30 x 26 x 22 box
    ((0, 0, 0), (29, 25, 21), (0, 0, 0), (29, 25, 21)),
    ((3, 5, 2), (17, 20, 15), (8, 1, 6), (25, 12, 21)),
    ((0, 0, 0), (8, 8, 8), (10, 0, 2), (16, 6, 9)),
    ((25, 20, 18), (29, 25, 21), (0, 0, 0), (4, 4, 4)),
    ((11, 12, 13), (11, 12, 13), (11, 12, 13), (11, 12, 13)),
]


@pytest.mark.parametrize("adjoint", [False, True])
def test_blocks_3d_fp32(adjoint):
    """3D operators (P = 64): ragged, beside, out-of-reach and one-voxel
    blocks against the oracle; the whole-box block bitwise the apply; several
    blocks in one plan (one launch each) bitwise their single plans."""
    from paper_1805_06018_gb300 import BlockPlan
    shape = (30, 26, 22)
    op, orc = make_pair(shape, workloads.regular_grid(shape, (3, 3, 3)), _skew3(shape, 4), "fp32")
    rng = np.random.default_rng(68)
    xs = []
    for t_lo, t_hi, s_lo, s_hi in BOXES3:
        sS = tuple(b - a + 1 for a, b in zip(s_lo, s_hi))
        x = rng.standard_normal((3,) + sS).astype(np.float32).astype(np.float64)
        xs.append(x)
        _, got = _run_block(op, t_lo, t_hi, s_lo, s_hi, x, adjoint)
        _check(got, ob.apply_block_translated(orc, t_lo, t_hi, s_lo, s_hi, x, adjoint), "fp32")
    xw = _dev(workloads.rhs(69, 3, shape), "fp32")
    whole = BlockPlan(op, *BOXES3[0], adjoint)
    ref = op.apply_adjoint(xw) if adjoint else op.apply(xw)
    assert torch.equal(whole.apply(xw), ref)
    whole.close()
    plan = BlockPlan(op, *[[b[i] for b in BOXES3] for i in range(4)], adjoint)
    ys = plan.apply_many([_dev(x, "fp32") for x in xs])
    torch.cuda.synchronize()
    plan.check()
    for b, x, y in zip(BOXES3, xs, ys):
        one = BlockPlan(op, *b, adjoint)
        assert torch.equal(one.apply(_dev(x, "fp32")), y)
        one.close()
    plan.close()
