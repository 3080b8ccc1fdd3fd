"""Autotuner (pc_build_spectra with a NULL pc_tuning, pc_autotune): the
operator it keeps matches the FP64 oracle at the FP32 tolerance, reports the
shape it chose and how many candidates it timed, and is bitwise the operator
built with that shape given explicitly.  Operators the multi-request kernel
does not batch (fft_size 64, FP64) are served alone, with the same result as
their own apply."""
import time

import numpy as np
import pytest

import workloads
from workloads import configs

from gpu_common import context, make_pair, rel_l2, run

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    context()


def _same_shape(info):
    if info["num_parts"] > 1:   # the per-patch shape choice won
        return dict(per_patch=True, ctas_per_sm=info["ctas_per_sm"])
    return dict(fft_size=info["fft_size"], tile=info["tile"], window_split=info["window_split"],
                ctas_per_sm=info["ctas_per_sm"])


@pytest.mark.parametrize("case", ["fp32_512", "wide_window"])
def test_autotuned_operator_matches_oracle(case):
    if case == "fp32_512":
        wl = configs.fp32_512(3)
        shape, cells, kern = wl.shape, wl.cells, wl.kernel
    else:
        # a kernel window (2R+1 = 61) that leaves the tuner a choice of sub-window splits
        shape = (150, 130)
        cells = workloads.regular_grid(shape, (4, 3))
        kern = workloads.GaussianAniso2D(lambda x: 4.0 + 0 * x[..., 0], lambda x: 6.0 + np.sin(x[..., 0] / 20.0),
                                         lambda x: 0.3 + 0 * x[..., 0], 30)
    op, orc = make_pair(shape, cells, kern, "fp32", autotune=True)
    info = op.info()
    assert info["autotuned"] == 1
    assert info["tuned_candidates"] >= 2
    assert info["tuned_ms"] > 0
    assert info["fft_size"] in (64, 128, 256) and info["window_split"] >= 1
    x = workloads.rhs(61, 3, shape)
    y = run(op, x)
    err = rel_l2(y, orc.apply(x))
    assert np.all(err <= 1e-5), err
    fixed, _ = make_pair(shape, cells, kern, "fp32", **_same_shape(info))
    assert fixed.info()["autotuned"] == 0
    assert np.array_equal(run(fixed, x), y)


def test_autotuned_fp64_operator():
    wl = configs.fp64_64()
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "fp64", autotune=True)
    assert op.info()["autotuned"] == 1
    x = workloads.rhs(62, 2, wl.shape).astype(np.float64)
    assert np.all(rel_l2(run(op, x), orc.apply(x)) <= 1e-10)


def test_pc_autotune_reports_a_buildable_shape():
    import paper_1805_06018_gb300 as pcg
    wl = configs.fp32_512(1)
    pts = pcg.pc_sample_points(wl.shape, wl.cells)
    phi = workloads.impulse_windows(wl.shape, pts, wl.kernel)
    best, ms = pcg.pc_autotune(context(), wl.shape, wl.cells, wl.radius, phi, "fp32", nrhs=4)
    assert ms > 0
    assert best["fft_size"] in (64, 128)


def test_unbatched_operators_are_served_alone():
    import paper_1805_06018_gb300 as pcg
    ops = []
    shape = (96, 80)
    kern = workloads.GaussianAniso2D(lambda x: 1.5 + 0 * x[..., 0], lambda x: 2.0 + np.sin(x[..., 0] / 15.0),
                                     lambda x: 0.3 + 0 * x[..., 0], 8)
    cells = workloads.regular_grid(shape, (4, 3))
    ops.append(make_pair(shape, cells, kern, "fp32", fft_size=64)[0])
    ops.append(make_pair(shape, cells, kern, "fp64")[0])
    ops.append(make_pair(shape, cells, kern, "fp32", fft_size=128)[0])
    srv = pcg.Server(context(), budget_bytes=4 << 30, streams=2, max_requests_per_launch=8)
    jobs = []
    for q in range(9):
        op = ops[q % 3]
        dt = torch.float64 if op.precision == "fp64" else torch.float32
        x = torch.from_numpy(workloads.rhs(300 + q, 1 + q % 4, shape)).to(device="cuda", dtype=dt)
        y = torch.full_like(x, float("nan"))
        jobs.append((op, x, y))
    torch.cuda.synchronize()
    tickets = [srv.submit(op, x, y) for op, x, y in jobs]
    t0 = time.time()
    done = {}
    while len(done) < len(tickets):
        for t in tickets:
            if t not in done:
                r = srv.poll(t)
                if r is not None:
                    done[t] = r
        assert time.time() - t0 < 60, "requests did not finish"
        time.sleep(0.001)
    for (op, x, y), t in zip(jobs, tickets):
        assert done[t]["status"] == 0
        alone = op.apply(x)
        torch.cuda.synchronize()
        assert torch.equal(y, alone)
    srv.close()
