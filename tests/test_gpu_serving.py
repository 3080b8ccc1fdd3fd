"""Serving loop (pc_serve_*): requests over several resident operators with
uneven right-hand-side counts are batched into shared persistent launches;
each result equals the same request applied alone (pc_apply_batched), within
the FP32 tolerance and in fact bit for bit."""
import time

import numpy as np
import pytest

import workloads
from workloads import configs

from gpu_common import context, make_pair, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ops():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    context()
    out = []
    wl = configs.fp32_512(1)
    out.append(make_pair(wl.shape, wl.cells, wl.kernel, "fp32")[0])
    for shape, npts, R in [((256, 256), (9, 9), 24), ((200, 300), (4, 6), 12)]:
        cells = workloads.regular_grid(shape, npts)
        kern = workloads.GaussianAniso2D(lambda x: 2.0 + 0 * x[..., 0], lambda x: 3.0 + np.sin(x[..., 0] / 30.0),
                                         lambda x: 0.4 + 0 * x[..., 0], R)
        out.append(make_pair(shape, cells, kern, "fp32", fft_size=128)[0])
    return out


def _wait(srv, tickets, timeout=60.0):
    done = {}
    t0 = time.time()
    while len(done) < len(tickets):
        for t in tickets:
            if t not in done:
                r = srv.poll(t)
                if r is not None:
                    done[t] = r
        assert time.time() - t0 < timeout, "requests did not finish"
        time.sleep(0.001)
    return done


def test_mixed_requests_match_alone(ops):
    import paper_1805_06018_gb300 as pcg
    srv = pcg.Server(context(), budget_bytes=8 << 30, streams=2, max_requests_per_launch=16)
    rng = np.random.default_rng(0)
    prepared = []
    for q in range(24):
        op = ops[q % len(ops)]
        nrhs = int(rng.integers(1, 8))
        x = torch.from_numpy(workloads.rhs(500 + q, nrhs, op.shape)).cuda()
        prepared.append((op, x, torch.full_like(x, float("nan"))))
    torch.cuda.synchronize()
    # submitted back to back: requests queue behind the busy launch slots
    jobs = [(op, x, y, srv.submit(op, x, y)) for op, x, y in prepared]
    done = _wait(srv, [j[3] for j in jobs])
    for op, x, y, t in jobs:
        alone = op.apply(x)
        torch.cuda.synchronize()
        assert np.all(rel_l2(y.cpu().numpy(), alone.cpu().numpy()) <= 1e-5)
        assert torch.equal(y, alone)
        assert done[t]["status"] == 0 and done[t]["finish_s"] >= done[t]["launch_s"] >= done[t]["submit_s"]
    st = srv.stats()
    assert st["completed"] == 24
    assert st["launches"] < 24                        # requests shared launches
    assert max(d["launch_requests"] for d in done.values()) > 1
    assert st["p99_latency_s"] >= st["p50_latency_s"] > 0
    srv.close()


def test_budget_admission(ops):
    import paper_1805_06018_gb300 as pcg
    big = max(op.info()["device_bytes"] for op in ops)
    # room for one operator at a time: requests on different operators serialise
    srv = pcg.Server(context(), budget_bytes=big + (4 << 20), streams=2)
    tickets, jobs = [], []
    for q in range(6):
        op = ops[q % len(ops)]
        x = torch.from_numpy(workloads.rhs(900 + q, 3, op.shape)).cuda()
        y = torch.empty_like(x)
        tickets.append(srv.submit(op, x, y))
        jobs.append((op, x, y))
    _wait(srv, tickets)
    for op, x, y in jobs:
        assert torch.equal(y, op.apply(x))
    st = srv.stats()
    assert st["peak_bytes"] <= big + (4 << 20)
    srv.close()
    small = pcg.Server(context(), budget_bytes=1 << 20)
    x = torch.zeros(1, *ops[0].shape, device="cuda")
    with pytest.raises(pcg.PCError) as e:
        small.submit(ops[0], x, torch.empty_like(x))
    assert e.value.status == pcg.binding.PC_ERR_BUDGET
    with pytest.raises(pcg.PCError):
        small.poll(12345)
    small.close()


def test_autotune_picks_a_valid_shape():
    import paper_1805_06018_gb300 as pcg
    wl = configs.fp32_512(1)
    pts = pcg.pc_sample_points(wl.shape, wl.cells)
    phi = workloads.impulse_windows(wl.shape, pts, wl.kernel)
    best, ms = pcg.pc_autotune(context(), wl.shape, wl.cells, wl.radius, phi, "fp32", nrhs=8)
    assert best["fft_size"] in (64, 128) and ms > 0
    op, orc = make_pair(wl.shape, wl.cells, wl.kernel, "fp32", fft_size=best["fft_size"], tile=best["tile"])
    x = workloads.rhs(3, 2, wl.shape)
    y = op.apply(torch.from_numpy(x).cuda()).cpu().numpy()
    assert np.all(rel_l2(y, orc.apply(x)) <= 1e-5)


def test_3d_requests_in_the_mix(ops):
    """3D operators (FP32 fused and BF16x3 tensor-core) served beside 2D ones:
    3D requests run through their operator's apply on a slot, one launch per operator at a time, and
    every result equals the request applied alone, bit for bit."""
    import paper_1805_06018_gb300 as pcg
    shape = (40, 36, 30)
    cells = workloads.regular_grid(shape, (3, 3, 3))
    kern = workloads.GaussianAxis3D(lambda x: 1.2 + 0.3 * np.sin(x[..., 0] / 7.0), lambda x: 1.6 + 0 * x[..., 0],
                                    lambda x: 1.0 + 0.2 * np.cos(x[..., 2] / 5.0), 5)
    op32 = make_pair(shape, cells, kern, "fp32")[0]
    op16 = make_pair(shape, cells, kern, "bf16x3")[0]
    # runs of 2D requests between the 3D ones: a FIFO queue (no overtaking)
    # merges the 2D requests of a run into one launch
    mix = [ops[0], ops[1], ops[2], op32, op16, ops[1], ops[0], op32, op16, op32]
    srv = pcg.Server(context(), budget_bytes=32 << 30, streams=3, max_requests_per_launch=8)
    rng = np.random.default_rng(1)
    prepared = []
    for q, op in enumerate(mix * 2):
        nrhs = int(rng.integers(1, 7))
        x = torch.from_numpy(workloads.rhs(600 + q, nrhs, op.shape)).cuda()
        prepared.append((op, x, torch.full_like(x, float("nan"))))
    torch.cuda.synchronize()
    jobs = [(op, x, y, srv.submit(op, x, y)) for op, x, y in prepared]
    done = _wait(srv, [j[3] for j in jobs], timeout=120.0)
    for op, x, y, t in jobs:
        alone = op.apply(x)
        torch.cuda.synchronize()
        assert torch.equal(y, alone)
        assert done[t]["status"] == 0
    st = srv.stats()
    assert st["completed"] == len(jobs)
    assert st["launches"] < len(jobs)                 # the 2D requests still share launches
    srv.close()


def test_adjoint_requests_in_the_mix(ops):
    """Adjoint requests (PC_SERVE_ADJOINT, the estimator's probes A~* Z)
    among forward ones, 2D and 3D: runs of one direction share launches, and
    every result equals the request applied alone, bit for bit, BF16x3
    adjoint requests included."""
    import paper_1805_06018_gb300 as pcg
    shape = (30, 28, 26)
    cells = workloads.regular_grid(shape, (3, 3, 3))
    kern = workloads.Skewed([0.7, -0.4, 0.3], lambda x: 1.1 + 0.3 * np.sin(x[..., 0] / 6.0), 4)
    op3 = make_pair(shape, cells, kern, "fp32")[0]
    mix = [(ops[0], True), (ops[1], True), (ops[2], False), (ops[0], False), (op3, True), (ops[1], True),
           (ops[2], True), (op3, False), (ops[0], True), (ops[1], False)]
    srv = pcg.Server(context(), budget_bytes=32 << 30, streams=2, max_requests_per_launch=8)
    rng = np.random.default_rng(2)
    prepared = []
    for q, (op, adj) in enumerate(mix * 2):
        nrhs = int(rng.integers(1, 7))
        x = torch.from_numpy(workloads.rhs(700 + q, nrhs, op.shape)).cuda()
        prepared.append((op, adj, x, torch.full_like(x, float("nan"))))
    torch.cuda.synchronize()
    jobs = [(op, adj, x, y, srv.submit(op, x, y, adjoint=adj)) for op, adj, x, y in prepared]
    done = _wait(srv, [j[4] for j in jobs], timeout=120.0)
    for op, adj, x, y, t in jobs:
        alone = op.apply_adjoint(x) if adj else op.apply(x)
        torch.cuda.synchronize()
        assert torch.equal(y, alone)
        assert done[t]["status"] == 0
    st = srv.stats()
    assert st["launches"] < len(jobs)
    op16 = make_pair(shape, cells, kern, "bf16x3")[0]
    x = torch.from_numpy(workloads.rhs(760, 3, shape)).cuda()
    y = torch.full_like(x, float("nan"))
    t = srv.submit(op16, x, y, adjoint=True)
    done = _wait(srv, [t], timeout=120.0)
    assert done[t]["status"] == 0
    alone = op16.apply_adjoint(x)
    torch.cuda.synchronize()
    assert torch.equal(y, alone)
    srv.close()


def test_early_completions_polled_while_their_launch_runs():
    """Requests that complete early (their last item raises a flag in mapped
    memory) are polled, and so released, while their launch still runs other
    requests; an operator with per-patch shapes runs its requests alone on the
    other slot meanwhile.  The slot keeps each request until its launch ends,
    so nothing it still lists is freed: every result must equal the request
    applied alone."""
    import paper_1805_06018_gb300 as pcg
    shape = (160, 150)
    cells = workloads.quadtree_grid(shape, 1, 4, lambda lo, hi: lo[0] < 50 and lo[1] < 50)
    pp, _ = make_pair(shape, cells, workloads.HeavyTailed(lambda x: 2.0 + 2.0 * (x[..., 0] / 160.0), 30), "fp32",
                      per_patch=True)
    assert pp.info()["num_parts"] >= 2
    small = []
    for shp, npts in [((96, 80), (4, 3)), ((128, 112), (5, 4))]:
        kern = workloads.GaussianAniso2D(lambda x: 1.5 + 0 * x[..., 0], lambda x: 2.0 + np.sin(x[..., 0] / 15.0),
                                         lambda x: 0.3 + 0 * x[..., 0], 8)
        small.append(make_pair(shp, workloads.regular_grid(shp, npts), kern, "fp32", fft_size=128)[0])
    ops = small + [pp]
    srv = pcg.Server(context(), budget_bytes=8 << 30, streams=2, max_requests_per_launch=16)
    rng = np.random.default_rng(3)
    jobs = []
    for q in range(120):
        op = ops[int(rng.integers(0, len(ops)))]
        nrhs = int(rng.integers(1, 9))
        x = torch.from_numpy(workloads.rhs(900 + q, nrhs, op.shape)).cuda()
        jobs.append((op, x, torch.full_like(x, float("nan"))))
    torch.cuda.synchronize()
    pending = {}
    for op, x, y in jobs:
        pending[srv.submit(op, x, y)] = (op, x, y)
        # poll in between submissions: early completions are collected at once
        for t in [t for t in pending if srv.poll(t) is not None]:
            pending.pop(t)
    t0 = time.time()
    while pending:
        for t in [t for t in pending if srv.poll(t) is not None]:
            pending.pop(t)
        assert time.time() - t0 < 120, "requests did not finish"
    srv.close()
    for op, x, y in jobs:
        alone = op.apply(x)
        torch.cuda.synchronize()
        assert torch.equal(y, alone)


def test_solo_requests_share_an_apply():
    """Requests on operators the multi-request kernel does not cover (3D FP32,
    BF16x3, per-patch shapes) queued back to back on the same operator and
    direction share one apply through the slot's staging buffer, up to 64
    right-hand sides: odd and even counts (each block starts at an even
    column, an odd block pairs its last column with a zero one), forward and
    adjoint runs, more right-hand sides than one apply takes.  Every result is
    bitwise the request applied alone, and there are fewer launches than
    requests."""
    import paper_1805_06018_gb300 as pcg
    shape = (40, 36, 30)
    cells = workloads.regular_grid(shape, (3, 3, 3))
    kern = workloads.GaussianAxis3D(lambda x: 1.2 + 0.3 * np.sin(x[..., 0] / 7.0), lambda x: 1.6 + 0 * x[..., 0],
                                    lambda x: 1.0 + 0.2 * np.cos(x[..., 2] / 5.0), 5)
    op32 = make_pair(shape, cells, kern, "fp32")[0]
    op16 = make_pair(shape, cells, kern, "bf16x3")[0]
    shp2 = (160, 150)
    pp = make_pair(shp2, workloads.quadtree_grid(shp2, 1, 4, lambda lo, hi: lo[0] < 50 and lo[1] < 50),
                   workloads.HeavyTailed(lambda x: 2.0 + 2.0 * (x[..., 0] / 160.0), 30), "fp32", per_patch=True)[0]
    assert pp.info()["num_parts"] >= 2
    rng = np.random.default_rng(5)
    plan = []
    for op, n in ((op32, 9), (pp, 8), (op16, 6)):
        for k in range(n):
            adj = op is op32 and k >= 6   # a run of adjoint requests after the forward ones
            plan.append((op, adj, int(rng.integers(1, 14))))
    srv = pcg.Server(context(), budget_bytes=16 << 30, streams=2, max_requests_per_launch=8)
    prepared = []
    for q, (op, adj, nrhs) in enumerate(plan):
        x = torch.from_numpy(workloads.rhs(1100 + q, nrhs, op.shape)).cuda()
        prepared.append((op, adj, x, torch.full_like(x, float("nan"))))
    torch.cuda.synchronize()
    jobs = [(op, adj, x, y, srv.submit(op, x, y, adjoint=adj)) for op, adj, x, y in prepared]
    done = _wait(srv, [j[4] for j in jobs], timeout=120.0)
    st = srv.stats()
    srv.close()
    for op, adj, x, y, t in jobs:
        assert done[t]["status"] == 0
        alone = op.apply_adjoint(x) if adj else op.apply(x)
        torch.cuda.synchronize()
        assert torch.equal(y, alone)
    assert st["completed"] == len(jobs)
    assert st["launches"] < len(jobs)
