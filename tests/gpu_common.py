"""Shared helpers for the GPU tests: build a library operator and the oracle
from the same seeded workload, and compare per right-hand side."""
import numpy as np

import workloads
from oracle import Grid, PCOracle

_CTX = None


def context():
    global _CTX
    import paper_1805_06018_gb300 as pcg
    from paper_1805_06018_gb300 import build
    if _CTX is None:
        build.build()
        _CTX = pcg.Context(0)
    return _CTX


def make_pair(shape, cells, kernel, precision="fp32", **tune):
    """(library operator, oracle) for one operator.  Both sides compute their
    own sample points; the impulse windows come from the shared generator."""
    import paper_1805_06018_gb300 as pcg
    g = Grid(shape, cells)
    pts_lib = pcg.pc_sample_points(shape, cells)
    assert np.array_equal(pts_lib, g.points)
    phi = workloads.impulse_windows(shape, pts_lib, kernel)
    op = pcg.Operator(context(), shape, cells, kernel.radius, phi, precision=precision, **tune)
    orc = PCOracle(shape, cells, workloads.impulse_windows(shape, g.points, kernel), kernel.radius)
    return op, orc


def rel_l2(got, ref):
    """Relative l2 error per right-hand side: ||got - ref|| / ||ref||."""
    got = np.asarray(got, dtype=np.float64).reshape(len(ref), -1)
    ref = np.asarray(ref, dtype=np.float64).reshape(len(ref), -1)
    return np.linalg.norm(got - ref, axis=1) / np.linalg.norm(ref, axis=1)


def run(op, x_np, plain=False):
    import torch
    dt = torch.float64 if op.precision == "fp64" else torch.float32
    x = torch.from_numpy(np.ascontiguousarray(x_np)).to(device="cuda", dtype=dt)
    y = op.apply_plain(x) if plain else op.apply(x)
    torch.cuda.synchronize()
    op.check()
    return y.cpu().numpy()
