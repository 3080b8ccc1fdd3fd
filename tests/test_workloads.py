"""Seeded input generators: SplitMix64 against its published definition,
Box-Muller moments, grid rules."""
import math

import numpy as np

import workloads
from workloads import configs


def _splitmix_scalar(seed, n):
    """Scalar restatement of SplitMix64 (Steele, Lea, Flood 2014) on Python ints."""
    M = (1 << 64) - 1
    x = seed & M
    out = []
    for _ in range(n):
        x = (x + 0x9E3779B97F4A7C15) & M
        z = x
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_matches_scalar_definition():
    for seed in (0, 1, 1234567, 2000, (1 << 63) + 5):
        v = workloads.splitmix64(seed, 0, 50)
        assert [int(a) for a in v] == _splitmix_scalar(seed, 50)
        # counter-based: a window starting mid-stream equals the tail
        w = workloads.splitmix64(seed, 17, 10)
        assert [int(a) for a in w] == _splitmix_scalar(seed, 27)[17:]


def test_splitmix64_seed0_published_vector():
    # First outputs of SplitMix64 seeded with 0, as printed by the reference
    # C implementation (splitmix64.c by S. Vigna, public domain).
    v = workloads.splitmix64(0, 0, 3)
    assert [int(a) for a in v] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_box_muller_moments():
    z = workloads.Stream(7).normal(400_000)
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.01
    assert abs(np.mean(z ** 4) - 3.0) < 0.05


def test_rhs_is_fp32_and_seeded():
    a = workloads.rhs(5, 3, (8, 9))
    b = workloads.rhs(5, 3, (8, 9))
    assert a.dtype == np.float32 and a.shape == (3, 8, 9)
    assert np.array_equal(a, b)


def test_regular_points_include_corners():
    assert workloads.regular_points_1d(64, 4).tolist() == [0, 21, 42, 63]
    p = workloads.regular_points_1d(512, 16)
    assert p[0] == 0 and p[-1] == 511 and len(p) == 16
    assert set(np.diff(p).tolist()) <= {34, 35}
    assert workloads.regular_points_1d(128, 8).tolist() == [0, 18, 36, 54, 73, 91, 109, 127]


def test_adaptive_workload_size():
    wl = configs.adaptive_1024()
    assert len(wl.cells) == 1408
    pts = set()
    for lo, hi in wl.cells:
        for a in (lo[0], hi[0]):
            for b in (lo[1], hi[1]):
                pts.add((int(a), int(b)))
    assert len(pts) == 1579


def test_smooth_field_range():
    f = workloads.SmoothField((64, 64), 2.0, 8.0, 11)
    x = np.stack(np.meshgrid(np.arange(64), np.arange(64), indexing="ij"), -1)
    v = f(x)
    assert v.min() >= 2.0 and v.max() <= 8.0 and v.max() - v.min() > 1.0


def test_impulse_windows_truncation_and_domain():
    kern = workloads.GaussianIso(lambda x: 2.0 + 0 * x[..., 0], 3)
    w = workloads.impulse_windows((10, 10), np.array([[0, 0], [5, 5]]), kern).reshape(2, 7, 7)
    # outside Omega - p is zero (point at the corner)
    assert np.all(w[0, :3, :] == 0) and np.all(w[0, :, :3] == 0)
    # Euclidean truncation |z| <= R, closed
    assert w[1, 0, 3] > 0 and w[1, 0, 0] == 0.0
    assert math.isclose(w[1, 3, 3], 1.0 / (2 * math.pi * 4.0), rel_tol=1e-15)
