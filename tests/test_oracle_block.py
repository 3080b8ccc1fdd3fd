"""Oracle block apply (Section 3.3) against what the paper and the mathematics fix.

* the translation identity (phi * f)[T] = (phi_0 * f_0)[T'] against brute-force
  sums on tiny 1D/2D/3D boxes (targets inside, overlapping, beside and far
  from the sources; G inside, across and outside the kernel window);
* the per-term translated evaluation against the definition (zero-extended
  direct-sum apply, restricted) and against the dense entry matrix
  (Eq. conv_matrix_entries) restricted to rows T and columns S;
* duality <A~[T,S] f, g> = <f, (A~*)[S,T] g> and additivity over a split of S;
* planted mistakes (terms chosen by T instead of S, an unflipped kernel in the
  adjoint, an off-by-one T') fail these pins.
"""
from itertools import product

import numpy as np
import pytest

import workloads
from oracle import Grid, PCOracle
from oracle import block as ob
from oracle.dense import dense_pc

from test_oracle_geometry import ADAPTIVE_CELLS, ADAPTIVE_SHAPE

CASES = [
    ("1d", (23,), workloads.regular_grid((23,), (4,))),
    ("2d", (14, 17), workloads.regular_grid((14, 17), (3, 4))),
    ("2d-adaptive", ADAPTIVE_SHAPE, np.array(ADAPTIVE_CELLS)),
    ("3d", (7, 8, 6), workloads.regular_grid((7, 8, 6), (3, 3, 2))),
]


def _oracle(shape, cells, R=3):
    d = len(shape)
    L = float(max(shape))
    kern = workloads.Skewed([0.7, -0.4, 0.3][:d], lambda x: 1.1 + 0.5 * np.sin(2 * np.pi * x[..., 0] / L), R)
    g = Grid(shape, cells)
    return PCOracle(shape, cells, workloads.impulse_windows(shape, g.points, kern), R)


def _boxes(shape, rng, n):
    out = []
    for _ in range(n):
        lo, hi = [], []
        for m in shape:
            a, b = sorted(rng.integers(0, m, 2))
            lo.append(int(a))
            hi.append(int(b))
        out.append((np.array(lo), np.array(hi)))
    return out


def _brute(phi_win, R, f, s_lo, s_hi, t_lo, t_hi):
    d = len(s_lo)
    w = phi_win.reshape((2 * R + 1,) * d)
    nT = tuple(int(b - a + 1) for a, b in zip(t_lo, t_hi))
    out = np.zeros(nT)
    for t in product(*[range(a, b + 1) for a, b in zip(t_lo, t_hi)]):
        acc = 0.0
        for s in product(*[range(a, b + 1) for a, b in zip(s_lo, s_hi)]):
            z = np.array(t) - np.array(s)
            if np.all(np.abs(z) <= R):
                acc += f[tuple(np.array(s) - s_lo)] * w[tuple(z + R)]
        out[tuple(np.array(t) - t_lo)] = acc
    return out


@pytest.mark.parametrize("d", [1, 2, 3])
def test_translation_identity_brute_force(d):
    rng = np.random.default_rng(40 + d)
    R = 2
    shape = (19, 13, 9)[:d]
    phi = rng.standard_normal((2 * R + 1) ** d)
    for (s_lo, s_hi), (t_lo, t_hi) in zip(_boxes(shape, rng, 12), _boxes(shape, rng, 12)):
        f = rng.standard_normal(tuple(s_hi - s_lo + 1))
        got = ob.translated_convolution(phi, R, f, s_lo, s_hi, t_lo, t_hi)
        ref = _brute(phi, R, f, s_lo, s_hi, t_lo, t_hi)
        assert got.shape == ref.shape
        assert np.max(np.abs(got - ref)) <= 1e-12 * max(1.0, np.abs(ref).max())


def test_translation_identity_far_and_adjacent_boxes():
    rng = np.random.default_rng(44)
    R = 3
    phi = rng.standard_normal(2 * R + 1)
    f = rng.standard_normal(5)
    # T beyond the kernel's reach: zero; T touching S at distance R: one term
    assert np.all(ob.translated_convolution(phi, R, f, [10], [14], [18], [25]) == 0)
    y = ob.translated_convolution(phi, R, f, [10], [14], [17], [17])
    assert np.isclose(y[0], f[4] * phi[2 * R])


@pytest.mark.parametrize("name,shape,cells", CASES)
@pytest.mark.parametrize("adjoint", [False, True])
def test_translated_terms_equal_the_definition(name, shape, cells, adjoint):
    orc = _oracle(shape, cells)
    rng = np.random.default_rng(50)
    for (t_lo, t_hi), (s_lo, s_hi) in zip(_boxes(shape, rng, 5), _boxes(shape, rng, 5)):
        x = rng.standard_normal((2,) + tuple(s_hi - s_lo + 1))
        a = ob.apply_block(orc, t_lo, t_hi, s_lo, s_hi, x, adjoint)
        b = ob.apply_block_translated(orc, t_lo, t_hi, s_lo, s_hi, x, adjoint)
        assert np.max(np.abs(a - b)) <= 1e-12 * max(1.0, np.abs(a).max())


def _flat(shape, lo, hi):
    idx = np.arange(int(np.prod(shape))).reshape(shape)
    return idx[tuple(slice(int(a), int(b) + 1) for a, b in zip(lo, hi))].ravel()


@pytest.mark.parametrize("name,shape,cells", CASES[:3])
def test_block_is_the_dense_submatrix(name, shape, cells):
    orc = _oracle(shape, cells)
    A = dense_pc(orc)
    rng = np.random.default_rng(51)
    for (t_lo, t_hi), (s_lo, s_hi) in zip(_boxes(shape, rng, 6), _boxes(shape, rng, 6)):
        rows, cols = _flat(shape, t_lo, t_hi), _flat(shape, s_lo, s_hi)
        x = rng.standard_normal(len(cols))
        y = ob.apply_block_translated(orc, t_lo, t_hi, s_lo, s_hi, x).ravel()
        ya = ob.apply_block_translated(orc, t_lo, t_hi, s_lo, s_hi, x, adjoint=True).ravel()
        ref = A[np.ix_(rows, cols)] @ x
        refa = A.T[np.ix_(rows, cols)] @ x
        assert np.max(np.abs(y - ref)) <= 1e-12 * max(1.0, np.abs(ref).max())
        assert np.max(np.abs(ya - refa)) <= 1e-12 * max(1.0, np.abs(refa).max())


@pytest.mark.parametrize("name,shape,cells", CASES)
def test_duality_and_additivity(name, shape, cells):
    orc = _oracle(shape, cells)
    rng = np.random.default_rng(52)
    for (t_lo, t_hi), (s_lo, s_hi) in zip(_boxes(shape, rng, 4), _boxes(shape, rng, 4)):
        f = rng.standard_normal(tuple(s_hi - s_lo + 1))
        g = rng.standard_normal(tuple(t_hi - t_lo + 1))
        Af = ob.apply_block_translated(orc, t_lo, t_hi, s_lo, s_hi, f)[0]
        Atg = ob.apply_block_translated(orc, s_lo, s_hi, t_lo, t_hi, g, adjoint=True)[0]
        lhs, rhs = np.sum(Af * g), np.sum(f * Atg)
        assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Af) * np.linalg.norm(g) + 1e-300
        # split S along axis 0 (when it has two or more layers)
        if s_hi[0] > s_lo[0]:
            m = (s_lo[0] + s_hi[0]) // 2
            hi_a = s_hi.copy()
            hi_a[0] = m
            lo_b = s_lo.copy()
            lo_b[0] = m + 1
            fa, fb = f[: m - s_lo[0] + 1], f[m - s_lo[0] + 1:]
            parts = (ob.apply_block_translated(orc, t_lo, t_hi, s_lo, hi_a, fa)[0] +
                     ob.apply_block_translated(orc, t_lo, t_hi, lo_b, s_hi, fb)[0])
            assert np.max(np.abs(parts - Af)) <= 1e-12 * max(1.0, np.abs(Af).max())


def test_planted_mistakes_fail(monkeypatch):
    shape, cells = CASES[2][1], CASES[2][2]
    orc = _oracle(shape, cells)
    rng = np.random.default_rng(53)
    t_lo, t_hi = np.array([0, 0]), np.array([9, 7])
    s_lo, s_hi = np.array([6, 5]), np.array([15, 12])
    x = rng.standard_normal((1, 10, 8))
    ref = ob.apply_block(orc, t_lo, t_hi, s_lo, s_hi, x)
    refa = ob.apply_block(orc, t_lo, t_hi, s_lo, s_hi, x, adjoint=True)

    def far(a, b):
        return np.max(np.abs(a - b)) > 1e-6 * np.abs(b).max()

    real_terms = ob.block_terms
    # terms chosen by T for the forward block
    monkeypatch.setattr(ob, "block_terms", lambda o, tl, th, sl, sh, adj=False: real_terms(o, tl, th, sl, sh, not adj))
    assert far(ob.apply_block_translated(orc, t_lo, t_hi, s_lo, s_hi, x), ref)
    monkeypatch.setattr(ob, "block_terms", real_terms)
    # T' off by one
    real_tc = ob.translated_convolution

    def shifted(phi, R, f, sl, sh, tl, th):
        return real_tc(phi, R, f, sl, sh, np.asarray(tl) + 1, np.asarray(th) + 1)
    monkeypatch.setattr(ob, "translated_convolution", shifted)
    assert far(ob.apply_block_translated(orc, t_lo, t_hi, s_lo, s_hi, x), ref)
    monkeypatch.setattr(ob, "translated_convolution", real_tc)
    # the adjoint with an unflipped kernel (the window is asymmetric)

    def unflipped(phi, R, f, sl, sh, tl, th):
        return real_tc(phi[(slice(None, None, -1),) * phi.ndim], R, f, sl, sh, tl, th)
    monkeypatch.setattr(ob, "translated_convolution", unflipped)
    assert far(ob.apply_block_translated(orc, t_lo, t_hi, s_lo, s_hi, x, adjoint=True), refa)
