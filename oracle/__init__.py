"""FP64 CPU oracle for the adaptive product-convolution operator.

TEST INFRASTRUCTURE.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import or run anything in this package.
The library's product path never calls it, and the two share no code: the
only shared module is ``workloads`` (seeded inputs, no method arithmetic).

What it computes, step by step, in the paper's order and notation:

1. Grid (Section 2.2): sample points {p_k} = corners of the leaf cells,
   cells(p_k) by closed containment, blocky neighbourhoods U_k, nbrs(k).
   -> :mod:`oracle.grid`
2. Harmonic partition-of-unity weights w_k (Section 2.4): vertex values
   delta_kj, piecewise-linear edges (1D Laplace), then the discrete Laplace
   equation (graph Laplacian) on each face / cell with Dirichlet data, solved
   exactly in a sine eigenbasis.  -> :mod:`oracle.weights`
3. Extended impulse responses phi_k^E (Section 2.5): counting functions c_k,
   v_k = 1/c_k, v_k^(j) (Eq. vj_def) and phi_k^E = sum_j v_k^(j) phi_j
   (Eq. def_varphiE).  -> :mod:`oracle.extension`
4. Apply (Eq. conv_op_approx_main with the convolution of Eq.
   convolution_definition) by direct summation, plain C with OpenMP over
   output points only: for each y, for k ascending, for x in bbox(U_k) with
   y - x in the window [-R, R]^d: acc += (w_k[x] f[x]) phi_k^E[y - x] (the
   impulse responses vanish outside |z|_2 <= R).  -> :mod:`oracle.apply`
5. Tiny boxes: dense A~ from the entry formula (Eq. conv_matrix_entries),
   W_k (Eq. Wj_def), F_k (Eq. translation_failure_operator), F (Eq.
   defn_of_F) and the sets mu_k^E (Eq. skew_cylinder_set).  -> :mod:`oracle.dense`
6. Blocks A~[T, S] and (A~*)[T, S] applied to vectors (Section 3.3): the
   restricted definition, and the translated small convolution per term.
   -> :mod:`oracle.block`
7. The randomized a-posteriori estimator (Section 2.6, Eq.
   randomized_estimator_ec): eta_C from A~* Z and the caller's Y = A* Z.
   -> :mod:`oracle.estimator`
8. The adaptive construction (Algorithm 1) with anisotropic splits (Section
   2.7).  -> :mod:`oracle.adaptive`

Readings where the paper is silent (each one is listed with its reason in the
design notes): n-point regular grids include the box corners, midpoints round
down, truncation is Euclidean |y - x|_2 <= R, a neighbour contributes to the
extension wherever its domain Omega - p_j contains z (Section 1.3's meaning of
support), the extension uses the plain average, data are real, the oracle
consumes the FP32-rounded right-hand side promoted to FP64, and in 3D a split
that would break a facet crosswise (its pieces meeting at a point that is no
cell's corner, where Section 2.4's recursion gives no value) is skipped for
the cell's next direction.

Parity pins: every function here is checked by the ``-m "not gpu"`` tests
against closed forms and invariants the paper fixes (partition of unity,
delta property, bilinear/trilinear hats on conforming cells, discrete
harmonicity, Lemma 4.1, Lemma 4.2, Proposition 4.3, Proposition 4.4,
Theorem 4.5, exactness at sample points, exact reproduction of a
translation-invariant operator against an independent library convolution,
A~ = A when every point is a sample point, and entry-formula vs direct-sum
agreement).  3D leaves with hanging nodes take their weights through the
pieces of their broken facets (Section 2.4), pinned by harmonicity on every
leaf and piece, partition of unity and agreement across shared facets.
"""
from .grid import Grid  # noqa: F401
from .weights import harmonic_weights  # noqa: F401
from .extension import extend_impulse_responses  # noqa: F401
from .apply import PCOracle  # noqa: F401
