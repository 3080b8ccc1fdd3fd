// Harmonic weights on leaves that carry hanging nodes (Section 2.4): 2D
// leaves, and 3D leaves whose broken facets are split into their constituent
// boxes (see harmonic_cell_3d below).
//
// On a leaf C = [0, M] x [0, N] (local coordinates) the weight w_k is the
// discrete-harmonic function (five-point graph Laplacian) whose boundary
// values are linear along every edge segment between consecutive sample
// points, with w_k = delta_kj at the sample points.  We split the boundary
// data g into
//
//   g = b + r,   b = the bilinear interpolant of the four corner values,
//
// b being harmonic with linear edge data, and r vanishing at the corners.
// Each edge's part of r is extended separately, exactly, by separation of
// variables for the discrete operator: along an edge of N intervals the
// discrete sine vectors sin(pi m j / N), m = 1..N-1, diagonalise the 1D
// Laplacian, and each mode decays into the cell as
//
//   S_m(i) = sinh(kappa_m (M - i)) / sinh(kappa_m M),  cosh kappa_m = 2 - cos(pi m / N),
//
// which solves S(i+1) + S(i-1) = (4 - 2 cos(pi m / N)) S(i), S(0) = 1,
// S(M) = 0, i.e. the five-point equation for the mode.  The sinh ratio is
// evaluated as exp(-kappa i) (1 - exp(-2 kappa (M - i))) / (1 - exp(-2 kappa M)).
#include <cmath>
#include <vector>

#include "pc_internal.h"

namespace pc {

namespace {

const double kPi = 3.14159265358979323846264338327950288;

// Add to u (rows 0..M, cols 0..N, row-major (N+1)) the discrete-harmonic
// extension of data h given on one edge and zero on the other three.  `edge`
// 0: row 0, 1: row M, 2: column 0, 3: column N.  h has the edge's length + 1
// values and vanishes at both ends.
void add_edge_solution(std::vector<double> &u, int M, int N, int edge, const std::vector<double> &h) {
    const bool horiz = edge < 2;          // data along a row, decay along columns
    const int L = horiz ? N : M;          // intervals along the edge
    const int D = horiz ? M : N;          // intervals across
    if (L < 2 || D < 1) return;
    std::vector<double> coef(L), sv(L + 1);
    for (int m = 1; m < L; ++m) {
        double acc = 0.0;
        for (int j = 1; j < L; ++j) acc += h[j] * std::sin(kPi * double(m) * double(j) / double(L));
        coef[m] = acc * 2.0 / double(L);
    }
    std::vector<double> decay(D + 1);
    for (int m = 1; m < L; ++m) {
        if (coef[m] == 0.0) continue;
        const double c = 2.0 - std::cos(kPi * double(m) / double(L));
        const double kappa = std::log(c + std::sqrt(c * c - 1.0));
        const double den = 1.0 - std::exp(-2.0 * kappa * double(D));
        for (int d = 0; d <= D; ++d)   // d = distance from the data edge
            decay[d] = std::exp(-kappa * double(d)) * (1.0 - std::exp(-2.0 * kappa * double(D - d))) / den;
        for (int j = 0; j <= L; ++j) sv[j] = coef[m] * std::sin(kPi * double(m) * double(j) / double(L));
        for (int d = 1; d < D; ++d) {      // interior rows/columns only; the boundary is set separately
            const double f = decay[d];
            for (int j = 1; j < L; ++j) {
                int i0, j0;
                if (edge == 0) { i0 = d; j0 = j; }
                else if (edge == 1) { i0 = M - d; j0 = j; }
                else if (edge == 2) { i0 = j; j0 = d; }
                else { i0 = j; j0 = N - d; }
                u[size_t(i0) * (N + 1) + j0] += f * sv[j];
            }
        }
    }
}

}  // namespace

// The discrete-harmonic function on the rectangle [0, M] x [0, N] (row-major,
// N + 1 columns) with edge data e[0] (row 0), e[1] (row M), e[2] (column 0),
// e[3] (column N), each with its edge's length + 1 values.
pc_status harmonic_rect_2d(int M, int N, const std::vector<double> (&e)[4], std::vector<double> &vals,
                           std::string &err) {
    vals.assign(size_t(M + 1) * (N + 1), 0.0);
    if (e[0].size() != size_t(N + 1) || e[2].size() != size_t(M + 1) || e[0][0] != e[2][0] || e[0][N] != e[3][0] ||
        e[1][0] != e[2][M] || e[1][N] != e[3][M]) {
        err = "inconsistent corner values";
        return PC_ERR_GRID;
    }
    const double c00 = e[0][0], c0N = e[0][N], cM0 = e[1][0], cMN = e[1][N];
    // bilinear part everywhere
    for (int i = 0; i <= M; ++i)
        for (int j = 0; j <= N; ++j) {
            const double s = double(i) / double(M), t = double(j) / double(N);
            vals[size_t(i) * (N + 1) + j] =
                (1 - s) * (1 - t) * c00 + (1 - s) * t * c0N + s * (1 - t) * cM0 + s * t * cMN;
        }
    // residual edge data and its harmonic extension
    for (int q = 0; q < 4; ++q) {
        const bool horiz = q < 2;
        const int L = horiz ? N : M;
        std::vector<double> r(L + 1);
        bool nonzero = false;
        for (int s = 0; s <= L; ++s) {
            const int i = horiz ? (q == 0 ? 0 : M) : s;
            const int j = horiz ? s : (q == 2 ? 0 : N);
            r[s] = e[q][s] - vals[size_t(i) * (N + 1) + j];
            if (s > 0 && s < L && r[s] != 0.0) nonzero = true;
        }
        r[0] = r[L] = 0.0;
        if (nonzero) add_edge_solution(vals, M, N, q, r);
    }
    // boundary values exactly as prescribed
    for (int s = 0; s <= N; ++s) {
        vals[s] = e[0][s];
        vals[size_t(M) * (N + 1) + s] = e[1][s];
    }
    for (int s = 0; s <= M; ++s) {
        vals[size_t(s) * (N + 1)] = e[2][s];
        vals[size_t(s) * (N + 1) + N] = e[3][s];
    }
    return PC_OK;
}

namespace {

// w_k = delta_kj at the sample points of leaf c; is_node says whether x is one
double node_value(const Geometry &g, int c, int k, const I3 &x, bool &is_node) {
    for (int j : g.points_of[c])
        if (g.pts[j][0] == x[0] && g.pts[j][1] == x[1] && g.pts[j][2] == x[2]) {
            is_node = true;
            return j == k ? 1.0 : 0.0;
        }
    is_node = false;
    return 0.0;
}

// Values on the segment from x0 along axis f (len + 1 points): linear between
// consecutive sample points of leaf c (the 1D discrete Laplace solution);
// both ends must be sample points.
bool segment_values(const Geometry &g, int c, int k, I3 x0, int f, int len, std::vector<double> &v) {
    v.assign(size_t(len) + 1, 0.0);
    std::vector<int> nodes;
    for (int s = 0; s <= len; ++s) {
        I3 x = x0;
        x[size_t(f)] += s;
        bool is_node = false;
        const double nv = node_value(g, c, k, x, is_node);
        if (is_node) {
            v[size_t(s)] = nv;
            nodes.push_back(s);
        }
    }
    if (nodes.empty() || nodes.front() != 0 || nodes.back() != len) return false;
    for (size_t q = 0; q + 1 < nodes.size(); ++q) {
        const int s0 = nodes[q], s1 = nodes[q + 1];
        for (int s = s0 + 1; s < s1; ++s)
            v[size_t(s)] = v[size_t(s0)] + (v[size_t(s1)] - v[size_t(s0)]) * double(s - s0) / double(s1 - s0);
    }
    return true;
}

// Orthonormal DST-I matrix of size m: S_ij = sqrt(2/(m+1)) sin(pi i j/(m+1)), i, j = 1..m
void dst_matrix(int m, std::vector<double> &S, std::vector<double> &lam) {
    S.assign(size_t(m) * m, 0.0);
    lam.assign(size_t(m), 0.0);
    const double f = std::sqrt(2.0 / double(m + 1));
    for (int i = 0; i < m; ++i) {
        lam[size_t(i)] = 2.0 - 2.0 * std::cos(kPi * double(i + 1) / double(m + 1));
        for (int j = 0; j < m; ++j) S[size_t(i) * m + j] = f * std::sin(kPi * double(i + 1) * double(j + 1) / double(m + 1));
    }
}

// Replace the interior of the box u (extents E0 x E1 x E2, row-major) by the
// solution of the discrete Laplace equation (seven-point graph Laplacian)
// whose boundary layer holds the Dirichlet data.  The Kronecker-sum operator
// is diagonal in the product of the DST-I bases of the three axes.
void dirichlet_box_3d(std::vector<double> &u, const int64_t E[3]) {
    const int m0 = int(E[0]) - 2, m1 = int(E[1]) - 2, m2 = int(E[2]) - 2;
    if (m0 <= 0 || m1 <= 0 || m2 <= 0) return;
    auto at = [&](int64_t i, int64_t j, int64_t l) -> double & { return u[size_t((i * E[1] + j) * E[2] + l)]; };
    // right-hand side: the boundary neighbours of every interior node
    std::vector<double> b(size_t(m0) * m1 * m2, 0.0);
    auto B = [&](int i, int j, int l) -> double & { return b[size_t((size_t(i) * m1 + j) * m2 + l)]; };
    for (int i = 0; i < m0; ++i)
        for (int j = 0; j < m1; ++j)
            for (int l = 0; l < m2; ++l) {
                double acc = 0.0;
                if (i == 0) acc += at(0, j + 1, l + 1);
                if (i == m0 - 1) acc += at(m0 + 1, j + 1, l + 1);
                if (j == 0) acc += at(i + 1, 0, l + 1);
                if (j == m1 - 1) acc += at(i + 1, m1 + 1, l + 1);
                if (l == 0) acc += at(i + 1, j + 1, 0);
                if (l == m2 - 1) acc += at(i + 1, j + 1, m2 + 1);
                B(i, j, l) = acc;
            }
    std::vector<double> S0, S1, S2, l0, l1, l2;
    dst_matrix(m0, S0, l0);
    dst_matrix(m1, S1, l1);
    dst_matrix(m2, S2, l2);
    // apply S along each axis (S is symmetric and its own inverse)
    auto transform = [&](std::vector<double> &x) {
        std::vector<double> t(x.size());
        for (int i = 0; i < m0; ++i)        // axis 2
            for (int j = 0; j < m1; ++j)
                for (int l = 0; l < m2; ++l) {
                    double acc = 0.0;
                    for (int q = 0; q < m2; ++q) acc += S2[size_t(l) * m2 + q] * x[size_t((size_t(i) * m1 + j) * m2 + q)];
                    t[size_t((size_t(i) * m1 + j) * m2 + l)] = acc;
                }
        for (int i = 0; i < m0; ++i)        // axis 1
            for (int j = 0; j < m1; ++j)
                for (int l = 0; l < m2; ++l) {
                    double acc = 0.0;
                    for (int q = 0; q < m1; ++q) acc += S1[size_t(j) * m1 + q] * t[size_t((size_t(i) * m1 + q) * m2 + l)];
                    x[size_t((size_t(i) * m1 + j) * m2 + l)] = acc;
                }
        for (int i = 0; i < m0; ++i)        // axis 0
            for (int j = 0; j < m1; ++j)
                for (int l = 0; l < m2; ++l) {
                    double acc = 0.0;
                    for (int q = 0; q < m0; ++q) acc += S0[size_t(i) * m0 + q] * x[size_t((size_t(q) * m1 + j) * m2 + l)];
                    t[size_t((size_t(i) * m1 + j) * m2 + l)] = acc;
                }
        x.swap(t);
    };
    transform(b);
    for (int i = 0; i < m0; ++i)
        for (int j = 0; j < m1; ++j)
            for (int l = 0; l < m2; ++l) B(i, j, l) /= l0[size_t(i)] + l1[size_t(j)] + l2[size_t(l)];
    transform(b);
    for (int i = 0; i < m0; ++i)
        for (int j = 0; j < m1; ++j)
            for (int l = 0; l < m2; ++l) at(i + 1, j + 1, l + 1) = B(i, j, l);
}

}  // namespace

pc_status harmonic_cell_2d(const Geometry &g, int c, int k, std::vector<double> &vals, std::string &err) {
    const I3 &lo = g.cell_lo[c], &hi = g.cell_hi[c];
    const int M = int(hi[0] - lo[0]), N = int(hi[1] - lo[1]);
    // piecewise-linear edge data between consecutive sample points
    std::vector<double> e[4];
    const I3 starts[4] = {{lo[0], lo[1], 0}, {hi[0], lo[1], 0}, {lo[0], lo[1], 0}, {lo[0], hi[1], 0}};
    for (int q = 0; q < 4; ++q)
        if (!segment_values(g, c, k, starts[q], q < 2 ? 1 : 0, q < 2 ? N : M, e[q])) {
            err = "edge ends must be sample points";
            return PC_ERR_GRID;
        }
    return harmonic_rect_2d(M, N, e, vals, err);
}

pc_status harmonic_cell_3d(const Geometry &g, int c, int k, std::vector<double> &vals, std::string &err) {
    const I3 &lo = g.cell_lo[c], &hi = g.cell_hi[c];
    const int64_t E[3] = {hi[0] - lo[0] + 1, hi[1] - lo[1] + 1, hi[2] - lo[2] + 1};
    vals.assign(size_t(E[0] * E[1] * E[2]), 0.0);
    std::vector<double> piece, e[4];
    for (int a = 0; a < 3; ++a) {
        const int b1 = a == 0 ? 1 : 0, b2 = a == 2 ? 1 : 2;   // the facet's axes, ascending
        for (int side = 0; side < 2; ++side) {
            const int64_t plane = side ? hi[a] : lo[a];
            // the facet's constituent boxes (Section 2.4): the facet itself on the
            // boundary of Omega, else its intersections with the leaves across it
            std::vector<std::pair<I3, I3>> pieces;
            I3 flo = lo, fhi = hi;
            flo[size_t(a)] = fhi[size_t(a)] = plane;
            if ((side == 0 && plane == 0) || (side == 1 && plane == g.shape[size_t(a)] - 1)) {
                pieces.push_back({flo, fhi});
            } else {
                int64_t area = 0;
                for (int n = 0; n < int(g.cell_lo.size()); ++n) {
                    if (n == c) continue;
                    if (side ? g.cell_lo[n][a] != plane : g.cell_hi[n][a] != plane) continue;
                    I3 plo = flo, phi = fhi;
                    for (int b : {b1, b2}) {
                        plo[size_t(b)] = std::max(lo[b], g.cell_lo[n][b]);
                        phi[size_t(b)] = std::min(hi[b], g.cell_hi[n][b]);
                    }
                    if (plo[size_t(b1)] < phi[size_t(b1)] && plo[size_t(b2)] < phi[size_t(b2)]) {
                        pieces.push_back({plo, phi});
                        area += (phi[size_t(b1)] - plo[size_t(b1)]) * (phi[size_t(b2)] - plo[size_t(b2)]);
                    }
                }
                if (area != (hi[b1] - lo[b1]) * (hi[b2] - lo[b2])) {
                    err = "the leaves across a facet do not tile it";
                    return PC_ERR_GRID;
                }
            }
            for (const auto &pp : pieces) {
                const I3 &plo = pp.first, &phi = pp.second;
                const int M = int(phi[size_t(b1)] - plo[size_t(b1)]), N = int(phi[size_t(b2)] - plo[size_t(b2)]);
                I3 s0 = plo, s1 = plo, s2 = plo, s3 = plo;
                s1[size_t(b1)] = phi[size_t(b1)];   // row M
                s3[size_t(b2)] = phi[size_t(b2)];   // column N
                if (!segment_values(g, c, k, s0, b2, N, e[0]) || !segment_values(g, c, k, s1, b2, N, e[1]) ||
                    !segment_values(g, c, k, s2, b1, M, e[2]) || !segment_values(g, c, k, s3, b1, M, e[3])) {
                    err = "facet piece corners must be sample points";
                    return PC_ERR_GRID;
                }
                pc_status st = harmonic_rect_2d(M, N, e, piece, err);
                if (st != PC_OK) return st;
                for (int i = 0; i <= M; ++i)
                    for (int j = 0; j <= N; ++j) {
                        I3 x = plo;
                        x[size_t(b1)] += i;
                        x[size_t(b2)] += j;
                        vals[size_t(((x[0] - lo[0]) * E[1] + (x[1] - lo[1])) * E[2] + (x[2] - lo[2]))] =
                            piece[size_t(i) * (N + 1) + j];
                    }
            }
        }
    }
    dirichlet_box_3d(vals, E);
    return PC_OK;
}

}  // namespace pc
