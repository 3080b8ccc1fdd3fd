// Harmonic weights on 2D leaves that carry hanging nodes (Section 2.4).
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

pc_status harmonic_cell_2d(const Geometry &g, int c, int k, std::vector<double> &vals, std::string &err) {
    const I3 &lo = g.cell_lo[c], &hi = g.cell_hi[c];
    const int M = int(hi[0] - lo[0]), N = int(hi[1] - lo[1]);
    vals.assign(size_t(M + 1) * (N + 1), 0.0);
    // node values on the boundary: delta_kj at the sample points of the leaf
    auto node_value = [&](int64_t a0, int64_t a1, bool &is_node) {
        for (int j : g.points_of[c])
            if (g.pts[j][0] == a0 && g.pts[j][1] == a1) {
                is_node = true;
                return j == k ? 1.0 : 0.0;
            }
        is_node = false;
        return 0.0;
    };
    // piecewise-linear edge data between consecutive sample points
    auto edge_data = [&](int edge) {
        const bool horiz = edge < 2;
        const int L = horiz ? N : M;
        std::vector<double> v(L + 1, 0.0);
        std::vector<int> nodes;
        for (int s = 0; s <= L; ++s) {
            const int64_t a0 = horiz ? (edge == 0 ? lo[0] : hi[0]) : lo[0] + s;
            const int64_t a1 = horiz ? lo[1] + s : (edge == 2 ? lo[1] : hi[1]);
            bool is_node = false;
            const double nv = node_value(a0, a1, is_node);
            if (is_node) {
                v[s] = nv;
                nodes.push_back(s);
            }
        }
        for (size_t q = 0; q + 1 < nodes.size(); ++q) {
            const int s0 = nodes[q], s1 = nodes[q + 1];
            for (int s = s0 + 1; s < s1; ++s)
                v[s] = v[s0] + (v[s1] - v[s0]) * double(s - s0) / double(s1 - s0);
        }
        return v;
    };
    std::vector<double> e[4];
    for (int q = 0; q < 4; ++q) e[q] = edge_data(q);
    if (e[0].empty() || e[0][0] != e[2][0] || e[0][N] != e[3][0] || e[1][0] != e[2][M] || e[1][N] != e[3][M]) {
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

}  // namespace pc
