// Refinement step of the adaptive construction (Algorithm 1, Section 2.7),
// host code: the overall estimate eta_Omega, the choice of leaves by eta_C,
// the subdivision direction of largest change of phi^E, and (3D) the check
// that a split keeps every facet piece's corners at sample points.
//
//   eta_Omega = sqrt(sum_C eta_C^2) / y_rms,  y_rms = ||Y||_F / sqrt(q)
//
// (the overall estimator of Algorithm 1 as a relative estimate; a point on a
// shared facet counts in each leaf that holds it).  Direction of a leaf
// C = [c_min, c_max]: among the axes i with c_max^i - c_min^i > 2, the one
// that maximises || phi^{i+} - phi^{i-} || over the window offsets z with
// c_mid + z in Omega, where phi^{i+-} averages phi_k^E over the 2^{d-1}
// corners of C on its front / back face along i; values within a relative
// 1e-9 of the largest are a tie, won by the lowest axis.  The split is at
// floor((c_min + c_max) / 2).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "pc_api_util.h"
#include "pc_internal.h"

using pc::fail;

namespace {

using Box = std::pair<pc::I3, pc::I3>;   // closed leaf box (lo, hi); unused axes 0

int point_index(const pc::Geometry &g, const pc::I3 &p) {
    const auto it = std::lower_bound(g.pts.begin(), g.pts.end(), p);
    return it != g.pts.end() && *it == p ? int(it - g.pts.begin()) : -1;
}

// Axes of leaf c, best first (Section 2.7); phiE [r][(2R+1)^d].
std::vector<int> split_directions(const pc::Geometry &g, int R, const std::vector<double> &phiE, int c) {
    const int d = g.d;
    const int64_t W = 2 * R + 1;
    int64_t wsz = 1;
    for (int a = 0; a < d; ++a) wsz *= W;
    const pc::I3 &lo = g.cell_lo[c], &hi = g.cell_hi[c];
    int64_t cmid[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) cmid[a] = (lo[a] + hi[a]) / 2;
    // offsets z (C order over [-R, R]^d) with c_mid + z inside the box
    std::vector<char> mask(size_t(wsz), 1);
    for (int64_t q = 0; q < wsz; ++q) {
        int64_t rest = q;
        for (int a = d - 1; a >= 0; --a) {
            const int64_t z = rest % W - R;
            rest /= W;
            if (cmid[a] + z < 0 || cmid[a] + z >= g.shape[a]) mask[size_t(q)] = 0;
        }
    }
    const double scale = std::ldexp(1.0, 1 - d);
    std::vector<std::pair<int, double>> scores;
    for (int i = 0; i < d; ++i) {
        if (hi[i] - lo[i] <= 2) continue;
        std::vector<double> front(size_t(wsz), 0.0), back(size_t(wsz), 0.0);
        // corners in lexicographic order of (lo/hi per axis), lo first
        for (int bits = 0; bits < (1 << d); ++bits) {
            pc::I3 p{0, 0, 0};
            for (int a = 0; a < d; ++a) p[a] = (bits >> (d - 1 - a)) & 1 ? hi[a] : lo[a];
            const int k = point_index(g, p);
            if (k < 0) continue;   // corners of a leaf are sample points (Section 2.2)
            std::vector<double> &acc = p[i] == hi[i] ? front : back;
            const double *ph = phiE.data() + size_t(k) * size_t(wsz);
            for (int64_t q = 0; q < wsz; ++q) acc[size_t(q)] += ph[q];
        }
        double ss = 0.0;
        for (int64_t q = 0; q < wsz; ++q)
            if (mask[size_t(q)]) {
                const double v = (front[size_t(q)] - back[size_t(q)]) * scale;
                ss += v * v;
            }
        scores.push_back({i, std::sqrt(ss)});
    }
    std::vector<int> out;
    while (!scores.empty()) {
        double top = 0.0;
        for (const auto &sv : scores) top = std::max(top, sv.second);
        size_t pick = 0;
        for (size_t j = 0; j < scores.size(); ++j)
            if (scores[j].second >= top - 1e-9 * top) {
                pick = j;   // lowest axis first: scores are in axis order
                break;
            }
        out.push_back(scores[pick].first);
        scores.erase(scores.begin() + long(pick));
    }
    return out;
}

// leaves with `box` replaced by its halves along axis i (the halves last)
std::vector<Box> split_leaf(const std::vector<Box> &cells, const Box &box, int i) {
    const int64_t m = (box.first[i] + box.second[i]) / 2;
    std::vector<Box> out;
    for (const Box &c : cells)
        if (!(c == box)) out.push_back(c);
    Box a = box, b = box;
    a.second[i] = m;
    b.first[i] = m;
    out.push_back(a);
    out.push_back(b);
    return out;
}

// Whether every facet piece of the leaves `fresh` (their facets' intersections
// of positive area with the facets of the leaves across) has leaf corners at
// its corners.  Pieces away from them are unchanged by a split.
bool pieces_end_at_points(const std::vector<Box> &cells, const std::vector<Box> &fresh, int d) {
    std::vector<pc::I3> corners;
    for (const Box &c : cells)
        for (int bits = 0; bits < (1 << d); ++bits) {
            pc::I3 p{0, 0, 0};
            for (int a = 0; a < d; ++a) p[a] = (bits >> a) & 1 ? c.second[a] : c.first[a];
            corners.push_back(p);
        }
    std::sort(corners.begin(), corners.end());
    corners.erase(std::unique(corners.begin(), corners.end()), corners.end());
    auto is_corner = [&](const pc::I3 &p) { return std::binary_search(corners.begin(), corners.end(), p); };
    for (const Box &bx : fresh)
        for (int a = 0; a < d; ++a)
            for (int far = 1; far >= 0; --far) {
                const int64_t plane = far ? bx.first[a] : bx.second[a];
                for (const Box &n : cells) {
                    // a leaf across: its opposite facet lies on the same plane
                    if ((far ? n.second[a] : n.first[a]) != plane || (far ? n.first[a] : n.second[a]) == plane) continue;
                    pc::I3 plo{0, 0, 0}, phi{0, 0, 0};
                    bool empty = false;
                    for (int b = 0; b < d; ++b) {
                        plo[b] = std::max(bx.first[b], n.first[b]);
                        phi[b] = std::min(bx.second[b], n.second[b]);
                        if (b != a && plo[b] >= phi[b]) empty = true;
                    }
                    if (empty) continue;
                    plo[a] = phi[a] = plane;
                    for (int bits = 0; bits < (1 << d); ++bits) {
                        pc::I3 p{0, 0, 0};
                        for (int b = 0; b < d; ++b) p[b] = (bits >> b) & 1 ? phi[b] : plo[b];
                        if (!is_corner(p)) return false;
                    }
                }
            }
    return true;
}

std::vector<Box> leaves_of(const pc::Geometry &g) {
    std::vector<Box> cells;
    for (size_t c = 0; c < g.cell_lo.size(); ++c) cells.push_back({g.cell_lo[c], g.cell_hi[c]});
    return cells;
}

}  // namespace

extern "C" {

pc_status pc_split_directions(const pc_box *box, const pc_grid *grid, int32_t radius, const double *impulse,
                              int32_t cell, int32_t *dirs, int32_t *ndirs) {
    if (!impulse || !dirs || !ndirs) return fail(nullptr, PC_ERR_ARG, "null impulse, dirs or ndirs");
    if (radius < 1) return fail(nullptr, PC_ERR_ARG, "radius must be >= 1");
    pc::Geometry g;
    std::string err;
    pc_status st = pc::build_geometry(box, grid, g, err);
    if (st != PC_OK) return fail(nullptr, st, err);
    if (cell < 0 || cell >= int32_t(g.cell_lo.size())) return fail(nullptr, PC_ERR_ARG, "no such leaf");
    std::vector<double> phiE;
    pc::build_extension(g, radius, impulse, phiE);
    const std::vector<int> out = split_directions(g, radius, phiE, cell);
    *ndirs = int32_t(out.size());
    for (size_t j = 0; j < out.size(); ++j) dirs[j] = out[j];
    return PC_OK;
}

pc_status pc_split_is_admissible(const pc_box *box, const pc_grid *grid, int32_t cell, int32_t axis, int32_t *ok) {
    if (!ok) return fail(nullptr, PC_ERR_ARG, "ok is null");
    pc::Geometry g;
    std::string err;
    pc_status st = pc::build_geometry(box, grid, g, err);
    if (st != PC_OK) return fail(nullptr, st, err);
    if (cell < 0 || cell >= int32_t(g.cell_lo.size()) || axis < 0 || axis >= g.d)
        return fail(nullptr, PC_ERR_ARG, "no such leaf or axis");
    if (g.cell_hi[cell][axis] - g.cell_lo[cell][axis] < 2) return fail(nullptr, PC_ERR_ARG, "leaf too thin to split");
    const std::vector<Box> cells = leaves_of(g);
    const std::vector<Box> nxt = split_leaf(cells, cells[size_t(cell)], axis);
    *ok = g.d == 2 || pieces_end_at_points(nxt, {nxt[nxt.size() - 2], nxt.back()}, g.d) ? 1 : 0;
    return PC_OK;
}

pc_status pc_refine(const pc_box *box, const pc_grid *grid, int32_t radius, const double *impulse,
                    const double *eta_c, double y_rms, double tau, int32_t batch, double *eta_omega,
                    int32_t *cells_out, int32_t *num_cells_out) {
    if (!impulse || !eta_c || !eta_omega || !cells_out || !num_cells_out)
        return fail(nullptr, PC_ERR_ARG, "null argument");
    if (radius < 1 || batch < 1 || !(y_rms > 0.0)) return fail(nullptr, PC_ERR_ARG, "radius, batch or y_rms out of range");
    pc::Geometry g;
    std::string err;
    pc_status st = pc::build_geometry(box, grid, g, err);
    if (st != PC_OK) return fail(nullptr, st, err);
    const int nc = int(g.cell_lo.size()), d = g.d;
    double ss = 0.0;
    for (int c = 0; c < nc; ++c) ss += eta_c[c] * eta_c[c];
    *eta_omega = std::sqrt(ss) / y_rms;
    std::vector<Box> cells = leaves_of(g);
    if (*eta_omega > tau) {
        std::vector<double> phiE;
        pc::build_extension(g, radius, impulse, phiE);
        std::vector<int> order(static_cast<size_t>(nc));
        for (int c = 0; c < nc; ++c) order[size_t(c)] = c;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return eta_c[a] > eta_c[b]; });
        std::vector<Box> trial = cells;   // the leaves as split so far this pass
        std::vector<std::pair<int, int>> picks;
        for (int c : order) {
            for (int i : split_directions(g, radius, phiE, c)) {
                std::vector<Box> nxt = split_leaf(trial, cells[size_t(c)], i);
                if (d == 2 || pieces_end_at_points(nxt, {nxt[nxt.size() - 2], nxt.back()}, d)) {
                    trial.swap(nxt);
                    picks.push_back({c, i});
                    break;
                }
            }
            if (int(picks.size()) == batch) break;
        }
        // highest leaf index first: the others keep their places, the halves go last
        std::sort(picks.begin(), picks.end(), [](const std::pair<int, int> &a, const std::pair<int, int> &b) {
            return a.first > b.first;
        });
        for (const auto &ci : picks) {
            const Box bx = cells[size_t(ci.first)];
            cells.erase(cells.begin() + ci.first);
            const int64_t m = (bx.first[ci.second] + bx.second[ci.second]) / 2;
            Box a = bx, b = bx;
            a.second[ci.second] = m;
            b.first[ci.second] = m;
            cells.push_back(a);
            cells.push_back(b);
        }
    }
    *num_cells_out = int32_t(cells.size());
    for (size_t c = 0; c < cells.size(); ++c)
        for (int a = 0; a < d; ++a) {
            cells_out[(c * 2 + 0) * size_t(d) + size_t(a)] = int32_t(cells[c].first[a]);
            cells_out[(c * 2 + 1) * size_t(d) + size_t(a)] = int32_t(cells[c].second[a]);
        }
    return PC_OK;
}

}  // extern "C"
