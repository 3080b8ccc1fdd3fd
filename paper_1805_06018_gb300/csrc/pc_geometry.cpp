// Host-side construction of the product-convolution operator's geometry,
// weights, extended impulse responses and apply schedule (FP64).
//
//   Section 2.2  grid: sample points = corners of the leaves, cells(p_k) by
//                closed containment, U_k = union of cells(p_k), nbrs(k).
//   Section 2.4  harmonic weights: on a leaf whose only sample points are its
//                2^d corners the recursive Laplace construction (linear edges,
//                then discrete-harmonic faces/cells) yields the multilinear
//                hat exactly, because a multilinear function is annihilated
//                by the Kronecker-sum graph Laplacian and is linear on every
//                edge; leaves with hanging nodes are solved in
//                pc_harmonic.cpp.
//   Section 2.5  extension: c_k, v_k = 1/c_k and phi_k^E = sum_j v_k^(j) phi_j
//                (Eqs. vj_def, def_varphiE), neighbours contributing wherever
//                their domain Omega - p_j contains z.
//   Section 3.3  patches: each term phi_k^E * (w_k . x) only reads x on
//                bbox(U_k) and only writes bbox(U_k) (+) [-R, R]^d, so it is
//                evaluated as a small padded FFT convolution of that box.
#include <algorithm>
#include <cstring>
#include <map>
#include <numeric>

#include "pc_internal.h"

namespace pc {

pc_status harmonic_cell_2d(const Geometry &g, int c, int k, std::vector<double> &vals, std::string &err);
// 3D leaf with hanging nodes: its facets as their constituent boxes (the
// intersections with the leaves across them), each with the 2D harmonic
// extension of its node-split edges, then the 3D interior (Section 2.4).
pc_status harmonic_cell_3d(const Geometry &g, int c, int k, std::vector<double> &vals, std::string &err);

static bool lex_less(const I3 &a, const I3 &b) {
    for (int i = 0; i < 3; ++i)
        if (a[i] != b[i]) return a[i] < b[i];
    return false;
}

pc_status build_geometry(const pc_box *box, const pc_grid *grid, Geometry &g, std::string &err) {
    if (!box || !grid) {
        err = "null box or grid";
        return PC_ERR_ARG;
    }
    if (box->ndim != 2 && box->ndim != 3) {
        err = "ndim must be 2 or 3";
        return PC_ERR_ARG;
    }
    g.d = box->ndim;
    int64_t N = 1;
    for (int a = 0; a < 3; ++a) g.shape[a] = 1;
    for (int a = 0; a < g.d; ++a) {
        if (box->shape[a] < 2 || box->shape[a] > (1 << 20)) {
            err = "box extents must be in [2, 2^20]";
            return PC_ERR_ARG;
        }
        g.shape[a] = box->shape[a];
        N *= box->shape[a];
    }
    if (N > (int64_t(1) << 31)) {
        err = "box too large";
        return PC_ERR_ARG;
    }
    if (grid->num_cells <= 0 || !grid->cells) {
        err = "grid has no cells";
        return PC_ERR_GRID;
    }
    const int nc = grid->num_cells;
    g.cell_lo.assign(nc, I3{0, 0, 0});
    g.cell_hi.assign(nc, I3{0, 0, 0});
    for (int c = 0; c < nc; ++c) {
        for (int a = 0; a < g.d; ++a) {
            int64_t lo = grid->cells[(c * 2 + 0) * g.d + a];
            int64_t hi = grid->cells[(c * 2 + 1) * g.d + a];
            if (lo < 0 || hi >= g.shape[a] || hi <= lo) {
                err = "cell " + std::to_string(c) + " is outside the box or degenerate";
                return PC_ERR_GRID;
            }
            g.cell_lo[c][a] = lo;
            g.cell_hi[c][a] = hi;
        }
    }
    // interiors pairwise disjoint
    for (int c = 0; c < nc; ++c)
        for (int e = c + 1; e < nc; ++e) {
            bool overlap = true;
            for (int a = 0; a < g.d && overlap; ++a)
                overlap = g.cell_lo[c][a] < g.cell_hi[e][a] && g.cell_lo[e][a] < g.cell_hi[c][a];
            if (overlap) {
                err = "cells " + std::to_string(c) + " and " + std::to_string(e) + " overlap";
                return PC_ERR_GRID;
            }
        }
    // every point covered (closed boxes)
    {
        std::vector<uint8_t> cov(N, 0);
        for (int c = 0; c < nc; ++c)
            for (int64_t i0 = g.cell_lo[c][0]; i0 <= g.cell_hi[c][0]; ++i0)
                for (int64_t i1 = g.cell_lo[c][1]; i1 <= g.cell_hi[c][1]; ++i1)
                    for (int64_t i2 = g.cell_lo[c][2]; i2 <= g.cell_hi[c][2]; ++i2)
                        cov[(i0 * g.shape[1] + i1) * g.shape[2] + i2] = 1;
        for (int64_t i = 0; i < N; ++i)
            if (!cov[i]) {
                err = "leaves do not cover the box";
                return PC_ERR_GRID;
            }
    }
    // sample points = corners of the leaves
    std::vector<I3> pts;
    pts.reserve(size_t(nc) << g.d);
    for (int c = 0; c < nc; ++c)
        for (int m = 0; m < (1 << g.d); ++m) {
            I3 p{0, 0, 0};
            for (int a = 0; a < g.d; ++a) p[a] = ((m >> a) & 1) ? g.cell_hi[c][a] : g.cell_lo[c][a];
            pts.push_back(p);
        }
    std::sort(pts.begin(), pts.end(), lex_less);
    pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
    g.pts = pts;
    const int r = int(pts.size());
    // points_of / cells_of (closed containment)
    g.points_of.assign(nc, {});
    g.cells_of.assign(r, {});
    for (int c = 0; c < nc; ++c) {
        // candidate points: binary search the lexicographic range of the first coordinate
        I3 lo_key{g.cell_lo[c][0], INT64_MIN, INT64_MIN};
        auto it = std::lower_bound(g.pts.begin(), g.pts.end(), lo_key, lex_less);
        for (; it != g.pts.end() && (*it)[0] <= g.cell_hi[c][0]; ++it) {
            bool in = true;
            for (int a = 0; a < g.d && in; ++a) in = (*it)[a] >= g.cell_lo[c][a] && (*it)[a] <= g.cell_hi[c][a];
            if (in) {
                int k = int(it - g.pts.begin());
                g.points_of[c].push_back(k);
                g.cells_of[k].push_back(c);
            }
        }
    }
    g.nbrs.assign(r, {});
    g.bb_lo.assign(r, I3{0, 0, 0});
    g.bb_hi.assign(r, I3{0, 0, 0});
    for (int k = 0; k < r; ++k) {
        std::vector<int32_t> nb;
        I3 lo{INT64_MAX, INT64_MAX, INT64_MAX}, hi{INT64_MIN, INT64_MIN, INT64_MIN};
        for (int c : g.cells_of[k]) {
            nb.insert(nb.end(), g.points_of[c].begin(), g.points_of[c].end());
            for (int a = 0; a < 3; ++a) {
                lo[a] = std::min(lo[a], g.cell_lo[c][a]);
                hi[a] = std::max(hi[a], g.cell_hi[c][a]);
            }
        }
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        g.nbrs[k] = nb;
        g.bb_lo[k] = lo;
        g.bb_hi[k] = hi;
    }
    return PC_OK;
}

pc_status build_weights(const Geometry &g, std::vector<double> &w, std::vector<int64_t> &off, std::string &err) {
    const int r = int(g.pts.size());
    off.assign(r, 0);
    int64_t tot = 0;
    for (int k = 0; k < r; ++k) {
        off[k] = tot;
        tot += g.bbox_elems(k);
    }
    w.assign(size_t(tot), 0.0);
    std::vector<double> vals;
    for (int c = 0; c < int(g.cell_lo.size()); ++c) {
        const I3 &lo = g.cell_lo[c], &hi = g.cell_hi[c];
        const bool conforming = int(g.points_of[c].size()) == (1 << g.d);
        for (int k : g.points_of[c]) {
            const I3 &bl = g.bb_lo[k], &bh = g.bb_hi[k];
            const int64_t e1 = bh[1] - bl[1] + 1, e2 = g.d == 3 ? bh[2] - bl[2] + 1 : 1;
            double *wk = w.data() + off[k];
            if (conforming) {
                // multilinear hat of corner p_k on the leaf
                for (int64_t i0 = lo[0]; i0 <= hi[0]; ++i0)
                    for (int64_t i1 = lo[1]; i1 <= hi[1]; ++i1)
                        for (int64_t i2 = lo[2]; i2 <= hi[2]; ++i2) {
                            const int64_t x[3] = {i0, i1, i2};
                            double v = 1.0;
                            for (int a = 0; a < g.d; ++a) {
                                const double len = double(hi[a] - lo[a]);
                                v *= (g.pts[k][a] == lo[a]) ? double(hi[a] - x[a]) / len : double(x[a] - lo[a]) / len;
                            }
                            wk[((i0 - bl[0]) * e1 + (i1 - bl[1])) * e2 + (i2 - bl[2])] = v;
                        }
            } else if (g.d == 2) {
                pc_status st = harmonic_cell_2d(g, c, k, vals, err);
                if (st != PC_OK) return st;
                const int64_t m1 = hi[1] - lo[1] + 1;
                for (int64_t i0 = lo[0]; i0 <= hi[0]; ++i0)
                    for (int64_t i1 = lo[1]; i1 <= hi[1]; ++i1)
                        wk[(i0 - bl[0]) * e1 + (i1 - bl[1])] = vals[(i0 - lo[0]) * m1 + (i1 - lo[1])];
            } else {
                pc_status st = harmonic_cell_3d(g, c, k, vals, err);
                if (st != PC_OK) return st;
                const int64_t m1 = hi[1] - lo[1] + 1, m2 = hi[2] - lo[2] + 1;
                for (int64_t i0 = lo[0]; i0 <= hi[0]; ++i0)
                    for (int64_t i1 = lo[1]; i1 <= hi[1]; ++i1)
                        for (int64_t i2 = lo[2]; i2 <= hi[2]; ++i2)
                            wk[((i0 - bl[0]) * e1 + (i1 - bl[1])) * e2 + (i2 - bl[2])] =
                                vals[size_t(((i0 - lo[0]) * m1 + (i1 - lo[1])) * m2 + (i2 - lo[2]))];
            }
        }
    }
    return PC_OK;
}

void build_extension(const Geometry &g, int R, const double *phi, std::vector<double> &phiE) {
    const int r = int(g.pts.size());
    const int64_t W = 2 * R + 1;
    const int64_t wz[3] = {W, W, g.d == 3 ? W : 1};
    const int64_t wsz = wz[0] * wz[1] * wz[2];
    phiE.assign(size_t(r) * wsz, 0.0);
    auto inside = [&](int j, int64_t z0, int64_t z1, int64_t z2) {
        const int64_t z[3] = {z0, z1, z2};
        for (int a = 0; a < g.d; ++a) {
            const int64_t y = g.pts[j][a] + z[a];
            if (y < 0 || y >= g.shape[a]) return false;
        }
        return true;
    };
    for (int k = 0; k < r; ++k) {
        double *out = phiE.data() + size_t(k) * wsz;
        for (int64_t a0 = 0; a0 < wz[0]; ++a0)
            for (int64_t a1 = 0; a1 < wz[1]; ++a1)
                for (int64_t a2 = 0; a2 < wz[2]; ++a2) {
                    const int64_t z0 = a0 - R, z1 = a1 - R, z2 = g.d == 3 ? a2 - R : 0;
                    const int64_t zi = (a0 * wz[1] + a1) * wz[2] + a2;
                    if (inside(k, z0, z1, z2)) {
                        out[zi] = phi[size_t(k) * wsz + zi];
                        continue;
                    }
                    // z outside Omega - p_k: plain average of the neighbours defined there
                    double sum = 0.0;
                    int cnt = 0;
                    for (int j : g.nbrs[k]) {
                        if (j == k || !inside(j, z0, z1, z2)) continue;
                        sum += phi[size_t(j) * wsz + zi];
                        ++cnt;
                    }
                    out[zi] = cnt ? sum / double(cnt) : 0.0;
                }
    }
}

void build_schedule(const Geometry &g, int R, int T, const WindowSplit &wsp, const std::vector<int64_t> &w_off,
                    Schedule &s, const std::vector<int32_t> &patches) {
    const int r = int(g.pts.size());
    const int W = 2 * R + 1;
    int nsubd = 1;
    for (int a = 0; a < g.d; ++a) nsubd *= wsp.nsub;
    std::vector<Tile> tiles;
    const int nk = patches.empty() ? r : int(patches.size());
    for (int q = 0; q < nk; ++q) {
        const int k = patches.empty() ? q : patches[size_t(q)];
        int64_t ext[3] = {1, 1, 1}, nt[3] = {1, 1, 1};
        for (int a = 0; a < g.d; ++a) {
            ext[a] = g.bb_hi[k][a] - g.bb_lo[k][a] + 1;
            nt[a] = (ext[a] + T - 1) / T;
        }
        const int64_t e1 = ext[1], e2 = ext[2];
        for (int64_t t0 = 0; t0 < nt[0]; ++t0)
            for (int64_t t1 = 0; t1 < nt[1]; ++t1)
                for (int64_t t2 = 0; t2 < nt[2]; ++t2) {
                    Tile t{};
                    t.patch = k;
                    const int64_t ti[3] = {t0, t1, t2};
                    int64_t rel[3] = {0, 0, 0};
                    for (int a = 0; a < 3; ++a) {
                        // balanced split: the first (ext % nt) tiles are one longer
                        const int64_t base = ext[a] / nt[a], rem = ext[a] % nt[a];
                        rel[a] = ti[a] * base + std::min<int64_t>(ti[a], rem);
                        t.in_ext[a] = int32_t(base + (ti[a] < rem ? 1 : 0));
                        t.in_lo[a] = int32_t((a < g.d ? g.bb_lo[k][a] : 0) + rel[a]);
                    }
                    if (g.d == 2) {
                        t.w_ld[0] = int32_t(e1);
                        t.w_ld[1] = 1;
                        t.w_base = w_off[k] + rel[0] * e1 + rel[1];
                    } else {
                        t.w_ld[0] = int32_t(e1 * e2);
                        t.w_ld[1] = int32_t(e2);
                        t.w_base = w_off[k] + (rel[0] * e1 + rel[1]) * e2 + rel[2];
                    }
                    // one work unit per kernel sub-window
                    for (int sidx = 0; sidx < nsubd; ++sidx) {
                        Tile u = t;
                        u.spec = q * nsubd + sidx;
                        int rest = sidx;
                        for (int a = g.d - 1; a >= 0; --a) {
                            const int sa = rest % wsp.nsub;
                            rest /= wsp.nsub;
                            const int o = sa * wsp.ws;
                            u.kext[a] = std::min(wsp.ws, W - o);
                            u.out_lo[a] = u.in_lo[a] - R + o;
                        }
                        for (int a = g.d; a < 3; ++a) {
                            u.kext[a] = 1;
                            u.out_lo[a] = 0;
                        }
                        tiles.push_back(u);
                    }
                }
    }
    const int nt = int(tiles.size());
    // output boxes, clipped to Omega, and input boxes: the forward apply adds
    // into the output box, the adjoint into the input box, so two tiles
    // conflict when either box pair overlaps
    std::vector<std::array<int64_t, 6>> ob(nt), ib(nt);
    for (int i = 0; i < nt; ++i)
        for (int a = 0; a < 3; ++a) {
            ob[i][a] = std::max<int64_t>(0, tiles[i].out_lo[a]);
            ob[i][3 + a] = std::min<int64_t>(g.shape[a] - 1,
                                             int64_t(tiles[i].out_lo[a]) + tiles[i].in_ext[a] + tiles[i].kext[a] - 2);
            ib[i][a] = tiles[i].in_lo[a];
            ib[i][3 + a] = int64_t(tiles[i].in_lo[a]) + tiles[i].in_ext[a] - 1;
        }
    auto boxes_meet = [](const std::array<int64_t, 6> &u, const std::array<int64_t, 6> &v) {
        for (int a = 0; a < 3; ++a)
            if (u[3 + a] < v[a] || v[3 + a] < u[a]) return false;
        return true;
    };
    auto overlap = [&](int i, int j) { return boxes_meet(ob[i], ob[j]) || boxes_meet(ib[i], ib[j]); };
    std::vector<std::vector<int32_t>> nbr(nt);
    for (int i = 0; i < nt; ++i)
        for (int j = i + 1; j < nt; ++j)
            if (overlap(i, j)) {
                nbr[i].push_back(j);
                nbr[j].push_back(i);
            }
    // greedy colouring in tile order
    std::vector<int32_t> color(nt, -1);
    int ncol = 0;
    for (int i = 0; i < nt; ++i) {
        std::vector<char> used(nbr[i].size() + 1, 0);
        for (int j : nbr[i])
            if (color[j] >= 0 && color[j] < int(used.size())) used[color[j]] = 1;
        int c = 0;
        while (used[c]) ++c;
        color[i] = c;
        ncol = std::max(ncol, c + 1);
    }
    // stable sort by colour
    std::vector<int32_t> order(nt);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return color[a] < color[b]; });
    std::vector<int32_t> pos(nt);
    for (int i = 0; i < nt; ++i) pos[order[i]] = i;
    s.tiles.resize(nt);
    s.color_start.assign(ncol + 1, 0);
    for (int i = 0; i < nt; ++i) {
        s.tiles[i] = tiles[order[i]];
        s.color_start[color[order[i]] + 1]++;
    }
    for (int c = 0; c < ncol; ++c) s.color_start[c + 1] += s.color_start[c];
    s.dep_start.assign(nt + 1, 0);
    s.dep.clear();
    for (int i = 0; i < nt; ++i) {
        const int t = order[i];
        std::vector<int32_t> d;
        for (int j : nbr[t])
            if (color[j] < color[t]) d.push_back(pos[j]);
        std::sort(d.begin(), d.end());
        s.dep.insert(s.dep.end(), d.begin(), d.end());
        s.dep_start[i + 1] = int32_t(s.dep.size());
    }
}

}  // namespace pc
