// C ABI of libpc: contexts, operator construction, applies, status.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "pc_api_util.h"
#include "pc_internal.h"

namespace {

std::mutex g_err_mu;
std::string g_err;  // last error of context-free calls

}  // namespace

namespace pc {

pc_status fail(pc_context *ctx, pc_status st, const std::string &msg) {
    if (ctx) {
        ctx->last_error = msg;
    } else {
        std::lock_guard<std::mutex> lk(g_err_mu);
        g_err = msg;
    }
    return st;
}

pc_status cuda_fail(pc_context *ctx, cudaError_t e, const char *what) {
    return fail(ctx, e == cudaErrorMemoryAllocation ? PC_ERR_NOMEM : PC_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

ApplyParams part_params(const pc_operator *op, const Part &pt, const ApplyParams &p) {
    ApplyParams q = p;
    q.tiles = op->d_tiles + pt.tile_off;
    q.color_start = op->d_color_start + pt.cs_off;
    q.n_colors = pt.n_colors;
    q.dep_start = op->d_dep_start + pt.ds_off;
    q.dep = op->d_dep + pt.dep_off;
    q.done = p.done + int64_t(pt.tile_off) * p.done_ld;
    q.spec = static_cast<const char *>(op->d_spec) + size_t(pt.spec_off) * 2 * op->elem;
    q.spec_stride = pt.spec_stride;
    q.tw = pt.d_tw;
    q.total_items = int64_t(pt.n_tiles) * p.npairs;
    return q;
}

}  // namespace pc

using pc::cuda_fail;
using pc::DeviceGuard;
using pc::fail;
using pc::upload;

namespace {

// W_P^j = exp(-2 pi i j / P), j < P, from long-double cos/sin of the full
// angle 2 pi j / P, rounded once to double; exact values on the axes.
std::vector<double> twiddles64(int P) {
    std::vector<double> tw(2 * size_t(P));
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int j = 0; j < P; ++j) {
        const long double ang = 2.0L * pi * (long double)j / (long double)P;
        tw[2 * j] = double(std::cos(ang));
        tw[2 * j + 1] = double(-std::sin(ang));
    }
    // exact values on the axes
    for (int j = 0; j < P; j += P / 4) {
        const int q = j / (P / 4);
        tw[2 * j] = q == 0 ? 1.0 : q == 2 ? -1.0 : 0.0;
        tw[2 * j + 1] = q == 1 ? -1.0 : q == 3 ? 1.0 : 0.0;
    }
    return tw;
}

// Frees everything the operator owns; returns the first failing step (or
// nullptr) so that teardown errors are reported instead of left pending.
const char *free_operator(pc_operator *op) {
    if (!op) return nullptr;
    const char *bad = nullptr;
    auto chk = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && !bad) bad = what;
    };
    pc::plain_free(op);
    chk(cudaFree(op->d_spec), "spectra");
    chk(cudaFree(op->d_w), "weights");
    chk(cudaFree(op->d_tiles), "tiles");
    chk(cudaFree(op->d_color_start), "colours");
    chk(cudaFree(op->d_dep_start), "dependency starts");
    chk(cudaFree(op->d_dep), "dependencies");
    chk(cudaFree(op->d_done), "ordering flags");
    chk(cudaFree(op->d_ctrl), "control block");
    for (pc::Part &pt : op->parts)
        if (pt.d_tw && pt.d_tw != op->d_tw) chk(cudaFree(pt.d_tw), "twiddles");
    chk(cudaFree(op->d_tw), "twiddles");
    chk(cudaFree(op->d_scratch), "scratch volumes");
    chk(cudaFree(op->d_big_scratch), "256^2 scratch fields");
    chk(cudaFree(op->d_tc_ops), "tensor-core operands");
    chk(cudaFree(op->d_tc_ops_adj), "tensor-core operands (adjoint)");
    for (auto &kv : op->tc_orders) chk(cudaFree(kv.second), "unit orders");
    chk(cudaFree(op->d_cells), "cells");
    chk(cudaFree(op->d_cell_sums), "cell sums");
    chk(cudaFree(op->d_est), "estimator scratch");
    chk(cudaFree(op->d_entry_mem), "entry tables");
    chk(cudaFree(op->d_host_stage), "host-apply staging");
    if (op->h_host_desc) chk(cudaFreeHost(op->h_host_desc), "host-apply descriptor");
    chk(cudaFree(op->d_host_desc), "host-apply descriptor");
    chk(cudaFree(op->d_host_seg_done), "host-apply counters");
    if (op->h_host_ready) chk(cudaFreeHost(op->h_host_ready), "host-apply ready words");
    for (cudaEvent_t ev : op->host_in_ev) chk(cudaEventDestroy(ev), "host-apply events");
    if (op->h_host_flags) chk(cudaFreeHost(op->h_host_flags), "host-apply flags");
    for (cudaEvent_t ev : op->host_ev)
        if (ev) chk(cudaEventDestroy(ev), "host-apply events");
    if (op->s_h2d) chk(cudaStreamDestroy(op->s_h2d), "copy streams");
    if (op->s_d2h) chk(cudaStreamDestroy(op->s_d2h), "copy streams");
    for (cudaEvent_t ev : op->stage_ev) chk(cudaEventDestroy(ev), "stage events");
    if (op->ev_begin) chk(cudaEventDestroy(op->ev_begin), "events");
    if (op->ev_end) chk(cudaEventDestroy(op->ev_end), "events");
    delete op;
    return bad;
}

}  // namespace

extern "C" {

pc_status pc_context_create(int32_t device, pc_context **ctx) {
    if (!ctx) return fail(nullptr, PC_ERR_ARG, "ctx is null");
    *ctx = nullptr;
    int n = 0;
    cudaError_t e = cudaGetDeviceCount(&n);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDeviceCount");
    if (device < 0 || device >= n) return fail(nullptr, PC_ERR_ARG, "no such CUDA device");
    cudaDeviceProp prop;
    e = cudaGetDeviceProperties(&prop, device);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDeviceProperties");
    if (prop.major != 10 || prop.minor != 3)
        return fail(nullptr, PC_ERR_UNSUPPORTED,
                    "libpc is built for sm_103a (GB300); device is sm_" + std::to_string(prop.major) +
                        std::to_string(prop.minor));
    auto *c = new (std::nothrow) pc_context;
    if (!c) return fail(nullptr, PC_ERR_NOMEM, "out of host memory");
    c->device = device;
    c->num_sms = prop.multiProcessorCount;
    c->cc_major = prop.major;
    c->cc_minor = prop.minor;
    c->smem_optin = prop.sharedMemPerBlockOptin;
    *ctx = c;
    return PC_OK;
}

pc_status pc_context_destroy(pc_context *ctx) {
    delete ctx;
    return PC_OK;
}

const char *pc_last_error(pc_context *ctx) {
    if (ctx) return ctx->last_error.c_str();
    std::lock_guard<std::mutex> lk(g_err_mu);
    static thread_local std::string copy;
    copy = g_err;
    return copy.c_str();
}

pc_status pc_sample_points(const pc_box *box, const pc_grid *grid, int32_t *r, int32_t *points) {
    if (!r) return fail(nullptr, PC_ERR_ARG, "r is null");
    pc::Geometry g;
    std::string err;
    pc_status st = pc::build_geometry(box, grid, g, err);
    if (st != PC_OK) return fail(nullptr, st, err);
    *r = int32_t(g.pts.size());
    if (points)
        for (size_t k = 0; k < g.pts.size(); ++k)
            for (int a = 0; a < g.d; ++a) points[k * g.d + a] = int32_t(g.pts[k][a]);
    return PC_OK;
}

pc_status pc_neighbourhood_boxes(const pc_box *box, const pc_grid *grid, int32_t *lo, int32_t *hi) {
    pc::Geometry g;
    std::string err;
    pc_status st = pc::build_geometry(box, grid, g, err);
    if (st != PC_OK) return fail(nullptr, st, err);
    for (size_t k = 0; k < g.pts.size(); ++k)
        for (int a = 0; a < g.d; ++a) {
            if (lo) lo[k * g.d + a] = int32_t(g.bb_lo[k][a]);
            if (hi) hi[k * g.d + a] = int32_t(g.bb_hi[k][a]);
        }
    return PC_OK;
}

pc_status pc_harmonic_weights(const pc_box *box, const pc_grid *grid, int64_t *count, double *weights) {
    if (!count) return fail(nullptr, PC_ERR_ARG, "count is null");
    pc::Geometry g;
    std::string err;
    pc_status st = pc::build_geometry(box, grid, g, err);
    if (st != PC_OK) return fail(nullptr, st, err);
    int64_t tot = 0;
    for (size_t k = 0; k < g.pts.size(); ++k) tot += g.bbox_elems(int(k));
    *count = tot;
    if (!weights) return PC_OK;
    std::vector<double> w;
    std::vector<int64_t> off;
    st = pc::build_weights(g, w, off, err);
    if (st != PC_OK) return fail(nullptr, st, err);
    std::memcpy(weights, w.data(), sizeof(double) * w.size());
    return PC_OK;
}

pc_status pc_extend_impulse(const pc_box *box, const pc_grid *grid, int32_t radius, const double *impulse,
                            double *impulse_ext) {
    if (!impulse || !impulse_ext) return fail(nullptr, PC_ERR_ARG, "null impulse array");
    if (radius < 1) return fail(nullptr, PC_ERR_ARG, "radius must be >= 1");
    pc::Geometry g;
    std::string err;
    pc_status st = pc::build_geometry(box, grid, g, err);
    if (st != PC_OK) return fail(nullptr, st, err);
    std::vector<double> e;
    pc::build_extension(g, radius, impulse, e);
    std::memcpy(impulse_ext, e.data(), sizeof(double) * e.size());
    return PC_OK;
}

static pc_status build_operator(pc_context *ctx, const pc_box *box, const pc_grid *grid, int32_t radius,
                                const double *impulse, const double *weights, pc_precision prec,
                                const pc_tuning *tune, pc_operator **out) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!ctx) return fail(nullptr, PC_ERR_ARG, "ctx is null");
    if (!out || !impulse) return fail(ctx, PC_ERR_ARG, "null impulse or output handle");
    *out = nullptr;
    if (prec != PC_FP32 && prec != PC_FP64 && prec != PC_BF16X3)
        return fail(ctx, PC_ERR_UNSUPPORTED, "precision not built: use PC_FP32, PC_FP64 or (3D) PC_BF16X3");
    pc::Geometry g;
    std::string err;
    pc_status st = pc::build_geometry(box, grid, g, err);
    if (st != PC_OK) return fail(ctx, st, err);
    if (radius < 1) return fail(ctx, PC_ERR_ARG, "radius must be >= 1");
    const bool three = g.d == 3;
    if (three && prec == PC_FP64) return fail(ctx, PC_ERR_UNSUPPORTED, "3D operators are FP32 or BF16X3");
    if (!three && prec == PC_BF16X3)
        return fail(ctx, PC_ERR_UNSUPPORTED, "PC_BF16X3 (tensor-core first-axis DFTs) covers 3D operators");
    int P = tune && tune->fft_size ? tune->fft_size : (three || prec == PC_FP64 ? 64 : 128);
    if (three && P != 64) return fail(ctx, PC_ERR_UNSUPPORTED, "3D operators use fft_size 64");
    if (prec == PC_FP64 && P != 64) return fail(ctx, PC_ERR_UNSUPPORTED, "FP64 operators use fft_size 64");
    if (prec == PC_FP32 && P != 64 && P != 128) return fail(ctx, PC_ERR_UNSUPPORTED, "FP32 2D fft_size must be 64 or 128");
    // Input tiles of extent n and kernel (sub-)windows of extent ws need
    // n + ws - 1 <= P for the circular product to be the linear convolution;
    // the kernel stages the weight and two right-hand-side rows of a tile in
    // one workspace row of 2P reals (3n <= 2P).  When the window
    // 2R+1 leaves no room for a useful tile it is cut into nsub^2
    // sub-windows (nsub chosen to minimise the FFT work per input pixel,
    // nsub^2 / T^2).
    const int Wfull = 2 * radius + 1;
    // the 3D kernels gather directly, without staging; the tensor-core path
    // keeps GEMM-1 operands of K <= 2 kTc3dMaxTile in shared memory
    const int cap = three ? (prec == PC_BF16X3 ? pc::kTc3dMaxTile : P) : (2 * P) / 3;
    pc::WindowSplit split;
    int T = 0;
    const int forced_split = tune && tune->window_split > 0 ? tune->window_split : 0;
    if (forced_split > 8) return fail(ctx, PC_ERR_ARG, "window_split must be in [1, 8]");
    {
        double best = 1e300;
        for (int nsub = 1; nsub <= 8; ++nsub) {
            if (forced_split && nsub != forced_split) continue;
            const int ws = (Wfull + nsub - 1) / nsub;
            const int t = std::min(P - ws + 1, cap);
            if (t < 1 || (!forced_split && nsub == 1 && t < 16 && Wfull > 16)) continue;
            const double cost = double(nsub) * nsub / (double(t) * t);
            if (cost < best * 0.999) {
                best = cost;
                split.nsub = nsub;
                split.ws = ws;
                T = t;
            }
        }
        if (T < 1) return fail(ctx, PC_ERR_UNSUPPORTED, "radius too large for the FFT size");
    }
    if (tune && tune->tile) {
        if (tune->tile < 1 || tune->tile > T)
            return fail(ctx, PC_ERR_ARG, "tile must be in [1, min(fft_size - window + 1, 2 fft_size / 3)]");
        T = tune->tile;
    }
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return fail(ctx, PC_ERR_CUDA, "cannot select the context's device");
    int ctas_per_sm = 0;
    size_t smem = 0;
    cudaError_t e = three ? pc::fft3d_configure(&ctas_per_sm) : pc::fft2d_configure(P, prec, &ctas_per_sm, &smem);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "configuring the patch kernel");
    if (ctas_per_sm < 1) return fail(ctx, PC_ERR_UNSUPPORTED, "patch kernel does not fit on an SM");
    if (tune && tune->ctas_per_sm > 0) ctas_per_sm = std::min(ctas_per_sm, int(tune->ctas_per_sm));

    const int r = int(g.pts.size());
    const int64_t W = 2 * radius + 1, wsz = three ? W * W * W : W * W;
    // launch shapes: one for the whole operator, or (per_patch) one part per
    // (P, window split) that the work model picks for the patches
    struct Spec {
        int P, T;
        pc::WindowSplit split;
        std::vector<int32_t> patches;   // empty: every patch
    };
    std::vector<Spec> specs;
    if (!three && tune && tune->per_patch) {
        std::vector<std::array<int, 2>> shapes;
        pc::choose_patch_shapes(g, radius, prec, shapes);
        std::map<std::pair<int, int>, std::vector<int32_t>> groups;
        for (int k = 0; k < r; ++k) {
            if (shapes[size_t(k)][0] == 0) return fail(ctx, PC_ERR_UNSUPPORTED, "radius too large for the FFT sizes");
            groups[{shapes[size_t(k)][0], shapes[size_t(k)][1]}].push_back(int32_t(k));
        }
        for (auto &kv : groups) {
            Spec sp;
            sp.P = kv.first.first;
            sp.split.nsub = kv.first.second;
            sp.split.ws = (Wfull + sp.split.nsub - 1) / sp.split.nsub;
            sp.T = std::min(sp.P - sp.split.ws + 1, pc::tile_cap(sp.P));
            if (groups.size() > 1) sp.patches = kv.second;
            specs.push_back(sp);
        }
        if (specs.size() == 1) {
            P = specs[0].P;
            split = specs[0].split;
            T = specs[0].T;
        }
        for (const Spec &sp : specs) {
            int n = 0;
            if ((e = sp.P == pc::kBigFft ? pc::fft2d_big_configure(&n) : pc::fft2d_configure(sp.P, prec, &n, nullptr)) !=
                cudaSuccess)
                return cuda_fail(ctx, e, "configuring the patch kernel");
            ctas_per_sm = std::min(ctas_per_sm, n);
        }
        if (ctas_per_sm < 1) return fail(ctx, PC_ERR_UNSUPPORTED, "patch kernel does not fit on an SM");
    } else {
        specs.push_back(Spec{P, T, split, {}});
    }
    // weights
    std::vector<double> w;
    std::vector<int64_t> woff;
    if (weights) {
        int64_t tot = 0;
        woff.resize(r);
        for (int k = 0; k < r; ++k) {
            woff[k] = tot;
            tot += g.bbox_elems(k);
        }
        w.assign(weights, weights + tot);
    } else {
        st = pc::build_weights(g, w, woff, err);
        if (st != PC_OK) return fail(ctx, st, err);
    }
    // extension (Section 2.5)
    std::vector<double> phiE;
    pc::build_extension(g, radius, impulse, phiE);
    // schedule: one per launch shape, concatenated (colour classes and
    // dependency lists local to each part)
    pc::Schedule sch;
    std::vector<pc::Part> parts;
    for (const Spec &sp : specs) {
        pc::Schedule one;
        pc::build_schedule(g, radius, sp.T, sp.split, woff, one, sp.patches);
        pc::Part pt;
        pt.P = sp.P;
        pt.T = sp.T;
        pt.split = sp.split;
        pt.patches = sp.patches;
        pt.tile_off = int(sch.tiles.size());
        pt.n_tiles = int(one.tiles.size());
        pt.cs_off = int(sch.color_start.size());
        pt.n_colors = int(one.color_start.size()) - 1;
        pt.ds_off = int(sch.dep_start.size());
        pt.dep_off = int(sch.dep.size());
        sch.tiles.insert(sch.tiles.end(), one.tiles.begin(), one.tiles.end());
        sch.color_start.insert(sch.color_start.end(), one.color_start.begin(), one.color_start.end());
        sch.dep_start.insert(sch.dep_start.end(), one.dep_start.begin(), one.dep_start.end());
        sch.dep.insert(sch.dep.end(), one.dep.begin(), one.dep.end());
        parts.push_back(pt);
    }

    auto *op = new (std::nothrow) pc_operator;
    if (!op) return fail(ctx, PC_ERR_NOMEM, "out of host memory");
    op->ctx = ctx;
    op->d = g.d;
    op->shape = g.shape;
    op->N = g.shape[0] * g.shape[1] * g.shape[2];
    op->R = radius;
    op->P = P;
    op->T = T;
    op->split = split;
    op->r = r;
    op->prec = prec;
    op->elem = prec == PC_FP64 ? 8 : 4;
    op->n_tiles = int(sch.tiles.size());
    // parts: several shapes, or the 256^2 kernel (which runs as a part of its own)
    const bool use_parts = specs.size() > 1 || specs[0].P == pc::kBigFft;
    op->n_colors = use_parts ? 0 : int(sch.color_start.size()) - 1;
    if (use_parts) {
        op->parts = parts;
        for (const pc::Part &pt : parts) {
            op->n_colors += pt.n_colors;
            op->P = std::max(op->P, pt.P);
        }
    }
    op->ctas = ctx->num_sms * ctas_per_sm;
    op->ctas_per_sm = ctas_per_sm;
    op->wait_ns = tune && tune->wait_limit_us > 0 ? int64_t(tune->wait_limit_us) * 1000 : 0;
    op->color_start_h = sch.color_start;
    op->tiles_h = sch.tiles;
    op->dep_start_h = sch.dep_start;
    op->dep_h = sch.dep;
    size_t acct = 0;
    auto bail = [&](cudaError_t ee, const char *what) {
        pc_status s2 = cuda_fail(ctx, ee, what);
        free_operator(op);
        return s2;
    };
    // weights in compute precision
    if (prec == PC_FP64) {
        e = upload(reinterpret_cast<double **>(&op->d_w), w.data(), w.size(), acct);
    } else {
        std::vector<float> wf(w.begin(), w.end());
        e = upload(reinterpret_cast<float **>(&op->d_w), wf.data(), wf.size(), acct);
    }
    if (e != cudaSuccess) return bail(e, "uploading weights");
    op->w_bytes = w.size() * op->elem;
    if ((e = upload(&op->d_tiles, sch.tiles.data(), sch.tiles.size(), acct)) != cudaSuccess) return bail(e, "tiles");
    if ((e = upload(&op->d_color_start, sch.color_start.data(), sch.color_start.size(), acct)) != cudaSuccess)
        return bail(e, "colours");
    if ((e = upload(&op->d_dep_start, sch.dep_start.data(), sch.dep_start.size(), acct)) != cudaSuccess)
        return bail(e, "dependencies");
    std::vector<int32_t> depv = sch.dep;
    if (depv.empty()) depv.push_back(0);
    if ((e = upload(&op->d_dep, depv.data(), depv.size(), acct)) != cudaSuccess) return bail(e, "dependencies");
    {
        // leaf cells for the error estimator, on the canonical box (2D as (1, n0, n1))
        std::vector<int32_t> cells6;
        const int nc = int(g.cell_lo.size());
        for (int c = 0; c < nc; ++c) {
            if (g.d == 2) {
                const int32_t v[6] = {0, int32_t(g.cell_lo[c][0]), int32_t(g.cell_lo[c][1]),
                                      0, int32_t(g.cell_hi[c][0]), int32_t(g.cell_hi[c][1])};
                cells6.insert(cells6.end(), v, v + 6);
            } else {
                const int32_t v[6] = {int32_t(g.cell_lo[c][0]), int32_t(g.cell_lo[c][1]), int32_t(g.cell_lo[c][2]),
                                      int32_t(g.cell_hi[c][0]), int32_t(g.cell_hi[c][1]), int32_t(g.cell_hi[c][2])};
                cells6.insert(cells6.end(), v, v + 6);
            }
        }
        op->n_cells = nc;
        if ((e = upload(&op->d_cells, cells6.data(), cells6.size(), acct)) != cudaSuccess) return bail(e, "cells");
        if ((e = cudaMalloc(&op->d_cell_sums, sizeof(double) * std::max(nc, 1))) != cudaSuccess)
            return bail(e, "cell sums");
        acct += sizeof(double) * std::max(nc, 1);
    }
    {
        // O(1) matrix entries (Section 3.1): pixel -> one containing leaf cell,
        // cell -> its sample points, per-patch bbox and weight offsets, phi_k^E
        const int64_t N = g.shape[0] * g.shape[1] * g.shape[2];
        std::vector<int32_t> cell_of(size_t(N), 0), cstart(1, 0), cpts, bblo, bbext;
        for (size_t c = 0; c < g.cell_lo.size(); ++c) {
            for (int64_t a = g.cell_lo[c][0]; a <= g.cell_hi[c][0]; ++a)
                for (int64_t b = g.cell_lo[c][1]; b <= g.cell_hi[c][1]; ++b)
                    for (int64_t q = g.cell_lo[c][2]; q <= g.cell_hi[c][2]; ++q)
                        cell_of[size_t((a * g.shape[1] + b) * g.shape[2] + q)] = int32_t(c);
            for (int32_t k : g.points_of[c]) cpts.push_back(k);
            cstart.push_back(int32_t(cpts.size()));
        }
        for (int k = 0; k < r; ++k)
            for (int a = 0; a < 3; ++a) {
                bblo.push_back(a < g.d ? int32_t(g.bb_lo[k][a]) : 0);
                bbext.push_back(a < g.d ? int32_t(g.bb_hi[k][a] - g.bb_lo[k][a] + 1) : 1);
            }
        if (cpts.empty()) cpts.push_back(0);
        auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
        const size_t o_cell = 0, o_cs = o_cell + al(cell_of.size() * 4), o_cp = o_cs + al(cstart.size() * 4),
                     o_lo = o_cp + al(cpts.size() * 4), o_ext = o_lo + al(bblo.size() * 4),
                     o_wo = o_ext + al(bbext.size() * 4), o_phi = o_wo + al(woff.size() * 8),
                     total = o_phi + al(phiE.size() * 8);
        if ((e = cudaMalloc(&op->d_entry_mem, total)) != cudaSuccess) return bail(e, "entry tables");
        acct += total;
        char *base = static_cast<char *>(op->d_entry_mem);
        const std::pair<size_t, std::pair<const void *, size_t>> parts[] = {
            {o_cell, {cell_of.data(), cell_of.size() * 4}}, {o_cs, {cstart.data(), cstart.size() * 4}},
            {o_cp, {cpts.data(), cpts.size() * 4}},         {o_lo, {bblo.data(), bblo.size() * 4}},
            {o_ext, {bbext.data(), bbext.size() * 4}},     {o_wo, {woff.data(), woff.size() * 8}},
            {o_phi, {phiE.data(), phiE.size() * 8}}};
        for (const auto &pt : parts)
            if (e == cudaSuccess) e = cudaMemcpy(base + pt.first, pt.second.first, pt.second.second, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return bail(e, "entry tables");
        pc::EntryData &ed = op->entry;
        ed.d = g.d;
        ed.R = radius;
        for (int a = 0; a < 3; ++a) ed.n[a] = int32_t(g.shape[a]);
        ed.cell_of = reinterpret_cast<const int32_t *>(base + o_cell);
        ed.cpts_start = reinterpret_cast<const int32_t *>(base + o_cs);
        ed.cpts = reinterpret_cast<const int32_t *>(base + o_cp);
        ed.bb_lo = reinterpret_cast<const int32_t *>(base + o_lo);
        ed.bb_ext = reinterpret_cast<const int32_t *>(base + o_ext);
        ed.w_off = reinterpret_cast<const int64_t *>(base + o_wo);
        ed.phiE = reinterpret_cast<const double *>(base + o_phi);
        // host copies for the incremental estimator: points, bboxes, and a
        // 64-bit FNV-1a hash of each phi_k^E's FP64 bytes
        op->bb_lo_h = bblo;
        op->bb_ext_h = bbext;
        op->pts_h.assign(size_t(r) * 3, 0);
        op->phiE_hash.assign(size_t(r), 0);
        const size_t wsz = r > 0 ? phiE.size() / size_t(r) : 0;
        for (int k = 0; k < r; ++k) {
            for (int a = 0; a < g.d; ++a) op->pts_h[size_t(k) * 3 + size_t(a)] = int32_t(g.pts[k][a]);
            uint64_t h = 14695981039346656037ull;
            const unsigned char *bytes = reinterpret_cast<const unsigned char *>(phiE.data() + size_t(k) * wsz);
            for (size_t i = 0; i < wsz * sizeof(double); ++i) h = (h ^ bytes[i]) * 1099511628211ull;
            op->phiE_hash[size_t(k)] = h;
        }
    }
    if ((e = cudaMalloc(&op->d_ctrl, 64)) != cudaSuccess) return bail(e, "control block");
    acct += 64;
    if ((e = cudaMemset(op->d_ctrl, 0, 64)) != cudaSuccess) return bail(e, "control block");
    // twiddles
    std::vector<double> tw = twiddles64(P);
    double2 *d_tw64 = nullptr;
    if ((e = upload(reinterpret_cast<double **>(&d_tw64), tw.data(), tw.size(), acct)) != cudaSuccess)
        return bail(e, "twiddles");
    acct -= tw.size() * sizeof(double);
    if (prec == PC_FP64) {
        e = upload(reinterpret_cast<double **>(&op->d_tw), tw.data(), tw.size(), acct);
    } else {
        std::vector<float> twf(tw.begin(), tw.end());
        e = upload(reinterpret_cast<float **>(&op->d_tw), twf.data(), twf.size(), acct);
    }
    if (e != cudaSuccess) {
        cudaFree(d_tw64);
        return bail(e, "twiddles");
    }
    // spectra (FP64 on the device, rounded once), one per (patch, sub-window):
    // sub-window (s0, s1) of phi_k^E placed at [0, ws)^2, zero-padded; per
    // launch shape, for the shape's patches in ascending order
    op->spec_stride = three ? int64_t(P / 2 + 1) * P * P : int64_t(P / 2 + 1) * P;
    op->spec_bytes = 0;
    std::vector<int64_t> spec_off(specs.size(), 0);
    for (size_t q = 0; q < specs.size(); ++q) {
        const Spec &sp = specs[q];
        const int nk = sp.patches.empty() ? r : int(sp.patches.size());
        const int nsd = three ? sp.split.nsub * sp.split.nsub * sp.split.nsub : sp.split.nsub * sp.split.nsub;
        const int64_t stride = three ? int64_t(sp.P / 2 + 1) * sp.P * sp.P : int64_t(sp.P / 2 + 1) * sp.P;
        spec_off[q] = int64_t(op->spec_bytes / (2 * op->elem));
        op->spec_bytes += size_t(nk) * size_t(nsd) * size_t(stride) * 2 * op->elem;
        if (!op->parts.empty()) {
            op->parts[q].spec_off = spec_off[q];
            op->parts[q].spec_stride = stride;
        }
    }
    double *d_psi = nullptr;
    e = cudaMalloc(&op->d_spec, op->spec_bytes);
    if (e == cudaSuccess) acct += op->spec_bytes;
    for (size_t q = 0; q < specs.size() && e == cudaSuccess; ++q) {
        const Spec &sp = specs[q];
        const int ns = sp.split.nsub, ws = sp.split.ws;
        const int nk = sp.patches.empty() ? r : int(sp.patches.size());
        const int nsd = three ? ns * ns * ns : ns * ns;
        const int nspec = nk * nsd;
        const size_t wvol = three ? size_t(ws) * ws * ws : size_t(ws) * ws;
        std::vector<double> psi;
        const double *psi_src = phiE.data();
        if (ns > 1 || !sp.patches.empty()) {
            psi.assign(size_t(nspec) * wvol, 0.0);
            const int ns2 = three ? ns : 1, ws2 = three ? ws : 1, Wf2 = three ? Wfull : 1;
            for (int qk = 0; qk < nk; ++qk) {
                const int k = sp.patches.empty() ? qk : sp.patches[size_t(qk)];
                for (int s0 = 0; s0 < ns; ++s0)
                    for (int s1 = 0; s1 < ns; ++s1)
                        for (int s2 = 0; s2 < ns2; ++s2) {
                            double *dst = psi.data() + (size_t(qk) * nsd + (s0 * ns + s1) * ns2 + s2) * wvol;
                            for (int a = 0; a < ws && s0 * ws + a < Wfull; ++a)
                                for (int b = 0; b < ws && s1 * ws + b < Wfull; ++b)
                                    for (int c = 0; c < ws2 && s2 * ws2 + c < Wf2; ++c)
                                        dst[(size_t(a) * ws + b) * ws2 + c] =
                                            phiE[size_t(k) * wsz + ((size_t(s0 * ws + a) * Wfull + (s1 * ws + b)) *
                                                                        Wf2 +
                                                                    (s2 * ws2 + c))];
                        }
            }
            psi_src = psi.data();
        }
        const size_t psi_elems = size_t(nspec) * wvol;
        cudaFree(d_psi);
        d_psi = nullptr;
        e = cudaMalloc(&d_psi, sizeof(double) * psi_elems);
        // the twiddles of this shape's P (FP64 for the build; compute precision for the kernel)
        double2 *tw64 = d_tw64;
        std::vector<double> twq;
        if (e == cudaSuccess && sp.P != P) {
            twq = twiddles64(sp.P);
            size_t dummy = 0;
            e = upload(reinterpret_cast<double **>(&tw64), twq.data(), twq.size(), dummy);
            if (e == cudaSuccess && !op->parts.empty()) {
                if (prec == PC_FP64) {
                    e = upload(reinterpret_cast<double **>(&op->parts[q].d_tw), twq.data(), twq.size(), acct);
                } else {
                    std::vector<float> twf(twq.begin(), twq.end());
                    e = upload(reinterpret_cast<float **>(&op->parts[q].d_tw), twf.data(), twf.size(), acct);
                }
            }
        } else if (!op->parts.empty()) {
            op->parts[q].d_tw = op->d_tw;
        }
        if (e == cudaSuccess) e = cudaMemcpy(d_psi, psi_src, sizeof(double) * psi_elems, cudaMemcpyHostToDevice);
        char *dst = static_cast<char *>(op->d_spec) + size_t(spec_off[q]) * 2 * op->elem;
        if (e == cudaSuccess)
            e = three ? pc::build_spectra_3d(d_psi, nspec, ws, sp.P, dst, tw64, nullptr)
                      : pc::build_spectra_2d(d_psi, nspec, ws, sp.P, prec, dst, tw64, nullptr);
        if (tw64 != d_tw64) {
            const cudaError_t e2 = cudaDeviceSynchronize();
            cudaFree(tw64);
            if (e == cudaSuccess) e = e2;
        }
    }
    for (const pc::Part &pt : op->parts)
        if (e == cudaSuccess && pt.P == pc::kBigFft && !op->d_big_scratch) {
            const size_t sb = pc::fft2d_big_scratch_bytes(op->ctas);
            e = cudaMalloc(&op->d_big_scratch, sb);
            if (e == cudaSuccess) acct += sb;
        }
    if (e == cudaSuccess && three && prec == PC_FP32) {
        const size_t sb = pc::fft3d_scratch_bytes(op->ctas);
        e = cudaMalloc(&op->d_scratch, sb);
        if (e == cudaSuccess) acct += sb;
    }
    if (e == cudaSuccess && three && prec == PC_BF16X3) {
        // the chunk scratch volumes are allocated by the first apply (their
        // number depends on the batch)
        op->tc_k1cap = pc::tc3d_k1cap(T);
        e = pc::tc3d_configure();
        if (e == cudaSuccess) e = pc::tc3d_build_operands(op->tc_k1cap, &op->d_tc_ops);
        if (e == cudaSuccess) acct += size_t(op->tc_k1cap) * 512 + 65536;
        // the adjoint's GEMM 1 runs over every first-axis plane (K = 2 P)
        if (e == cudaSuccess) e = pc::tc3d_build_operands(2 * P, &op->d_tc_ops_adj);
        if (e == cudaSuccess) acct += size_t(2 * P) * 512 + 65536;
    }
    // every upload and spectrum kernel above has landed before the operator
    // is handed out (its applies run on the caller's streams)
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    cudaFree(d_psi);
    cudaFree(d_tw64);
    if (e != cudaSuccess) return bail(e, "building spectra");
    (void)wsz;
    op->device_bytes = acct;
    op->build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = op;
    return PC_OK;
}

pc_status pc_build_spectra(pc_context *ctx, const pc_box *box, const pc_grid *grid, int32_t radius,
                           const double *impulse, const double *weights, pc_precision prec,
                           const pc_tuning *tune, pc_operator **out) {
    if (tune) return build_operator(ctx, box, grid, radius, impulse, weights, prec, tune, out);
    return pc::autotune_build(ctx, box, grid, radius, impulse, weights, prec, out);
}

pc_status pc_operator_info_get(const pc_operator *op, pc_operator_info *info) {
    if (!op || !info) return fail(nullptr, PC_ERR_ARG, "null operator or info");
    std::memset(info, 0, sizeof(*info));
    info->ndim = op->d;
    for (int a = 0; a < 3; ++a) info->shape[a] = op->shape[a];
    info->radius = op->R;
    info->r = op->r;
    info->fft_size = op->P;
    info->tile = op->T;
    info->num_tiles = op->n_tiles;
    info->num_colors = op->n_colors;
    info->precision = op->prec;
    info->spectra_bytes = int64_t(op->spec_bytes);
    info->device_bytes = int64_t(op->device_bytes);
    info->build_seconds = op->build_seconds;
    info->window_split = op->split.nsub;
    info->ctas_per_sm = op->ctas_per_sm;
    info->autotuned = op->autotuned ? 1 : 0;
    info->tuned_candidates = op->tuned_candidates;
    info->tuned_ms = op->tuned_ms;
    info->num_parts = op->parts.empty() ? 1 : int32_t(op->parts.size());
    return PC_OK;
}

static pc_status ensure_done_capacity(pc_operator *op, int32_t npairs) {
    if (npairs <= op->done_cap) return PC_OK;
    cudaError_t e = cudaSuccess;
    if (op->last_stream || op->d_done) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(op->ctx, e, "synchronising before growing flags");
    cudaFree(op->d_done);
    op->d_done = nullptr;
    op->device_bytes -= sizeof(uint32_t) * size_t(op->n_tiles) * size_t(op->done_cap);
    const int32_t cap = std::max<int32_t>(npairs, 32);
    const size_t bytes = sizeof(uint32_t) * size_t(op->n_tiles) * cap;
    e = cudaMalloc(&op->d_done, bytes);
    if (e != cudaSuccess) {
        op->done_cap = 0;
        return cuda_fail(op->ctx, e, "allocating ordering flags");
    }
    op->device_bytes += bytes;
    e = pc::zero_now(op->d_done, bytes);
    if (e != cudaSuccess) return cuda_fail(op->ctx, e, "clearing ordering flags");
    op->done_cap = cap;
    op->epoch = 0;
    return PC_OK;
}

// 3D, BF16x3: the items run in chunks of at most kTc3dChunkItems through
// three kernels (phase 1 -> tensor-core first-axis transform -> phase 3),
// each item with its own scratch volume; stream-ordered like the fused path.
// BF16x3 3D: per-item scratch volumes for a chunk of min(total, kTc3dChunkItems) items
static pc_status ensure_split3d_scratch(pc_operator *op, int64_t total) {
    const int64_t chunk = std::min<int64_t>(total, pc::kTc3dChunkItems);
    if (op->scratch_items >= chunk) return PC_OK;
    cudaError_t e = cudaSuccess;
    if (op->d_scratch && (e = cudaDeviceSynchronize()) != cudaSuccess)
        return cuda_fail(op->ctx, e, "synchronising before growing the scratch volumes");
    cudaFree(op->d_scratch);
    op->d_scratch = nullptr;
    op->device_bytes -= size_t(op->scratch_items) * pc::fft3d_volume_bytes();
    op->scratch_items = 0;
    if ((e = cudaMalloc(&op->d_scratch, size_t(chunk) * pc::fft3d_volume_bytes())) != cudaSuccess)
        return cuda_fail(op->ctx, e, "allocating the 3D scratch volumes");
    op->scratch_items = chunk;
    op->device_bytes += size_t(chunk) * pc::fft3d_volume_bytes();
    return PC_OK;
}

static pc_status apply_split3d(pc_operator *op, const pc::ApplyParams &p, cudaStream_t s, bool adjoint) {
    pc_context *ctx = op->ctx;
    const int64_t total = p.total_items;
    const int64_t chunk = std::min<int64_t>(total, pc::kTc3dChunkItems);
    cudaError_t e = cudaSuccess;
    pc_status st0 = ensure_split3d_scratch(op, total);
    if (st0 != PC_OK) return st0;
    const int nchunks = int((total + chunk - 1) / chunk);
    int32_t *order = nullptr;
    auto oit = op->tc_orders.find(p.npairs);
    if (oit != op->tc_orders.end()) {
        order = oit->second;
    } else {
        // items of each chunk sorted by (tile, pair): the tensor stage then
        // visits the pairs of one tile and line block back to back.  One
        // table per batch shape, kept until the operator is destroyed, so
        // applies in flight never see their table replaced.
        const int32_t np = p.npairs;
        // [total] item indices, then [total] their tiles
        std::vector<int32_t> ord(static_cast<size_t>(2 * total));
        std::vector<std::pair<int64_t, int32_t>> key;
        for (int c = 0; c < nchunks; ++c) {
            const int64_t c0 = int64_t(c) * chunk, c1 = std::min<int64_t>(total, c0 + chunk);
            key.clear();
            for (int64_t item = c0; item < c1; ++item) {
                int col = 0;
                while (int64_t(op->color_start_h[col + 1]) * np <= item) ++col;
                const int64_t base = int64_t(op->color_start_h[col]) * np;
                const int ntc = op->color_start_h[col + 1] - op->color_start_h[col];
                const int64_t ti = op->color_start_h[col] + (item - base) % ntc, pair = (item - base) / ntc;
                key.emplace_back(ti * np + pair, int32_t(item));
            }
            std::sort(key.begin(), key.end());
            for (size_t i = 0; i < key.size(); ++i) {
                ord[size_t(c0) + i] = key[i].second;
                ord[size_t(total + c0) + i] = int32_t(key[i].first / np);
            }
        }
        if ((e = cudaMalloc(&order, ord.size() * sizeof(int32_t))) != cudaSuccess)
            return cuda_fail(ctx, e, "allocating the unit order");
        // ordered on s (a pageable source is staged before the call returns)
        if ((e = cudaMemcpyAsync(order, ord.data(), ord.size() * sizeof(int32_t), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess) {
            cudaFree(order);
            return cuda_fail(ctx, e, "uploading the unit order");
        }
        op->tc_orders[np] = order;
    }
    while (op->stage_ev.size() < size_t(nchunks) * 6) {
        cudaEvent_t ev = nullptr;
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) return cuda_fail(ctx, e, "creating events");
        op->stage_ev.push_back(ev);
    }
    if ((e = pc::launch_zero(p, op->N, op->prec, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "launching the zero kernel");
    cudaEventRecord(op->ev_begin, s);
    for (int c = 0; c < nchunks && e == cudaSuccess; ++c) {
        const int64_t c0 = int64_t(c) * chunk, c1 = std::min<int64_t>(total, c0 + chunk);
        const int ctas = int(std::min<int64_t>(op->ctas, c1 - c0));
        cudaEvent_t *ev = &op->stage_ev[size_t(c) * 6];
        cudaEventRecord(ev[0], s);
        e = pc::launch_fft3d_phase1(p, ctas, op->d_scratch, c0, c1, s, adjoint);
        cudaEventRecord(ev[1], s);
        if (e != cudaSuccess) break;
        cudaEventRecord(ev[2], s);
        e = adjoint ? pc::launch_tc3d_axis0_adjoint(p, ctx->num_sms, op->d_scratch, order, c0, c1, op->d_tc_ops_adj, s)
                    : pc::launch_tc3d_axis0(p, ctx->num_sms, op->d_scratch, order, c0, c1, op->d_tc_ops,
                                            op->tc_k1cap, s);
        cudaEventRecord(ev[3], s);
        if (e != cudaSuccess) break;
        cudaEventRecord(ev[4], s);
        e = pc::launch_fft3d_phase3(p, ctas, op->d_scratch, c0, c1, s, adjoint);
        cudaEventRecord(ev[5], s);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "launching the 3D split path");
    cudaEventRecord(op->ev_end, s);
    op->stage_chunks = nchunks;
    op->timed = true;
    op->last_stream = s;
    op->launches_last = 1 + 3 * int64_t(nchunks);
    return PC_OK;
}

// Grow what an apply of nrhs vectors allocates on demand (ordering flags,
// BF16x3 scratch), so that a later apply of at most nrhs vectors allocates
// nothing.  May synchronise the device when something grows.
static pc_status prepare_batch_impl(pc_operator *op, int32_t nrhs) {
    if (!op || nrhs < 1) return fail(op ? op->ctx : nullptr, PC_ERR_ARG, "bad operator or nrhs");
    DeviceGuard dg(op->ctx->device);
    if (!dg.ok) return fail(op->ctx, PC_ERR_CUDA, "cannot select the context's device");
    const int32_t npairs = (nrhs + 1) / 2;
    const bool split3d = op->d == 3 && op->prec == PC_BF16X3;
    pc_status st = ensure_done_capacity(op, npairs * pc::flag_groups(op->d, op->prec));
    if (st == PC_OK && split3d) st = ensure_split3d_scratch(op, int64_t(op->n_tiles) * npairs);
    return st;
}

// The parts of a per_patch operator, one launch each after the zero-fill
// (which also reset the claim counter for the first): each part's items run
// in its own colour order, and the parts add one after another, so y is
// still summed in a fixed order.
static pc_status apply_parts(pc_operator *op, const pc::ApplyParams &p, cudaStream_t s, bool adjoint) {
    cudaError_t e = cudaEventRecord(op->ev_begin, s);
    for (size_t q = 0; q < op->parts.size() && e == cudaSuccess; ++q) {
        const pc::ApplyParams pq = pc::part_params(op, op->parts[q], p);
        if (q > 0) e = cudaMemsetAsync(p.ctrl, 0, sizeof(unsigned long long), s);   // claim counter
        if (e != cudaSuccess) break;
        const int ctas = int(std::min<int64_t>(op->ctas, pq.total_items));
        if (ctas > 0)
            e = op->parts[q].P == pc::kBigFft ? pc::launch_fft2d_big(pq, ctas, op->d_big_scratch, s, adjoint)
                                              : pc::launch_fft2d(pq, op->parts[q].P, op->prec, ctas, s, adjoint);
    }
    if (e != cudaSuccess) return cuda_fail(op->ctx, e, "launching the patch kernel");
    cudaEventRecord(op->ev_end, s);
    op->timed = true;
    op->last_stream = s;
    op->launches_last = 1 + int64_t(op->parts.size());
    return PC_OK;
}

static pc_status apply_batched(pc_operator *op, int32_t nrhs, const void *x, int64_t ldx, void *y, int64_t ldy,
                               pc_stream stream, bool adjoint) {
    if (!op) return fail(nullptr, PC_ERR_ARG, "operator is null");
    pc_context *ctx = op->ctx;
    if (nrhs < 0) return fail(ctx, PC_ERR_ARG, "nrhs < 0");
    if (nrhs == 0) return PC_OK;
    if (!x || !y) return fail(ctx, PC_ERR_ARG, "null x or y");
    if (ldx < op->N || ldy < op->N) return fail(ctx, PC_ERR_ARG, "ldx and ldy must be >= N");
    const uintptr_t xa = reinterpret_cast<uintptr_t>(x), ya = reinterpret_cast<uintptr_t>(y);
    if (xa % op->elem || ya % op->elem) return fail(ctx, PC_ERR_ARG, "x and y must be aligned to the element size");
    const uintptr_t xe = xa + uintptr_t((int64_t(nrhs - 1) * ldx + op->N) * op->elem);
    const uintptr_t ye = ya + uintptr_t((int64_t(nrhs - 1) * ldy + op->N) * op->elem);
    if (xa < ye && ya < xe) return fail(ctx, PC_ERR_ARG, "x and y overlap");
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return fail(ctx, PC_ERR_CUDA, "cannot select the context's device");
    const int32_t npairs = (nrhs + 1) / 2;
    // 3D paths keep one flag per output-plane group
    const bool split3d = op->d == 3 && op->prec == PC_BF16X3;
    pc_status st = ensure_done_capacity(op, npairs * pc::flag_groups(op->d, op->prec));
    if (st != PC_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (++op->epoch == 0) op->epoch = 1;
    pc::ApplyParams p{};
    p.x = x;
    p.y = y;
    p.ldx = ldx;
    p.ldy = ldy;
    p.nrhs = nrhs;
    p.npairs = npairs;
    p.n[0] = int32_t(op->shape[0]);
    p.n[1] = int32_t(op->shape[1]);
    p.n[2] = int32_t(op->shape[2]);
    p.nx[0] = p.n[0];
    p.nx[1] = p.n[1];
    p.nx[2] = p.n[2];
    p.R = op->R;
    p.tiles = op->d_tiles;
    p.color_start = op->d_color_start;
    p.n_colors = op->n_colors;
    p.dep_start = op->d_dep_start;
    p.dep = op->d_dep;
    p.done = op->d_done;
    p.done_ld = op->done_cap;
    p.epoch = op->epoch;
    p.ctrl = op->d_ctrl;
    p.spec = op->d_spec;
    p.spec_stride = op->spec_stride;
    p.w = op->d_w;
    p.tw = op->d_tw;
    p.wait_ns = op->wait_ns;
    p.total_items = int64_t(op->n_tiles) * npairs;
    if (!op->ev_begin) {
        cudaError_t e = cudaEventCreate(&op->ev_begin);
        if (e == cudaSuccess) e = cudaEventCreate(&op->ev_end);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "creating events");
    }
    if (split3d) return apply_split3d(op, p, s, adjoint);
    cudaError_t e = pc::launch_zero(p, op->N, op->prec, s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "launching the zero kernel");
    if (!op->parts.empty()) return apply_parts(op, p, s, adjoint);
    const int ctas = int(std::min<int64_t>(op->ctas, p.total_items));
    cudaEventRecord(op->ev_begin, s);
    e = op->d == 3 ? pc::launch_fft3d(p, op->ctas, op->d_scratch, s, adjoint)
                   : pc::launch_fft2d(p, op->P, op->prec, ctas, s, adjoint);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "launching the patch kernel");
    cudaEventRecord(op->ev_end, s);
    op->timed = true;
    op->last_stream = s;
    op->launches_last = 2;
    return PC_OK;
}

pc_status pc_apply_batched(pc_operator *op, int32_t nrhs, const void *x, int64_t ldx, void *y, int64_t ldy,
                           pc_stream stream) {
    return apply_batched(op, nrhs, x, ldx, y, ldy, stream, false);
}

pc_status pc_apply_adjoint_batched(pc_operator *op, int32_t nrhs, const void *x, int64_t ldx, void *y, int64_t ldy,
                                   pc_stream stream) {
    return apply_batched(op, nrhs, x, ldx, y, ldy, stream, true);
}

}  // extern "C"

namespace {

pc_status ensure_host_resources(pc_operator *op, size_t stage_bytes) {
    pc_context *ctx = op->ctx;
    cudaError_t e = cudaSuccess;
    if (!op->s_h2d) {
        if ((e = cudaStreamCreateWithFlags(&op->s_h2d, cudaStreamNonBlocking)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&op->s_d2h, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(ctx, e, "creating copy streams");
        for (cudaEvent_t &ev : op->host_ev)
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(ctx, e, "creating pipeline events");
    }
    if (stage_bytes > op->host_stage_bytes) {
        if (op->d_host_stage && (e = cudaDeviceSynchronize()) != cudaSuccess)
            return cuda_fail(ctx, e, "synchronising before growing the staging buffers");
        cudaFree(op->d_host_stage);
        op->d_host_stage = nullptr;
        op->device_bytes -= op->host_stage_bytes;
        op->host_stage_bytes = 0;
        if ((e = cudaMalloc(&op->d_host_stage, stage_bytes)) != cudaSuccess)
            return cuda_fail(ctx, e, "allocating the staging buffers");
        op->host_stage_bytes = stage_bytes;
        op->device_bytes += stage_bytes;
    }
    return PC_OK;
}

cudaError_t copy_rows(void *dst, size_t dld, const void *src, size_t sld, size_t width, size_t rows,
                      cudaMemcpyKind kind, cudaStream_t s) {
    if (dld == width && sld == width) return cudaMemcpyAsync(dst, src, width * rows, kind, s);
    return cudaMemcpy2DAsync(dst, dld, src, sld, width, rows, kind, s);
}

// 2D host apply as one persistent launch over segments of c right-hand sides
// (c even, so each segment keeps the pairs of the whole batch).  The whole
// batch is staged on the device.  Chunk i is copied in on s_h2d; when this
// thread sees the copy's event complete it sets the segment's ready word (in
// mapped host memory), which a CTA reaching the segment's items waits for
// (bounded).  The kernel raises each segment's completion flag in mapped
// host memory when its last item has landed; this thread then copies the
// segment out on s_d2h.
pc_status apply_host_segmented(pc_operator *op, int32_t nrhs, const void *x, int64_t ldx, void *y, int64_t ldy,
                               bool adjoint, int32_t c, cudaStream_t s) {
    pc_context *ctx = op->ctx;
    const int32_t nch = (nrhs + c - 1) / c;
    const size_t vec = size_t(op->N) * op->elem;
    const int64_t el = int64_t(op->elem);
    cudaError_t e = cudaSuccess;
    if (!op->h_host_desc) {
        const size_t w = sizeof(uint32_t) * pc::kMaxSegments;
        if ((e = cudaHostAlloc(reinterpret_cast<void **>(&op->h_host_desc), sizeof(pc::LaunchDesc), 0)) != cudaSuccess ||
            (e = cudaMalloc(&op->d_host_desc, sizeof(pc::LaunchDesc))) != cudaSuccess ||
            (e = cudaMalloc(&op->d_host_seg_done, w)) != cudaSuccess ||
            (e = cudaHostAlloc(reinterpret_cast<void **>(&op->h_host_ready), w, cudaHostAllocMapped)) != cudaSuccess ||
            (e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&op->d_host_ready), op->h_host_ready, 0)) !=
                cudaSuccess ||
            (e = cudaHostAlloc(reinterpret_cast<void **>(&op->h_host_flags), w, cudaHostAllocMapped)) != cudaSuccess ||
            (e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&op->d_host_flags), op->h_host_flags, 0)) !=
                cudaSuccess)
            return cuda_fail(ctx, e, "allocating the segmented launch's descriptor and flags");
        std::memset(op->h_host_ready, 0, w);
        op->device_bytes += sizeof(pc::LaunchDesc) + w;
        op->host_in_ev.assign(size_t(pc::kMaxSegments), nullptr);
        for (cudaEvent_t &ev : op->host_in_ev)
            if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess)
                return cuda_fail(ctx, e, "creating copy events");
    }
    pc_status st = ensure_host_resources(op, 2 * vec * size_t(nrhs));
    if (st != PC_OK) return st;
    if ((st = ensure_done_capacity(op, (nrhs + 1) / 2)) != PC_OK) return st;
    size_t smem = 0;
    if ((e = pc::fft2d_configure(op->P, op->prec, nullptr, &smem)) != cudaSuccess)
        return cuda_fail(ctx, e, "configuring the patch kernel");
    if (++op->epoch == 0) op->epoch = 1;
    const uint32_t ep = op->epoch;
    char *xs = static_cast<char *>(op->d_host_stage), *ys = xs + vec * size_t(nrhs);
    pc::LaunchDesc &d = *op->h_host_desc;
    std::memset(&d, 0, sizeof(pc::LaunchDesc));
    volatile uint32_t *hf = op->h_host_flags;
    int64_t items = 0;
    for (int32_t i = 0; i < nch; ++i) {
        const int64_t b0 = int64_t(i) * c;
        const int32_t cnt = int32_t(std::min<int64_t>(c, nrhs - b0));
        const int32_t np = (cnt + 1) / 2;
        pc::Segment &sg = d.seg[i];
        pc::ApplyParams &p = sg.p;
        p.x = xs + size_t(b0) * vec;
        p.y = ys + size_t(b0) * vec;
        p.ldx = p.ldy = op->N;
        p.nrhs = cnt;
        p.npairs = np;
        p.n[0] = int32_t(op->shape[0]);
        p.n[1] = int32_t(op->shape[1]);
        p.n[2] = int32_t(op->shape[2]);
        p.nx[0] = p.n[0];
        p.nx[1] = p.n[1];
        p.nx[2] = p.n[2];
        p.R = op->R;
        p.tiles = op->d_tiles;
        p.color_start = op->d_color_start;
        p.n_colors = op->n_colors;
        p.dep_start = op->d_dep_start;
        p.dep = op->d_dep;
        p.done = op->d_done + int64_t(op->n_tiles) * (b0 / 2);   // disjoint per segment
        p.done_ld = np;
        p.epoch = ep;
        p.ctrl = op->d_ctrl;
        p.spec = op->d_spec;
        p.spec_stride = op->spec_stride;
        p.w = op->d_w;
        p.tw = op->d_tw;
        p.wait_ns = op->wait_ns;
        p.total_items = int64_t(op->n_tiles) * np;
        sg.item_begin = items;
        sg.ready = op->d_host_ready + i;
        sg.ready_val = ep;
        sg.slot = i;
        items += p.total_items;
        hf[i] = 0u;
    }
    d.nseg = nch;
    d.total_items = items;
    cudaEvent_t *ev = op->host_ev;
    // copies start after the work already queued on the caller's stream
    cudaEventRecord(ev[6], s);
    cudaStreamWaitEvent(op->s_h2d, ev[6], 0);
    cudaStreamWaitEvent(op->s_d2h, ev[6], 0);
    for (int32_t i = 0; i < nch; ++i) {
        const int64_t b0 = int64_t(i) * c;
        const size_t cnt = size_t(std::min<int64_t>(c, nrhs - b0));
        if ((e = copy_rows(xs + size_t(b0) * vec, vec, static_cast<const char *>(x) + b0 * ldx * el,
                           size_t(ldx * el), vec, cnt, cudaMemcpyHostToDevice, op->s_h2d)) != cudaSuccess)
            return cuda_fail(ctx, e, "copying a chunk in");
        if ((e = cudaEventRecord(op->host_in_ev[size_t(i)], op->s_h2d)) != cudaSuccess)
            return cuda_fail(ctx, e, "recording a copy event");
    }
    if ((e = cudaMemcpyAsync(op->d_host_desc, op->h_host_desc, sizeof(pc::LaunchDesc), cudaMemcpyHostToDevice, s)) !=
        cudaSuccess)
        return cuda_fail(ctx, e, "uploading the launch descriptor");
    if (!op->ev_begin) {
        if ((e = cudaEventCreate(&op->ev_begin)) == cudaSuccess) e = cudaEventCreate(&op->ev_end);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "creating events");
    }
    const int ctas = int(std::min<int64_t>(op->ctas, items));
    cudaEventRecord(op->ev_begin, s);
    if ((e = pc::launch_round(op->d_host_desc, reinterpret_cast<unsigned long long *>(op->d_ctrl), op->d_ctrl + 2,
                              op->d_host_seg_done, op->d_host_flags, ctas, smem, s, op->P, op->prec, adjoint)) !=
        cudaSuccess)
        return cuda_fail(ctx, e, "launching the segmented patch kernel");
    cudaEventRecord(op->ev_end, s);
    op->timed = true;
    op->last_stream = s;
    op->launches_last = 2;
    // mark each segment ready once its copy in has completed, and copy each
    // segment out once the kernel has finished it
    if ((e = cudaEventSynchronize(ev[6])) != cudaSuccess) return cuda_fail(ctx, e, "waiting for earlier work");
    // Failure-path tests set PC_TEST_WITHHOLD_READY=1: every segment after the
    // first is then never marked ready, so the kernel's bounded wait for it
    // runs out and the call must come back with PC_ERR_TIMEOUT.
    const char *withhold_env = std::getenv("PC_TEST_WITHHOLD_READY");
    const bool withhold = withhold_env && withhold_env[0] == '1';
    volatile uint32_t *hr = op->h_host_ready;
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::seconds(60);
    int32_t next_in = 0, next_out = 0;
    for (uint64_t polls = 0; next_out < nch; ++polls) {
        while (next_in < nch) {
            const cudaError_t q = cudaEventQuery(op->host_in_ev[size_t(next_in)]);
            if (q == cudaErrorNotReady) break;
            if (q != cudaSuccess) return cuda_fail(ctx, q, "copying a chunk in");
            if (!withhold || next_in == 0) hr[next_in] = ep;   // the kernel reads it with a system-scope acquire
            ++next_in;
        }
        bool progressed = false;
        while (next_out < next_in && hf[next_out] != 0u) {
            const int64_t b0 = int64_t(next_out) * c;
            const size_t cnt = size_t(std::min<int64_t>(c, nrhs - b0));
            if ((e = copy_rows(static_cast<char *>(y) + b0 * ldy * el, size_t(ldy * el), ys + size_t(b0) * vec, vec,
                               vec, cnt, cudaMemcpyDeviceToHost, op->s_d2h)) != cudaSuccess)
                return cuda_fail(ctx, e, "copying a chunk out");
            ++next_out;
            progressed = true;
        }
        if (progressed || (polls & 1023) != 1023) continue;
        const cudaError_t q = cudaStreamQuery(s);
        if (q != cudaSuccess && q != cudaErrorNotReady) return cuda_fail(ctx, q, "the segmented patch kernel");
        if (q == cudaSuccess && next_out < nch && next_in == nch && hf[next_out] == 0u) {
            // the launch ended early: a bounded device-side wait gave up (status word set)
            // or the kernel failed; let the copies already queued finish either way
            int32_t flag = 0;
            cudaError_t e2 = cudaStreamSynchronize(op->s_d2h);
            if (e2 == cudaSuccess) e2 = cudaMemcpy(&flag, op->d_ctrl + 2, sizeof(flag), cudaMemcpyDeviceToHost);
            if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "reading the launch status");
            if (flag != 0) {
                if ((e2 = pc::zero_now(op->d_ctrl + 2, sizeof(flag))) != cudaSuccess)
                    return cuda_fail(ctx, e2, "clearing the launch status");
                return fail(ctx, PC_ERR_TIMEOUT,
                            "a device-side wait of the segmented launch ran out (limit " +
                                std::to_string(op->wait_ns > 0 ? op->wait_ns / 1000 : 2000000) + " us)");
            }
            return fail(ctx, PC_ERR_CUDA, "the patch kernel ended without finishing a segment");
        }
        if (std::chrono::steady_clock::now() > deadline)
            return fail(ctx, PC_ERR_TIMEOUT, "the host apply did not finish within 60 s");
    }
    cudaEventRecord(ev[4], op->s_d2h);
    if ((e = cudaStreamWaitEvent(s, ev[4], 0)) != cudaSuccess)
        return cuda_fail(ctx, e, "ordering the caller's stream after the copies");
    return PC_OK;
}

// Chunked pipeline: chunk i copied in on s_h2d, applied on s, copied out on
// s_d2h, through two device staging slots.
pc_status apply_host_chunked(pc_operator *op, int32_t nrhs, const void *x, int64_t ldx, void *y, int64_t ldy,
                             bool adjoint, int32_t c, cudaStream_t s) {
    pc_context *ctx = op->ctx;
    const size_t vec = size_t(op->N) * op->elem;
    const int64_t el = int64_t(op->elem);
    pc_status st = ensure_host_resources(op, 4 * vec * size_t(c));
    if (st != PC_OK) return st;
    if ((st = prepare_batch_impl(op, c)) != PC_OK) return st;
    cudaEvent_t *ev = op->host_ev;
    char *base = static_cast<char *>(op->d_host_stage);
    const size_t slot = vec * size_t(c);
    // slot j: x at base + 2j * slot, y at base + (2j + 1) * slot
    cudaEventRecord(ev[6], s);
    cudaStreamWaitEvent(op->s_h2d, ev[6], 0);
    cudaStreamWaitEvent(op->s_d2h, ev[6], 0);
    const int32_t nch = (nrhs + c - 1) / c;
    int64_t launches = 0;
    cudaError_t e = cudaSuccess;
    for (int32_t i = 0; i < nch; ++i) {
        const int j = i & 1;
        const int64_t b0 = int64_t(i) * c;
        const int32_t cnt = int32_t(std::min<int64_t>(c, nrhs - b0));
        char *xs = base + 2 * j * slot, *ys = base + (2 * j + 1) * slot;
        // copy in once chunk i - 2 has been computed from this slot
        if (i >= 2) cudaStreamWaitEvent(op->s_h2d, ev[2 + j], 0);
        if ((e = copy_rows(xs, vec, static_cast<const char *>(x) + b0 * ldx * el, size_t(ldx * el), vec, size_t(cnt),
                           cudaMemcpyHostToDevice, op->s_h2d)) != cudaSuccess)
            return cuda_fail(ctx, e, "copying a chunk in");
        cudaEventRecord(ev[j], op->s_h2d);
        // compute once it is in and chunk i - 2's result has left this slot
        cudaStreamWaitEvent(s, ev[j], 0);
        if (i >= 2) cudaStreamWaitEvent(s, ev[4 + j], 0);
        st = apply_batched(op, cnt, xs, op->N, ys, op->N, s, adjoint);
        if (st != PC_OK) return st;
        launches += op->launches_last;
        cudaEventRecord(ev[2 + j], s);
        cudaStreamWaitEvent(op->s_d2h, ev[2 + j], 0);
        if ((e = copy_rows(static_cast<char *>(y) + b0 * ldy * el, size_t(ldy * el), ys, vec, vec, size_t(cnt),
                           cudaMemcpyDeviceToHost, op->s_d2h)) != cudaSuccess)
            return cuda_fail(ctx, e, "copying a chunk out");
        cudaEventRecord(ev[4 + j], op->s_d2h);
    }
    // the caller's stream continues once the last copy out (the copy stream is in order) is done
    if ((e = cudaStreamWaitEvent(s, ev[4 + ((nch - 1) & 1)], 0)) != cudaSuccess)
        return cuda_fail(ctx, e, "ordering the caller's stream after the copies");
    op->launches_last = launches;
    return PC_OK;
}

}  // namespace

extern "C" {

// The segmented launch needs the calling thread to run beside the kernel: it
// marks chunks ready while the kernel's CTAs wait for them.  Where a launch
// blocks the host until the kernel ends (CUDA_LAUNCH_BLOCKING set to a
// non-zero value), every CTA would wait out its bound; there, and where the
// caller asks for it (PC_HOST_PIPELINE=chunked, e.g. under a profiler that
// serialises launches), 2D operators take the chunked pipeline instead.
static bool segmented_host_apply() {
    const char *blocking = std::getenv("CUDA_LAUNCH_BLOCKING");
    if (blocking && blocking[0] && std::strcmp(blocking, "0") != 0) return false;
    const char *mode = std::getenv("PC_HOST_PIPELINE");
    return !(mode && std::strcmp(mode, "chunked") == 0);
}

pc_status pc_apply_host(pc_operator *op, int32_t nrhs, const void *x, int64_t ldx, void *y, int64_t ldy,
                        int32_t adjoint, int32_t chunk, pc_stream stream) {
    if (!op) return fail(nullptr, PC_ERR_ARG, "operator is null");
    pc_context *ctx = op->ctx;
    if (adjoint != 0 && adjoint != 1) return fail(ctx, PC_ERR_ARG, "adjoint must be 0 or 1");
    if (nrhs < 0 || chunk < 0) return fail(ctx, PC_ERR_ARG, "nrhs and chunk must be >= 0");
    if (nrhs == 0) return PC_OK;
    if (!x || !y) return fail(ctx, PC_ERR_ARG, "null x or y");
    if (ldx < op->N || ldy < op->N) return fail(ctx, PC_ERR_ARG, "ldx and ldy must be >= N");
    const int64_t el = int64_t(op->elem);
    const uintptr_t xa = reinterpret_cast<uintptr_t>(x), ya = reinterpret_cast<uintptr_t>(y);
    const uintptr_t xe = xa + uintptr_t((int64_t(nrhs - 1) * ldx + op->N) * el);
    const uintptr_t ye = ya + uintptr_t((int64_t(nrhs - 1) * ldy + op->N) * el);
    if (xa < ye && ya < xe) return fail(ctx, PC_ERR_ARG, "x and y overlap");
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return fail(ctx, PC_ERR_CUDA, "cannot select the context's device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    pc_status st = ensure_host_resources(op, 0);
    if (st != PC_OK) return st;
    // chunks of an even number of right-hand sides keep the pairs (and so the
    // rounding) of one apply of the whole batch
    auto even = [&](int32_t v) { return v >= nrhs ? nrhs : v + (v & 1); };
    if (op->d == 2) {
        // one segmented launch: chunks of about a quarter of the batch (a
        // segment's colour chain is its critical path, so smaller chunks run
        // longer), at most kMaxSegments of them
        int32_t c = even(std::max<int32_t>(chunk > 0 ? chunk : (nrhs + 3) / 4,
                                           (nrhs + pc::kMaxSegments - 1) / pc::kMaxSegments));
        if (segmented_host_apply() && op->parts.empty())
            return apply_host_segmented(op, nrhs, x, ldx, y, ldy, adjoint == 1, c, s);
        return apply_host_chunked(op, nrhs, x, ldx, y, ldy, adjoint == 1, c, s);
    }
    // 3D: the chunked pipeline, by default in one chunk (the 3D patch kernels
    // take nearly as long for a quarter of a batch as for all of it)
    const int32_t c = even(chunk > 0 ? chunk : nrhs);
    return apply_host_chunked(op, nrhs, x, ldx, y, ldy, adjoint == 1, c, s);
}

pc_status pc_estimate_cell_errors(pc_operator *op, int32_t q, const void *z, int64_t ldz, const void *y, int64_t ldy,
                                  double *eta, pc_stream stream) {
    if (!op) return fail(nullptr, PC_ERR_ARG, "operator is null");
    pc_context *ctx = op->ctx;
    if (q < 1) return fail(ctx, PC_ERR_ARG, "q must be >= 1");
    if (!z || !y || !eta) return fail(ctx, PC_ERR_ARG, "null z, y or eta");
    if (ldy < op->N) return fail(ctx, PC_ERR_ARG, "ldy must be >= N");
    if (reinterpret_cast<uintptr_t>(y) % op->elem) return fail(ctx, PC_ERR_ARG, "y must be aligned to the element size");
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return fail(ctx, PC_ERR_CUDA, "cannot select the context's device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e = cudaSuccess;
    if (op->est_cap < q) {
        if (op->d_est && (e = cudaDeviceSynchronize()) != cudaSuccess)
            return cuda_fail(ctx, e, "synchronising before growing the estimator scratch");
        cudaFree(op->d_est);
        op->d_est = nullptr;
        op->est_cap = 0;
        if ((e = cudaMalloc(&op->d_est, size_t(q) * size_t(op->N) * op->elem)) != cudaSuccess)
            return cuda_fail(ctx, e, "allocating the estimator scratch");
        op->est_cap = q;
    }
    // Y~ = A~* Z, then the per-cell sums of squares of Y~ - Y
    pc_status st = apply_batched(op, q, z, ldz, op->d_est, op->N, stream, true);
    if (st != PC_OK) return st;
    // extents of the canonical box's two fastest axes (2D grids as (1, n0, n1))
    const int64_t n1 = op->d == 2 ? op->shape[0] : op->shape[1];
    const int64_t n2 = op->d == 2 ? op->shape[1] : op->shape[2];
    if ((e = pc::launch_cell_sqdiff(op->prec, op->d_est, op->N, y, ldy, q, op->d_cells, op->n_cells, n1, n2,
                                    op->d_cell_sums, s)) != cudaSuccess)
        return cuda_fail(ctx, e, "launching the cell reduction");
    std::vector<double> sums(size_t(op->n_cells));
    if ((e = cudaMemcpyAsync(sums.data(), op->d_cell_sums, sizeof(double) * sums.size(), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(ctx, e, "reading the cell sums");
    for (int c = 0; c < op->n_cells; ++c) eta[c] = std::sqrt(sums[size_t(c)] / double(q));
    op->launches_last += 1;
    return PC_OK;
}

pc_status pc_entries(pc_operator *op, int64_t n, const int64_t *rows, const int64_t *cols, double *out,
                     pc_stream stream) {
    if (!op) return fail(nullptr, PC_ERR_ARG, "operator is null");
    if (n < 0) return fail(op->ctx, PC_ERR_ARG, "n < 0");
    if (n == 0) return PC_OK;
    if (!rows || !cols || !out) return fail(op->ctx, PC_ERR_ARG, "null rows, cols or out");
    DeviceGuard dg(op->ctx->device);
    if (!dg.ok) return fail(op->ctx, PC_ERR_CUDA, "cannot select the context's device");
    const cudaError_t e = pc::launch_entries(op->prec, n, rows, cols, out, op->entry, op->d_w,
                                             static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(op->ctx, e, "launching the entries kernel");
    return PC_OK;
}

pc_status pc_apply(pc_operator *op, const void *x, void *y, pc_stream stream) {
    if (!op) return fail(nullptr, PC_ERR_ARG, "operator is null");
    return pc_apply_batched(op, 1, x, op->N, y, op->N, stream);
}

pc_status pc_apply_plain(pc_operator *op, int32_t nrhs, const void *x, int64_t ldx, void *y, int64_t ldy,
                         pc_stream stream) {
    if (!op) return fail(nullptr, PC_ERR_ARG, "operator is null");
    pc_context *ctx = op->ctx;
    if (op->prec == PC_FP64) return fail(ctx, PC_ERR_UNSUPPORTED, "the plain path covers FP32 spectra (FP32, BF16X3)");
    if (!op->parts.empty())
        return fail(ctx, PC_ERR_UNSUPPORTED, "the plain path covers operators with one launch shape");
    if (nrhs < 0) return fail(ctx, PC_ERR_ARG, "nrhs < 0");
    if (nrhs == 0) return PC_OK;
    if (!x || !y) return fail(ctx, PC_ERR_ARG, "null x or y");
    if (ldx < op->N || ldy < op->N) return fail(ctx, PC_ERR_ARG, "ldx and ldy must be >= N");
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return fail(ctx, PC_ERR_CUDA, "cannot select the context's device");
    std::string err;
    pc_status st = pc::plain_apply(op, nrhs, x, ldx, y, ldy, static_cast<cudaStream_t>(stream), err);
    if (st != PC_OK) return fail(ctx, st, err);
    op->last_stream = static_cast<cudaStream_t>(stream);
    return PC_OK;
}

pc_status pc_operator_check(pc_operator *op) {
    if (!op) return fail(nullptr, PC_ERR_ARG, "operator is null");
    DeviceGuard dg(op->ctx->device);
    cudaError_t e = cudaStreamSynchronize(op->last_stream);
    if (e != cudaSuccess) return cuda_fail(op->ctx, e, "asynchronous CUDA error");
    int32_t ctrl[4] = {0, 0, 0, 0};
    e = cudaMemcpy(ctrl, op->d_ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(op->ctx, e, "reading the status word");
    if (ctrl[2]) {
        pc::zero_now(op->d_ctrl + 2, sizeof(int32_t));
        return fail(op->ctx, PC_ERR_TIMEOUT, "a bounded wait in the patch kernel timed out");
    }
    return PC_OK;
}

pc_status pc_operator_kernel_time(pc_operator *op, float *ms) {
    if (!op || !ms) return fail(nullptr, PC_ERR_ARG, "null argument");
    if (!op->timed) return fail(op->ctx, PC_ERR_NOT_READY, "no apply has been issued");
    DeviceGuard dg(op->ctx->device);
    cudaError_t e = cudaEventSynchronize(op->ev_end);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, op->ev_begin, op->ev_end);
    if (e != cudaSuccess) return cuda_fail(op->ctx, e, "reading kernel events");
    return PC_OK;
}

pc_status pc_operator_stage_time(pc_operator *op, int32_t stage, float *ms) {
    if (!op || !ms) return fail(nullptr, PC_ERR_ARG, "null argument");
    if (stage < 0 || stage > 2) return fail(op->ctx, PC_ERR_ARG, "stage must be 0, 1 or 2");
    if (!op->timed || op->stage_chunks == 0)
        return fail(op->ctx, PC_ERR_NOT_READY, "no staged (3D BF16X3) apply has been issued");
    DeviceGuard dg(op->ctx->device);
    cudaError_t e = cudaEventSynchronize(op->ev_end);
    float sum = 0.0f;
    for (int c = 0; c < op->stage_chunks && e == cudaSuccess; ++c) {
        float t = 0.0f;
        e = cudaEventElapsedTime(&t, op->stage_ev[size_t(c) * 6 + 2 * stage], op->stage_ev[size_t(c) * 6 + 2 * stage + 1]);
        sum += t;
    }
    if (e != cudaSuccess) return cuda_fail(op->ctx, e, "reading stage events");
    *ms = sum;
    return PC_OK;
}

pc_status pc_operator_launches(const pc_operator *op, int64_t *kernels_last_apply) {
    if (!op || !kernels_last_apply) return fail(nullptr, PC_ERR_ARG, "null argument");
    *kernels_last_apply = op->launches_last;
    return PC_OK;
}

pc_status pc_operator_destroy(pc_operator *op) {
    if (!op) return PC_OK;
    pc_context *ctx = op->ctx;
    DeviceGuard dg(ctx->device);
    const cudaError_t se = cudaDeviceSynchronize();
    const char *bad = free_operator(op);
    if (se != cudaSuccess) return cuda_fail(ctx, se, "synchronising before the operator was freed");
    if (bad) return fail(ctx, PC_ERR_CUDA, std::string("freeing the operator: ") + bad);
    return PC_OK;
}

}  // extern "C"

namespace pc {
pc_status prepare_batch(pc_operator *op, int32_t nrhs) { return prepare_batch_impl(op, nrhs); }
}  // namespace pc
