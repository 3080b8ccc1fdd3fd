// Autotuner: the launch shape of an operator chosen by timing candidates.
//
// pc_build_spectra with a NULL pc_tuning (and pc_autotune) enumerates the
// launch shapes an operator can take - padded FFT extent P, kernel-window
// split (sub-windows per axis), input tile extent T, persistent CTAs per SM -
// ranks them by a model of their FFT work, builds the most promising few and
// times a small batch on each with CUDA events on a private stream.  A
// candidate whose build or apply fails, or whose device status reports a
// timed-out wait, is dropped.  The fastest is kept.
//
// Work model of one candidate, per pair of right-hand sides (Section 3.2's
// FFT convolutions, one per input tile and kernel sub-window): a 2D item
// transforms its n1 non-zero input rows, all P columns forward and inverse,
// and its L1 = n1 + w1 - 1 output rows; a 3D item its n0 input planes (n1
// rows and P columns each), all P^2 first-axis lines forward and inverse,
// and its L0 output planes (P columns and L1 rows each).  Every line FFT of
// length P costs P log2 P.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

#include "pc_api_util.h"
#include "pc_internal.h"

namespace pc {
namespace {

struct Candidate {
    pc_tuning t{};
    double cost = 0;
};

// Tile extents of one axis of extent e cut into ceil(e / T) balanced tiles.
std::vector<int64_t> tile_extents(int64_t e, int T) {
    const int64_t nt = (e + T - 1) / T, base = e / nt, rem = e % nt;
    std::vector<int64_t> out;
    for (int64_t i = 0; i < nt; ++i) out.push_back(base + (i < rem ? 1 : 0));
    return out;
}

double model_cost(const Geometry &g, int R, int P, int nsub, int T) {
    const int W = 2 * R + 1, ws = (W + nsub - 1) / nsub;
    std::vector<int> wext;
    for (int s = 0; s < nsub; ++s) wext.push_back(std::min(ws, W - s * ws));
    const double line = double(P) * std::log2(double(P));
    double lines = 0;
    for (size_t k = 0; k < g.pts.size(); ++k) {
        const auto t0 = tile_extents(g.bb_hi[k][0] - g.bb_lo[k][0] + 1, T);
        const auto t1 = tile_extents(g.bb_hi[k][1] - g.bb_lo[k][1] + 1, T);
        if (g.d == 2) {
            for (int64_t a0 : t0)
                for (int w0 : wext)
                    lines += double(t1.size()) * nsub * double(a0 + 2 * P + (a0 + w0 - 1));
        } else {
            const auto t2 = tile_extents(g.bb_hi[k][2] - g.bb_lo[k][2] + 1, T);
            for (int64_t a0 : t0)
                for (int64_t a1 : t1)
                    for (int w0 : wext)
                        for (int w1 : wext)
                            lines += double(t2.size()) * nsub *
                                     double(a0 * (a1 + P) + 2.0 * P * P + (a0 + w0 - 1) * (P + (a1 + w1 - 1)));
        }
    }
    return lines * line;
}

// Modelled line-FFT work of patch k alone at shape (P, nsub, T), 2D.
double patch_cost(const Geometry &g, int k, int R, int P, int nsub, int T) {
    const int W = 2 * R + 1, ws = (W + nsub - 1) / nsub;
    const auto t0 = tile_extents(g.bb_hi[k][0] - g.bb_lo[k][0] + 1, T);
    const auto t1 = tile_extents(g.bb_hi[k][1] - g.bb_lo[k][1] + 1, T);
    double lines = 0;
    for (int64_t a0 : t0)
        for (int s = 0; s < nsub; ++s) {
            const int w0 = std::min(ws, W - s * ws);
            lines += double(t1.size()) * nsub * double(a0 + 2 * P + (a0 + w0 - 1));
        }
    return lines * double(P) * std::log2(double(P));
}

// Candidate launch shapes, best modelled first, at most `keep` of them, and
// in 2D the per-patch shape choice when the patches differ.
std::vector<Candidate> candidates(const Geometry &g, int R, pc_precision prec, int keep) {
    std::vector<Candidate> out;
    const bool three = g.d == 3;
    const int W = 2 * R + 1;
    std::vector<int> Ps = (three || prec == PC_FP64) ? std::vector<int>{64} : std::vector<int>{64, 128};
    for (int P : Ps)
        for (int nsub = 1; nsub <= 6; ++nsub) {
            const int ws = (W + nsub - 1) / nsub;
            const int cap = three ? P : (2 * P) / 3;
            const int tmax = std::min(P - ws + 1, cap);
            if (tmax < 8) continue;
            for (int T : {tmax, std::max(8, (tmax * 3) / 4)}) {
                if (T != tmax && T >= tmax - 2) continue;
                for (int ctas : three ? std::vector<int>{0, 2} : std::vector<int>{0}) {
                    Candidate c;
                    c.t.fft_size = P;
                    c.t.window_split = nsub;
                    c.t.tile = T;
                    c.t.ctas_per_sm = ctas;
                    // fewer resident 3D CTAs: the same work, ranked just behind
                    c.cost = model_cost(g, R, P, nsub, T) * (ctas ? 1.0001 : 1.0);
                    out.push_back(c);
                }
            }
        }
    std::stable_sort(out.begin(), out.end(), [](const Candidate &a, const Candidate &b) { return a.cost < b.cost; });
    if (int(out.size()) > keep) out.resize(size_t(keep));
    if (!three) {
        // one shape per patch (a part per shape), when the patches differ in their best shape
        std::vector<std::array<int, 2>> shapes;
        choose_patch_shapes(g, R, prec, shapes);
        bool mixed = false;
        for (const auto &sh : shapes) mixed = mixed || sh != shapes[0];
        if (mixed) {
            Candidate c;
            c.t.per_patch = 1;
            out.push_back(c);
        }
    }
    return out;
}

struct TimingBuffers {
    void *x = nullptr, *y = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    ~TimingBuffers() {
        if (s) cudaStreamSynchronize(s);
        cudaFree(x);
        cudaFree(y);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s) cudaStreamDestroy(s);
    }
};

// Time `nrhs` right-hand sides on op: one warm-up apply, then `reps`.
// Returns ms per apply, or a negative value if an apply or its status failed.
double time_apply(pc_operator *op, int32_t nrhs, int reps, TimingBuffers &tb) {
    const size_t bytes = size_t(nrhs) * size_t(op->N) * op->elem;
    if (!tb.x) {
        if (cudaMalloc(&tb.x, bytes) != cudaSuccess || cudaMalloc(&tb.y, bytes) != cudaSuccess ||
            cudaMemset(tb.x, 0, bytes) != cudaSuccess ||
            cudaStreamCreateWithFlags(&tb.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreate(&tb.e0) != cudaSuccess || cudaEventCreate(&tb.e1) != cudaSuccess ||
            cudaDeviceSynchronize() != cudaSuccess)
            return -1.0;
    }
    if (pc_apply_batched(op, nrhs, tb.x, op->N, tb.y, op->N, tb.s) != PC_OK) return -1.0;
    if (cudaEventRecord(tb.e0, tb.s) != cudaSuccess) return -1.0;
    for (int q = 0; q < reps; ++q)
        if (pc_apply_batched(op, nrhs, tb.x, op->N, tb.y, op->N, tb.s) != PC_OK) return -1.0;
    if (cudaEventRecord(tb.e1, tb.s) != cudaSuccess || cudaEventSynchronize(tb.e1) != cudaSuccess) return -1.0;
    if (pc_operator_check(op) != PC_OK) return -1.0;   // a wait that gave up invalidates the timing
    float ms = 0;
    if (cudaEventElapsedTime(&ms, tb.e0, tb.e1) != cudaSuccess) return -1.0;
    return double(ms) / reps;
}

// Build and time every candidate; the fastest operator is returned in *best
// (if best != nullptr), its tuning in *best_t and its time in *best_ms.
pc_status search(pc_context *ctx, const pc_box *box, const pc_grid *grid, int32_t radius, const double *impulse,
                 const double *weights, pc_precision prec, int32_t nrhs, pc_operator **best, pc_tuning *best_t,
                 double *best_ms, int *timed) {
    if (!ctx) return fail(nullptr, PC_ERR_ARG, "ctx is null");
    if (radius < 1) return fail(ctx, PC_ERR_ARG, "radius must be >= 1");
    Geometry g;
    std::string err;
    pc_status st = build_geometry(box, grid, g, err);
    if (st != PC_OK) return fail(ctx, st, err);
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return fail(ctx, PC_ERR_CUDA, "cannot select the context's device");
    std::vector<Candidate> cands;
    if (g.d == 3 && prec == PC_BF16X3) {
        cands.push_back(Candidate{});   // one shape: the tensor-core path fixes P and caps T
    } else {
        cands = candidates(g, radius, prec, g.d == 3 ? 3 : 4);
        if (cands.empty()) cands.push_back(Candidate{});   // the model's default shape
    }
    TimingBuffers tb;
    pc_operator *keep = nullptr;
    double bms = 1e300;
    pc_tuning bt{};
    std::string last_err = "no candidate";
    int n = 0;
    for (const Candidate &c : cands) {
        pc_operator *op = nullptr;
        if (pc_build_spectra(ctx, box, grid, radius, impulse, weights, prec, &c.t, &op) != PC_OK) {
            last_err = ctx->last_error;
            continue;
        }
        const double ms = time_apply(op, nrhs, g.d == 3 ? 2 : 3, tb);
        ++n;
        if (ms < 0) {
            last_err = "candidate apply failed: " + ctx->last_error;
            pc_operator_destroy(op);
            continue;
        }
        if (ms < bms) {
            bms = ms;
            bt = c.t;
            if (keep) pc_operator_destroy(keep);
            keep = best ? op : nullptr;
            if (!best) pc_operator_destroy(op);
        } else {
            pc_operator_destroy(op);
        }
    }
    if (timed) *timed = n;
    if (bms >= 1e300) return fail(ctx, PC_ERR_UNSUPPORTED, "no candidate launch shape could be built and timed: " + last_err);
    if (best) *best = keep;
    if (best_t) *best_t = bt;
    if (best_ms) *best_ms = bms;
    return PC_OK;
}

}  // namespace

void choose_patch_shapes(const Geometry &g, int R, pc_precision prec, std::vector<std::array<int, 2>> &shape) {
    const int W = 2 * R + 1;
    shape.assign(g.pts.size(), {0, 0});
    // FP32 patches take 128^2 or 256^2: 64^2 items do so little FFT work each
    // that their fixed cost (claim, barriers, spectrum copy, ordering wait)
    // dominates; measured on the adaptive 1024^2 workload, a {64, 128, 256}
    // choice ran 20.0 ms per 32 RHS against 16.0 ms for {128, 256}.  FP64: 64^2.
    std::vector<int> Ps = prec == PC_FP64 ? std::vector<int>{64} : std::vector<int>{128, kBigFft};
    for (size_t k = 0; k < g.pts.size(); ++k) {
        double best = 1e300;
        for (int P : Ps)
            for (int nsub = 1; nsub <= 8; ++nsub) {
                const int ws = (W + nsub - 1) / nsub;
                const int T = std::min(P - ws + 1, tile_cap(P));
                if (T < 8) continue;
                const double c = patch_cost(g, int(k), R, P, nsub, T);
                if (c < best * 0.999) {
                    best = c;
                    shape[k] = {P, nsub};
                }
            }
    }
}

pc_status autotune_build(pc_context *ctx, const pc_box *box, const pc_grid *grid, int32_t radius,
                         const double *impulse, const double *weights, pc_precision prec, pc_operator **out) {
    if (!out) return fail(ctx, PC_ERR_ARG, "null output handle");
    *out = nullptr;
    const auto t0 = std::chrono::steady_clock::now();
    pc_operator *op = nullptr;
    double ms = 0;
    int timed = 0;
    // batches as large as the workloads' (small batches favour shapes with
    // fewer, larger launches, which a 32-RHS apply no longer needs)
    const int32_t nrhs = box && box->ndim == 3 ? 8 : 32;
    pc_status st = search(ctx, box, grid, radius, impulse, weights, prec, nrhs, &op, nullptr, &ms, &timed);
    if (st != PC_OK) return st;
    op->autotuned = true;
    op->tuned_candidates = timed;
    op->tuned_ms = ms;
    op->build_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    *out = op;
    return PC_OK;
}

}  // namespace pc

extern "C" pc_status pc_autotune(pc_context *ctx, const pc_box *box, const pc_grid *grid, int32_t radius,
                                 const double *impulse, const double *weights, pc_precision prec, int32_t nrhs,
                                 pc_tuning *best, double *best_ms) {
    if (!ctx || !best || nrhs < 1) return pc::fail(ctx, PC_ERR_ARG, "null argument or nrhs < 1");
    return pc::search(ctx, box, grid, radius, impulse, weights, prec, nrhs, nullptr, best, best_ms, nullptr);
}
