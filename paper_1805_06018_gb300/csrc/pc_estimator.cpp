// Incremental randomized estimator for the adaptive construction
// (Algorithm 1, Section 2.8): per-point correlation blocks kept between the
// operators of successive refinement passes.
#include <algorithm>
#include <cmath>
#include <map>

#include "pc_api_util.h"
#include "pc_internal.h"

using pc::cuda_fail;
using pc::DeviceGuard;
using pc::fail;
using pc::upload_on;

extern "C" {

pc_status pc_estimator_create(pc_context *ctx, const pc_box *box, pc_precision prec, int32_t q, const void *z,
                              int64_t ldz, const void *y, int64_t ldy, pc_estimator **est) {
    if (!est) return fail(ctx, PC_ERR_ARG, "est is null");
    *est = nullptr;
    if (!ctx || !box || !z || !y) return fail(ctx, PC_ERR_ARG, "null context, box, z or y");
    if (box->ndim != 2) return fail(ctx, PC_ERR_UNSUPPORTED, "the incremental estimator covers 2D boxes");
    if (prec != PC_FP32 && prec != PC_FP64) return fail(ctx, PC_ERR_UNSUPPORTED, "precision must be PC_FP32 or PC_FP64");
    if (q < 1) return fail(ctx, PC_ERR_ARG, "q must be >= 1");
    const int64_t N = box->shape[0] * box->shape[1];
    if (box->shape[0] < 2 || box->shape[1] < 2 || ldz < N || ldy < N)
        return fail(ctx, PC_ERR_ARG, "bad box, or ldz / ldy < N");
    const size_t elem = prec == PC_FP64 ? 8 : 4;
    if (reinterpret_cast<uintptr_t>(z) % elem || reinterpret_cast<uintptr_t>(y) % elem)
        return fail(ctx, PC_ERR_ARG, "z and y must be aligned to the element size");
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return fail(ctx, PC_ERR_CUDA, "cannot select the context's device");
    auto *e = new (std::nothrow) pc_estimator;
    if (!e) return fail(ctx, PC_ERR_NOMEM, "out of host memory");
    e->ctx = ctx;
    e->prec = prec;
    e->elem = elem;
    e->shape[0] = box->shape[0];
    e->shape[1] = box->shape[1];
    e->N = N;
    e->q = q;
    e->z = z;
    e->ldz = ldz;
    e->y = y;
    e->ldy = ldy;
    const cudaError_t ce = cudaMalloc(&e->d_yt, elem * size_t(q) * size_t(N));
    if (ce != cudaSuccess) {
        delete e;
        return cuda_fail(ctx, ce, "allocating the estimator scratch");
    }
    *est = e;
    return PC_OK;
}

pc_status pc_estimator_update(pc_estimator *est, pc_operator *op, double *eta, int32_t *recomputed,
                              pc_stream stream) {
    if (!est) return fail(nullptr, PC_ERR_ARG, "estimator is null");
    pc_context *ctx = est->ctx;
    if (!op || !eta) return fail(ctx, PC_ERR_ARG, "null operator or eta");
    if (op->d != 2 || op->shape[0] != est->shape[0] || op->shape[1] != est->shape[1])
        return fail(ctx, PC_ERR_ARG, "the operator's box differs from the estimator's");
    if (op->prec != est->prec) return fail(ctx, PC_ERR_ARG, "the operator's precision differs from the estimator's");
    if (!op->parts.empty())
        return fail(ctx, PC_ERR_UNSUPPORTED, "the incremental estimator covers operators with one launch shape");
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return fail(ctx, PC_ERR_CUDA, "cannot select the context's device");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int r = op->r;
    const int32_t q = est->q, nsub = op->split.nsub, nsub2 = nsub * nsub;
    // layout of the new arena; kept blocks and points to recompute
    std::vector<int64_t> blk_off(size_t(std::max(r, 1)), 0), copies;
    std::vector<char> marked(size_t(std::max(r, 1)), 0);
    std::map<std::pair<int32_t, int32_t>, pc_estimator::Entry> next;
    int64_t total = 0;
    int32_t nmarked = 0;
    for (int k = 0; k < r; ++k) {
        pc_estimator::Entry ne{};
        for (int a = 0; a < 2; ++a) {
            ne.bb_lo[a] = op->bb_lo_h[size_t(k) * 3 + size_t(a)];
            ne.bb_ext[a] = op->bb_ext_h[size_t(k) * 3 + size_t(a)];
        }
        ne.hash = op->phiE_hash[size_t(k)];
        ne.P = op->P;
        ne.T = op->T;
        ne.nsub = nsub;
        ne.off = total;
        ne.len = int64_t(nsub2) * q * int64_t(ne.bb_ext[0]) * ne.bb_ext[1];
        blk_off[size_t(k)] = total;
        total += ne.len;
        const std::pair<int32_t, int32_t> key{op->pts_h[size_t(k) * 3], op->pts_h[size_t(k) * 3 + 1]};
        const auto it = est->cache.find(key);
        const bool same = it != est->cache.end() && it->second.hash == ne.hash && it->second.P == ne.P &&
                          it->second.T == ne.T && it->second.nsub == ne.nsub && it->second.len == ne.len &&
                          std::equal(ne.bb_lo, ne.bb_lo + 2, it->second.bb_lo) &&
                          std::equal(ne.bb_ext, ne.bb_ext + 2, it->second.bb_ext);
        if (same) {
            copies.insert(copies.end(), {it->second.off, ne.off, ne.len});
        } else {
            marked[size_t(k)] = 1;
            ++nmarked;
        }
        next[key] = ne;
    }
    // the recomputed points' tiles, each storing its block (one colour, no ordering needed)
    std::vector<pc::Tile> tiles;
    std::vector<pc::StoreDesc> sds;
    for (const pc::Tile &t : op->tiles_h) {
        const int k = t.patch;
        if (!marked[size_t(k)]) continue;
        const int sw = t.spec - k * nsub2;
        const int64_t lo0 = op->bb_lo_h[size_t(k) * 3], lo1 = op->bb_lo_h[size_t(k) * 3 + 1];
        const int64_t e0 = op->bb_ext_h[size_t(k) * 3], e1 = op->bb_ext_h[size_t(k) * 3 + 1];
        pc::StoreDesc sd{};
        sd.off = blk_off[size_t(k)] + int64_t(sw) * q * e0 * e1 + (t.in_lo[0] - lo0) * e1 + (t.in_lo[1] - lo1);
        sd.ld_rhs = e0 * e1;
        sd.ld_row = int32_t(e1);
        tiles.push_back(t);
        sds.push_back(sd);
    }
    const int32_t nt = int32_t(tiles.size());
    const int32_t npairs = (q + 1) / 2;
    // device work, all of it ordered on s (the host vectors outlive it: the
    // call ends by synchronising s); every buffer is released before it returns
    void *arena = nullptr;
    pc::Tile *d_tiles = nullptr;
    pc::StoreDesc *d_sd = nullptr;
    int32_t *d_cs = nullptr, *d_ds = nullptr, *d_dep = nullptr, *d_ctrl = nullptr;
    uint32_t *d_done = nullptr;
    int64_t *d_blk = nullptr, *d_copies = nullptr;
    double *d_sums = nullptr;
    size_t acct = 0;
    auto release = [&]() {
        cudaFree(d_tiles);
        cudaFree(d_sd);
        cudaFree(d_cs);
        cudaFree(d_ds);
        cudaFree(d_dep);
        cudaFree(d_ctrl);
        cudaFree(d_done);
        cudaFree(d_blk);
        cudaFree(d_copies);
        cudaFree(d_sums);
    };
    auto bail = [&](cudaError_t ce, const char *what) {
        cudaStreamSynchronize(s);
        release();
        cudaFree(arena);
        return cuda_fail(ctx, ce, what);
    };
    cudaError_t e = cudaMalloc(&arena, est->elem * size_t(std::max<int64_t>(total, 1)));
    if (e != cudaSuccess) return bail(e, "allocating the correlation arena");
    if (!copies.empty()) {
        if ((e = upload_on(&d_copies, copies.data(), copies.size(), acct, s)) != cudaSuccess)
            return bail(e, "uploading the block copies");
        if ((e = pc::launch_block_copies(est->prec, d_copies, int32_t(copies.size() / 3), est->arena, arena, s)) !=
            cudaSuccess)
            return bail(e, "launching the block copies");
    }
    if (nt > 0) {
        const std::vector<int32_t> cs{0, nt}, ds(size_t(nt) + 1, 0), dep{0};
        if ((e = upload_on(&d_tiles, tiles.data(), tiles.size(), acct, s)) != cudaSuccess ||
            (e = upload_on(&d_sd, sds.data(), sds.size(), acct, s)) != cudaSuccess ||
            (e = upload_on(&d_cs, cs.data(), cs.size(), acct, s)) != cudaSuccess ||
            (e = upload_on(&d_ds, ds.data(), ds.size(), acct, s)) != cudaSuccess ||
            (e = upload_on(&d_dep, dep.data(), dep.size(), acct, s)) != cudaSuccess ||
            (e = cudaMalloc(&d_done, sizeof(uint32_t) * size_t(nt) * size_t(npairs))) != cudaSuccess ||
            (e = cudaMemsetAsync(d_done, 0, sizeof(uint32_t) * size_t(nt) * size_t(npairs), s)) != cudaSuccess ||
            (e = cudaMalloc(&d_ctrl, 64)) != cudaSuccess || (e = cudaMemsetAsync(d_ctrl, 0, 64, s)) != cudaSuccess)
            return bail(e, "uploading the correlation work list");
        pc::ApplyParams p{};
        p.x = est->z;
        p.y = est->d_yt;   // not written in store mode
        p.ldx = est->ldz;
        p.ldy = est->N;
        p.nrhs = q;
        p.npairs = npairs;
        p.n[0] = int32_t(est->shape[0]);
        p.n[1] = int32_t(est->shape[1]);
        p.n[2] = 1;
        p.nx[0] = p.n[0];
        p.nx[1] = p.n[1];
        p.nx[2] = p.n[2];
        p.R = op->R;
        p.tiles = d_tiles;
        p.color_start = d_cs;
        p.n_colors = 1;
        p.dep_start = d_ds;
        p.dep = d_dep;
        p.done = d_done;
        p.done_ld = npairs;
        p.epoch = 1u;
        p.ctrl = d_ctrl;
        p.spec = op->d_spec;
        p.spec_stride = op->spec_stride;
        p.w = op->d_w;
        p.tw = op->d_tw;
        p.wait_ns = op->wait_ns;
        p.total_items = int64_t(nt) * npairs;
        p.store = d_sd;
        p.store_base = arena;
        const int ctas = int(std::min<int64_t>(op->ctas, p.total_items));
        if ((e = pc::launch_fft2d(p, op->P, op->prec, ctas, s, true)) != cudaSuccess)
            return bail(e, "launching the correlations");
    }
    if ((e = upload_on(&d_blk, blk_off.data(), blk_off.size(), acct, s)) != cudaSuccess)
        return bail(e, "uploading the block offsets");
    if ((e = pc::launch_corr_combine(est->prec, op->entry, op->d_w, arena, d_blk, nsub2, q, est->d_yt, est->N, s)) !=
        cudaSuccess)
        return bail(e, "launching the combination");
    if ((e = cudaMalloc(&d_sums, sizeof(double) * size_t(std::max(op->n_cells, 1)))) != cudaSuccess)
        return bail(e, "allocating the cell sums");
    if ((e = pc::launch_cell_sqdiff(est->prec, est->d_yt, est->N, est->y, est->ldy, q, op->d_cells, op->n_cells,
                                    est->shape[0], est->shape[1], d_sums, s)) != cudaSuccess)
        return bail(e, "launching the cell reduction");
    std::vector<double> sums(size_t(op->n_cells));
    int32_t ctrl[4] = {0, 0, 0, 0};
    if ((e = cudaMemcpyAsync(sums.data(), d_sums, sizeof(double) * sums.size(), cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess ||
        (d_ctrl && (e = cudaMemcpyAsync(ctrl, d_ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost, s)) != cudaSuccess) ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return bail(e, "reading the cell sums");
    release();
    if (ctrl[2]) {
        // the new blocks are not trusted: keep the previous cache
        cudaFree(arena);
        return fail(ctx, PC_ERR_TIMEOUT, "a bounded wait in the correlation kernel timed out");
    }
    cudaFree(est->arena);
    est->arena = arena;
    est->cache.swap(next);
    est->recomputed_total += nmarked;
    if (recomputed) *recomputed = nmarked;
    for (int c = 0; c < op->n_cells; ++c) eta[c] = std::sqrt(sums[size_t(c)] / double(q));
    return PC_OK;
}

pc_status pc_estimator_destroy(pc_estimator *est) {
    if (!est) return PC_OK;
    pc_context *ctx = est->ctx;
    DeviceGuard dg(ctx->device);
    const cudaError_t se = cudaDeviceSynchronize();
    const cudaError_t e1 = cudaFree(est->d_yt), e2 = cudaFree(est->arena);
    delete est;
    if (se != cudaSuccess) return cuda_fail(ctx, se, "synchronising before freeing the estimator");
    if (e1 != cudaSuccess || e2 != cudaSuccess) return fail(ctx, PC_ERR_CUDA, "freeing the estimator");
    return PC_OK;
}

}  // extern "C"
