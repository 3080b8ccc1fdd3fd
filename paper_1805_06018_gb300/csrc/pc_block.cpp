// Block apply (Section 3.3): plans of one or several blocks A~[T, S] or
// (A~*)[T, S] of an operator, and their launches.
#include <algorithm>
#include <cstring>
#include <utility>

#include "pc_api_util.h"
#include "pc_internal.h"

using pc::cuda_fail;
using pc::DeviceGuard;
using pc::fail;
using pc::upload;

namespace {

// Schedule of a block apply (Section 3.3), from the operator's schedule.
// A tile convolves its input box (inside bbox(U_k)) with one sub-window of
// phi_k^E; restricting x to a box C only clips that input box, and shifting
// the input box by delta shifts the tile's output box by delta with the same
// sub-window (the translation of Section 3.3), so the tile keeps its
// spectrum.  Forward: C = S and the output box must meet T; adjoint (which
// gathers x over the output box and adds into the input box): C = T and the
// output box must meet S.  Kept tiles are re-expressed in block coordinates:
// input boxes relative to C, output boxes relative to the other box.  A
// subset of a proper colouring is proper, and a clipped tile overlaps only
// tiles its original overlapped, so the colour order and the dependency
// lists restricted to kept tiles still order every sum.
struct BlockSchedule {
    std::vector<pc::Tile> tiles;
    std::vector<int32_t> color_start{0}, dep_start{0}, dep;
    int terms = 0;
};

void build_block_schedule(const pc_operator *op, const int64_t *t_lo, const int64_t *t_hi, const int64_t *s_lo,
                          const int64_t *s_hi, bool adjoint, BlockSchedule &b) {
    const int d = op->d;
    const int64_t *clo = adjoint ? t_lo : s_lo, *chi = adjoint ? t_hi : s_hi;
    const int64_t *olo = adjoint ? s_lo : t_lo, *ohi = adjoint ? s_hi : t_hi;
    std::vector<int32_t> remap(op->tiles_h.size(), -1);
    std::vector<char> used(size_t(op->r), 0);
    for (int c = 0; c < op->n_colors; ++c) {
        for (int ti = op->color_start_h[size_t(c)]; ti < op->color_start_h[size_t(c) + 1]; ++ti) {
            const pc::Tile &t = op->tiles_h[size_t(ti)];
            int64_t delta[3] = {0, 0, 0}, ext[3] = {1, 1, 1};
            bool keep = true;
            for (int a = 0; a < d && keep; ++a) {
                const int64_t lo = std::max<int64_t>(t.in_lo[a], clo[a]);
                const int64_t hi = std::min<int64_t>(int64_t(t.in_lo[a]) + t.in_ext[a] - 1, chi[a]);
                delta[a] = lo - t.in_lo[a];
                ext[a] = hi - lo + 1;
                const int64_t o_lo = t.out_lo[a] + delta[a];
                const int64_t o_hi = o_lo + ext[a] + t.kext[a] - 2;
                keep = ext[a] > 0 && o_hi >= olo[a] && o_lo <= ohi[a];
            }
            if (!keep) continue;
            pc::Tile u = t;
            for (int a = 0; a < d; ++a) {
                u.in_lo[a] = int32_t(t.in_lo[a] + delta[a] - clo[a]);
                u.in_ext[a] = int32_t(ext[a]);
                u.out_lo[a] = int32_t(t.out_lo[a] + delta[a] - olo[a]);
            }
            // weight strides: 2D {ext1, 1}; 3D {ext1 * ext2, ext2} with unit stride on the last axis
            u.w_base = t.w_base + delta[0] * t.w_ld[0] + delta[1] * t.w_ld[1] + (d == 3 ? delta[2] : 0);
            remap[size_t(ti)] = int32_t(b.tiles.size());
            b.tiles.push_back(u);
            for (int q = op->dep_start_h[size_t(ti)]; q < op->dep_start_h[size_t(ti) + 1]; ++q) {
                const int32_t m = remap[size_t(op->dep_h[size_t(q)])];
                if (m >= 0) b.dep.push_back(m);
            }
            b.dep_start.push_back(int32_t(b.dep.size()));
            if (!used[size_t(t.patch)]) {
                used[size_t(t.patch)] = 1;
                ++b.terms;
            }
        }
        if (int32_t(b.tiles.size()) > b.color_start.back()) b.color_start.push_back(int32_t(b.tiles.size()));
    }
}

const char *free_block_plan(pc_block_plan *bp) {
    if (!bp) return nullptr;
    const char *bad = nullptr;
    auto chk = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && !bad) bad = what;
    };
    chk(cudaFree(bp->d_tiles), "tiles");
    chk(cudaFree(bp->d_color_start), "colours");
    chk(cudaFree(bp->d_dep_start), "dependency starts");
    chk(cudaFree(bp->d_dep), "dependencies");
    chk(cudaFree(bp->d_done), "ordering flags");
    chk(cudaFree(bp->d_ctrl), "control block");
    for (pc::LaunchDesc *h : bp->h_desc) chk(cudaFreeHost(h), "launch descriptors");
    for (char *h : bp->h_runs) chk(cudaFreeHost(h), "run tables");
    chk(cudaFree(bp->d_runs), "run tables");
    chk(cudaFree(bp->d_desc), "launch descriptors");
    chk(cudaFree(bp->d_seg_done), "segment counters");
    if (bp->desc_ev) chk(cudaEventDestroy(bp->desc_ev), "descriptor event");
    delete bp;
    return bad;
}

}  // namespace

extern "C" {

pc_status pc_block_plan_create_many(pc_operator *op, int32_t nblocks, const int64_t *t_lo, const int64_t *t_hi,
                                    const int64_t *s_lo, const int64_t *s_hi, int32_t adjoint, pc_block_plan **plan) {
    if (!plan) return fail(op ? op->ctx : nullptr, PC_ERR_ARG, "plan is null");
    *plan = nullptr;
    if (!op) return fail(nullptr, PC_ERR_ARG, "operator is null");
    pc_context *ctx = op->ctx;
    if (nblocks < 1) return fail(ctx, PC_ERR_ARG, "nblocks must be >= 1");
    if (!t_lo || !t_hi || !s_lo || !s_hi) return fail(ctx, PC_ERR_ARG, "null box bound");
    if (adjoint != 0 && adjoint != 1) return fail(ctx, PC_ERR_ARG, "adjoint must be 0 or 1");
    if (!op->parts.empty()) return fail(ctx, PC_ERR_UNSUPPORTED, "block plans cover operators with one launch shape");
    if (op->prec == PC_BF16X3) return fail(ctx, PC_ERR_UNSUPPORTED, "block applies cover FP32 and FP64 operators");
    const int d = op->d;
    for (int32_t i = 0; i < nblocks; ++i)
        for (int a = 0; a < d; ++a) {
            const int64_t j = int64_t(i) * d + a;
            if (t_lo[j] < 0 || t_lo[j] > t_hi[j] || t_hi[j] >= op->shape[size_t(a)])
                return fail(ctx, PC_ERR_ARG, "target box T must satisfy 0 <= lo <= hi < shape");
            if (s_lo[j] < 0 || s_lo[j] > s_hi[j] || s_hi[j] >= op->shape[size_t(a)])
                return fail(ctx, PC_ERR_ARG, "source box S must satisfy 0 <= lo <= hi < shape");
        }
    auto *bp = new (std::nothrow) pc_block_plan;
    if (!bp) return fail(ctx, PC_ERR_NOMEM, "out of host memory");
    bp->op = op;
    bp->adjoint = adjoint == 1;
    std::vector<pc::Tile> tiles;
    std::vector<int32_t> cs, ds, dep;
    for (int32_t i = 0; i < nblocks; ++i) {
        BlockSchedule b;
        build_block_schedule(op, t_lo + d * i, t_hi + d * i, s_lo + d * i, s_hi + d * i, adjoint == 1, b);
        pc_block_plan::Block blk{};
        for (int a = 0; a < 3; ++a) {
            blk.t_ext[a] = a < d ? t_hi[d * i + a] - t_lo[d * i + a] + 1 : 1;
            blk.s_ext[a] = a < d ? s_hi[d * i + a] - s_lo[d * i + a] + 1 : 1;
        }
        blk.nT = blk.t_ext[0] * blk.t_ext[1] * blk.t_ext[2];
        blk.nS = blk.s_ext[0] * blk.s_ext[1] * blk.s_ext[2];
        blk.tile_off = int32_t(tiles.size());
        blk.n_tiles = int32_t(b.tiles.size());
        blk.cs_off = int32_t(cs.size());
        blk.n_colors = int32_t(b.color_start.size()) - 1;
        blk.ds_off = int32_t(ds.size());
        blk.dep_off = int32_t(dep.size());
        blk.terms = b.terms;
        tiles.insert(tiles.end(), b.tiles.begin(), b.tiles.end());
        cs.insert(cs.end(), b.color_start.begin(), b.color_start.end());
        ds.insert(ds.end(), b.dep_start.begin(), b.dep_start.end());
        dep.insert(dep.end(), b.dep.begin(), b.dep.end());
        bp->blocks.push_back(blk);
        bp->n_tiles += blk.n_tiles;
        bp->terms += blk.terms;
    }
    if (dep.empty()) dep.push_back(0);
    bp->cs_h = cs;
    DeviceGuard dg(ctx->device);
    if (!dg.ok) {
        free_block_plan(bp);
        return fail(ctx, PC_ERR_CUDA, "cannot select the context's device");
    }
    size_t acct = 0;
    auto bail = [&](cudaError_t ee, const char *what) {
        pc_status s2 = cuda_fail(ctx, ee, what);
        free_block_plan(bp);
        return s2;
    };
    cudaError_t e;
    if (!tiles.empty() && (e = upload(&bp->d_tiles, tiles.data(), tiles.size(), acct)) != cudaSuccess)
        return bail(e, "tiles");
    if ((e = upload(&bp->d_color_start, cs.data(), cs.size(), acct)) != cudaSuccess ||
        (e = upload(&bp->d_dep_start, ds.data(), ds.size(), acct)) != cudaSuccess ||
        (e = upload(&bp->d_dep, dep.data(), dep.size(), acct)) != cudaSuccess)
        return bail(e, "colours and dependencies");
    if ((e = cudaMalloc(&bp->d_ctrl, 64)) != cudaSuccess) return bail(e, "control block");
    if ((e = cudaMemset(bp->d_ctrl, 0, 64)) != cudaSuccess) return bail(e, "control block");
    if (nblocks > 1 && d == 2) {
        const int rounds = (nblocks + pc::kMaxSegments - 1) / pc::kMaxSegments;
        for (int rnd = 0; rnd < rounds; ++rnd) {
            int32_t runs = 0;
            for (int32_t i = rnd * pc::kMaxSegments; i < std::min(nblocks, (rnd + 1) * pc::kMaxSegments); ++i)
                runs += bp->blocks[size_t(i)].n_colors;
            bp->run_cap = std::max(bp->run_cap, runs);
        }
        const size_t run_bytes = 8 * size_t(bp->run_cap + 1) + 8 * size_t(bp->run_cap);
        for (int rnd = 0; rnd < rounds; ++rnd) {
            pc::LaunchDesc *h = nullptr;
            char *hr = nullptr;
            if ((e = cudaHostAlloc(reinterpret_cast<void **>(&h), sizeof(pc::LaunchDesc), 0)) != cudaSuccess)
                return bail(e, "launch descriptors");
            bp->h_desc.push_back(h);
            if ((e = cudaHostAlloc(reinterpret_cast<void **>(&hr), run_bytes, 0)) != cudaSuccess)
                return bail(e, "run tables");
            bp->h_runs.push_back(hr);
        }
        if ((e = cudaMalloc(&bp->d_runs, run_bytes * size_t(rounds))) != cudaSuccess) return bail(e, "run tables");
        if ((e = cudaMalloc(&bp->d_desc, sizeof(pc::LaunchDesc) * size_t(rounds))) != cudaSuccess ||
            (e = cudaMalloc(&bp->d_seg_done, sizeof(uint32_t) * pc::kMaxSegments)) != cudaSuccess ||
            (e = cudaEventCreateWithFlags(&bp->desc_ev, cudaEventDisableTiming)) != cudaSuccess)
            return bail(e, "launch descriptors");
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return bail(e, "synchronising after the plan's uploads");
    *plan = bp;
    return PC_OK;
}

pc_status pc_block_plan_create(pc_operator *op, const int64_t *t_lo, const int64_t *t_hi, const int64_t *s_lo,
                               const int64_t *s_hi, int32_t adjoint, pc_block_plan **plan) {
    return pc_block_plan_create_many(op, 1, t_lo, t_hi, s_lo, s_hi, adjoint, plan);
}

pc_status pc_block_apply_many(pc_block_plan *bp, int32_t nrhs, const void *const *x, const int64_t *ldx,
                              void *const *y, const int64_t *ldy, pc_stream stream) {
    if (!bp) return fail(nullptr, PC_ERR_ARG, "plan is null");
    pc_operator *op = bp->op;
    pc_context *ctx = op->ctx;
    if (nrhs < 0) return fail(ctx, PC_ERR_ARG, "nrhs < 0");
    if (nrhs == 0) return PC_OK;
    if (!x || !ldx || !y || !ldy) return fail(ctx, PC_ERR_ARG, "null pointer array");
    const int32_t nb = int32_t(bp->blocks.size());
    const int64_t el = int64_t(op->elem);
    std::vector<std::pair<uintptr_t, uintptr_t>> yr(static_cast<size_t>(nb));
    for (int32_t i = 0; i < nb; ++i) {
        const pc_block_plan::Block &b = bp->blocks[size_t(i)];
        if (!x[i] || !y[i]) return fail(ctx, PC_ERR_ARG, "null x or y");
        if (ldx[i] < b.nS || ldy[i] < b.nT) return fail(ctx, PC_ERR_ARG, "need ldx >= |S| and ldy >= |T|");
        const uintptr_t xa = reinterpret_cast<uintptr_t>(x[i]), ya = reinterpret_cast<uintptr_t>(y[i]);
        if (xa % op->elem || ya % op->elem) return fail(ctx, PC_ERR_ARG, "x and y must be aligned to the element size");
        const uintptr_t xe = xa + uintptr_t((int64_t(nrhs - 1) * ldx[i] + b.nS) * el);
        const uintptr_t ye = ya + uintptr_t((int64_t(nrhs - 1) * ldy[i] + b.nT) * el);
        if (xa < ye && ya < xe) return fail(ctx, PC_ERR_ARG, "x and y overlap");
        yr[size_t(i)] = {ya, ye};
    }
    if (nb > 1) {
        std::sort(yr.begin(), yr.end());
        for (size_t i = 1; i < yr.size(); ++i)
            if (yr[i].first < yr[i - 1].second) return fail(ctx, PC_ERR_ARG, "the blocks' y arrays overlap");
    }
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return fail(ctx, PC_ERR_CUDA, "cannot select the context's device");
    const int32_t npairs = (nrhs + 1) / 2;
    // flags per (tile, pair): one per output-plane group of a 3D apply
    const int32_t nflags = npairs * pc::flag_groups(op->d, op->prec);
    cudaError_t e = cudaSuccess;
    if (bp->n_tiles > 0 && nflags > bp->done_cap) {
        if (bp->launched && (e = cudaDeviceSynchronize()) != cudaSuccess)
            return cuda_fail(ctx, e, "synchronising before growing the plan's flags");
        cudaFree(bp->d_done);
        bp->d_done = nullptr;
        bp->done_cap = 0;
        const int32_t cap = std::max<int32_t>(nflags, 32);
        const size_t bytes = sizeof(uint32_t) * size_t(bp->n_tiles) * size_t(cap);
        if ((e = cudaMalloc(&bp->d_done, bytes)) != cudaSuccess) return cuda_fail(ctx, e, "allocating plan flags");
        if ((e = pc::zero_now(bp->d_done, bytes)) != cudaSuccess) return cuda_fail(ctx, e, "clearing plan flags");
        bp->done_cap = cap;
        bp->epoch = 0;
    }
    if (++bp->epoch == 0) bp->epoch = 1;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    auto params = [&](int32_t i) {
        const pc_block_plan::Block &b = bp->blocks[size_t(i)];
        pc::ApplyParams p{};
        p.x = x[i];
        p.y = y[i];
        p.ldx = ldx[i];
        p.ldy = ldy[i];
        p.nrhs = nrhs;
        p.npairs = npairs;
        for (int a = 0; a < 3; ++a) {
            p.n[a] = int32_t(b.t_ext[a]);
            p.nx[a] = int32_t(b.s_ext[a]);
        }
        p.R = op->R;
        p.tiles = bp->d_tiles ? bp->d_tiles + b.tile_off : nullptr;
        p.color_start = bp->d_color_start + b.cs_off;
        p.n_colors = b.n_colors;
        p.dep_start = bp->d_dep_start + b.ds_off;
        p.dep = bp->d_dep + b.dep_off;
        p.done = bp->d_done ? bp->d_done + int64_t(b.tile_off) * bp->done_cap : nullptr;
        p.done_ld = bp->done_cap;
        p.epoch = bp->epoch;
        p.ctrl = bp->d_ctrl;
        p.spec = op->d_spec;
        p.spec_stride = op->spec_stride;
        p.w = op->d_w;
        p.tw = op->d_tw;
        p.wait_ns = op->wait_ns;
        p.total_items = int64_t(b.n_tiles) * npairs;
        return p;
    };
    int64_t launches = 0;
    if (nb == 1 || op->d == 3) {
        // one block per launch (3D: the patch kernel runs one block at a time, on
        // the operator's scratch volumes)
        for (int32_t i = 0; i < nb; ++i) {
            const pc::ApplyParams p = params(i);
            if ((e = pc::launch_zero(p, bp->blocks[size_t(i)].nT, op->prec, s)) != cudaSuccess)
                return cuda_fail(ctx, e, "launching the zero kernel");
            ++launches;
            if (p.total_items > 0) {
                const int ctas = int(std::min<int64_t>(op->ctas, p.total_items));
                e = op->d == 3 ? pc::launch_fft3d(p, op->ctas, op->d_scratch, s, bp->adjoint)
                               : pc::launch_fft2d(p, op->P, op->prec, ctas, s, bp->adjoint);
                if (e != cudaSuccess) return cuda_fail(ctx, e, "launching the patch kernel");
                ++launches;
            }
        }
    } else {
        size_t smem = 0;
        if ((e = pc::fft2d_configure(op->P, op->prec, nullptr, &smem)) != cudaSuccess)
            return cuda_fail(ctx, e, "configuring the patch kernel");
        // the previous call's descriptor uploads have completed before the host descriptors are rewritten
        if (bp->launched && (e = cudaEventSynchronize(bp->desc_ev)) != cudaSuccess)
            return cuda_fail(ctx, e, "waiting for the previous descriptor upload");
        for (int32_t b0 = 0, rnd = 0; b0 < nb; b0 += pc::kMaxSegments, ++rnd) {
            const int32_t nseg = std::min<int32_t>(pc::kMaxSegments, nb - b0);
            pc::LaunchDesc &d = *bp->h_desc[size_t(rnd)];
            std::memset(&d, 0, sizeof(pc::LaunchDesc));
            int32_t maxc = 0;
            for (int32_t q = 0; q < nseg; ++q) {
                pc::Segment &sg = d.seg[q];
                sg.p = params(b0 + q);
                sg.slot = -1;
                maxc = std::max(maxc, bp->blocks[size_t(b0 + q)].n_colors);
            }
            // run table: colour-major across the round's blocks, so that every
            // colour step holds work of all of them; each run's dependencies
            // (lower colours of its own block) come earlier in the order
            const size_t run_bytes = 8 * size_t(bp->run_cap + 1) + 8 * size_t(bp->run_cap);
            char *hr = bp->h_runs[size_t(rnd)];
            int64_t *run_begin = reinterpret_cast<int64_t *>(hr);
            int32_t *run_segcol = reinterpret_cast<int32_t *>(hr + 8 * size_t(bp->run_cap + 1));
            int32_t nrun = 0;
            int64_t items = 0;
            for (int32_t c = 0; c < maxc; ++c)
                for (int32_t q = 0; q < nseg; ++q) {
                    const pc_block_plan::Block &b = bp->blocks[size_t(b0 + q)];
                    if (c >= b.n_colors) continue;
                    const int32_t ntc = bp->cs_h[size_t(b.cs_off + c + 1)] - bp->cs_h[size_t(b.cs_off + c)];
                    run_begin[nrun] = items;
                    run_segcol[2 * nrun] = q;
                    run_segcol[2 * nrun + 1] = c;
                    items += int64_t(ntc) * npairs;
                    ++nrun;
                }
            run_begin[nrun] = items;
            char *dr = bp->d_runs + run_bytes * size_t(rnd);
            d.nseg = nseg;
            d.nrun = nrun;
            d.total_items = items;
            d.run_begin = reinterpret_cast<const int64_t *>(dr);
            d.run_segcol = reinterpret_cast<const int32_t *>(dr + 8 * size_t(bp->run_cap + 1));
            pc::LaunchDesc *dd = bp->d_desc + rnd;
            if ((e = cudaMemcpyAsync(dd, &d, sizeof(pc::LaunchDesc), cudaMemcpyHostToDevice, s)) != cudaSuccess ||
                (e = cudaMemcpyAsync(dr, hr, run_bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
                return cuda_fail(ctx, e, "uploading a launch descriptor");
            const int ctas = int(std::max<int64_t>(1, std::min<int64_t>(op->ctas, items)));
            if ((e = pc::launch_round(dd, reinterpret_cast<unsigned long long *>(bp->d_ctrl), bp->d_ctrl + 2,
                                      bp->d_seg_done, nullptr, ctas, smem, s, op->P, op->prec, bp->adjoint)) !=
                cudaSuccess)
                return cuda_fail(ctx, e, "launching the blocks");
            launches += 2;
        }
        cudaEventRecord(bp->desc_ev, s);
    }
    bp->last_stream = s;
    bp->launched = true;
    (void)launches;
    return PC_OK;
}

pc_status pc_block_apply(pc_block_plan *bp, int32_t nrhs, const void *x, int64_t ldx, void *y, int64_t ldy,
                         pc_stream stream) {
    if (bp && bp->blocks.size() != 1)
        return fail(bp->op->ctx, PC_ERR_ARG, "the plan holds several blocks: use pc_block_apply_many");
    return pc_block_apply_many(bp, nrhs, &x, &ldx, &y, &ldy, stream);
}

pc_status pc_block_plan_info(const pc_block_plan *bp, int32_t *terms, int32_t *tiles) {
    if (!bp) return fail(nullptr, PC_ERR_ARG, "plan is null");
    if (terms) *terms = bp->terms;
    if (tiles) *tiles = bp->n_tiles;
    return PC_OK;
}

pc_status pc_block_plan_check(pc_block_plan *bp) {
    if (!bp) return fail(nullptr, PC_ERR_ARG, "plan is null");
    pc_context *ctx = bp->op->ctx;
    DeviceGuard dg(ctx->device);
    cudaError_t e = cudaStreamSynchronize(bp->last_stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "asynchronous CUDA error");
    int32_t ctrl[4] = {0, 0, 0, 0};
    if ((e = cudaMemcpy(ctrl, bp->d_ctrl, sizeof(ctrl), cudaMemcpyDeviceToHost)) != cudaSuccess)
        return cuda_fail(ctx, e, "reading the status word");
    if (ctrl[2]) {
        pc::zero_now(bp->d_ctrl + 2, sizeof(int32_t));
        return fail(ctx, PC_ERR_TIMEOUT, "a bounded wait in the patch kernel timed out");
    }
    return PC_OK;
}

pc_status pc_block_plan_destroy(pc_block_plan *bp) {
    if (!bp) return PC_OK;
    pc_context *ctx = bp->op->ctx;
    DeviceGuard dg(ctx->device);
    const cudaError_t se = cudaDeviceSynchronize();
    const char *bad = free_block_plan(bp);
    if (se != cudaSuccess) return cuda_fail(ctx, se, "synchronising before freeing the plan");
    if (bad) return fail(ctx, PC_ERR_CUDA, std::string("freeing the plan: ") + bad);
    return PC_OK;
}

}  // extern "C"
