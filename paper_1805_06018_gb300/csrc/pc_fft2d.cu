// Fused 2D patch kernel for y = sum_k phi_k^E * (w_k . x)  (Eq. conv_op_approx_main).
//
// One work item = (input tile of bbox(U_k), pair of right-hand sides).  Two
// real right-hand sides travel as the real and imaginary parts of one complex
// field: since phi_k^E is real, IFFT(FFT(u0 + i u1) . phi^_k) = (phi*u0) +
// i (phi*u1), so one complex P x P FFT serves two vectors with no unpacking.
//
//   phase A  gather w_k . x for the tile rows (coalesced global loads),
//            row FFTs (length P, pruned to the tile's n1 non-zero rows)
//   phase B  per column: FFT over the n1 non-zero rows, product with the
//            stored spectrum phi^_k (Section 3.2: convolution theorem after
//            zero padding to P >= n + 2R, so the circular product is the
//            linear convolution), inverse FFT; all in registers, one shared
//            memory round trip per column
//   phase C  inverse row FFTs of the L1 = n1 + 2R needed rows, then the
//            overlap-add of the L1 x L2 output box (clipped to Omega) into y
//
// Overlap-add order: tiles carry a colour such that tiles of one colour have
// disjoint output boxes; before adding, a tile waits (bounded spin) until
// every overlapping lower-colour tile of the same right-hand-side pair has
// added.  Each output pixel therefore sums its contributions in colour order,
// which makes y bitwise reproducible.  Items are taken from an atomic counter
// in colour-major order, so a tile only ever waits on items that were taken
// earlier by running CTAs: the wait always ends.
//
// The adjoint y = sum_k w_k . (flip(phi_k^E) * x) (Eq. adjoint_random_z, real
// data) is the same kernel with ADJ = true: phase A gathers x (unweighted)
// over the tile's output box, phase B multiplies by the conjugate spectrum
// (a correlation, free of wrap-around for the same P >= n + 2R), and phase
// C keeps the n1 x n2 input box, weights it by w_k and adds it there.  Tiles
// of one colour also have disjoint input boxes, so the adjoint sums in
// colour order as well.
#include "pc_fftcore.cuh"
#include "pc_internal.h"
#include "pc_overlap.cuh"
#include "pc_ptx.cuh"

namespace pc {

constexpr int kThreads2d = 512;
// Threads per CTA.  16 warps with 128 registers keep a line's 16 values and
// its 16 twiddles in registers; 32 warps at 64 registers (one line per
// column) spilled and measured slower on GB300 (1.22 ms vs 1.07 ms for the
// 512^2 x 64 workload).
template <typename T, int P> struct KCfg {
    static constexpr int threads = kThreads2d;
};

// Shared memory: the P x P complex workspace (padded rows, PadLayout), then
// the patch's half spectrum ([P/2+1] columns of P values, each followed by a
// copy of its value 0 at index P, so that the mirrored read of phase B,
// index P - k for k = 0 .. P-1, needs no wrap; rows padded to P + 8 values),
// then an mbarrier.
template <typename T, int P> struct Smem2d {
    using C = typename Cx<T>::type;
    static constexpr int PITCH = PadLayout<P>::pitch;
    static constexpr int SPLD = P + 8;
    // phase C reuses the spectrum region as one FP32 staging row per line:
    // re part [0, P+4), im part [P+12, 2P+16); the stride 2P+24 is 24 banks
    // mod 32, so the four lines of a warp write disjoint banks
    static constexpr int STAGE = 2 * P + 24;
    static constexpr int IMOFF = P + 12;
    static constexpr size_t ws = size_t(P) * PITCH * sizeof(C);
    static constexpr size_t spec = size_t(P / 2 + 1) * SPLD * sizeof(C);
    static constexpr size_t stage = size_t(KCfg<T, P>::threads / FftShape<P>::R2) * STAGE * sizeof(float);
    static constexpr size_t sp = spec > stage ? spec : stage;
    static constexpr size_t bytes = ws + sp + 16;
};

constexpr int kMaxColorsCached = 63;

// Column that line `line` transforms in phase B (round `rnd`): the two lines
// of a half-warp take columns c and c + 4, whose padded-workspace walks fall
// in disjoint banks (PadLayout).  A bijection of [0, LINES) for each round.
template <int LINES>
__device__ __forceinline__ int phase_b_col(int line, int rnd) {
    return rnd * LINES + (line & ~7) + ((line >> 1) & 3) + 4 * (line & 1);
}

// colour-major order: item -> (tile index, right-hand-side pair).  `cs` holds
// the colour offsets (shared-memory copy when there are few colours).  The
// search starts at colour `c` (in: a colour <= the item's, out: the item's):
// a CTA's claims only increase, so its previous item's colour is a valid
// start and the search is a step or two even with hundreds of colours.
__device__ __forceinline__ void decode_item(const ApplyParams &p, const int *cs, int64_t item, int &ti, int &pair,
                                            int &c) {
    while (int64_t(cs[c + 1]) * p.npairs <= item) ++c;
    const int64_t base = int64_t(cs[c]) * p.npairs;
    const int ntc = cs[c + 1] - cs[c];
    pair = int((item - base) / ntc);
    ti = cs[c] + int((item - base) % ntc);
}

__device__ __forceinline__ void prefetch_l2(const void *ptr) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(ptr));
}

// Pull the rows that `item` will gather into L2, one 128-byte line per
// thread-iteration: the weights and both right-hand sides over the input box
// (forward), or the right-hand sides over the output box clipped to the box x
// lives on (adjoint).
template <typename T, bool ADJ>
__device__ __forceinline__ void prefetch_item(const ApplyParams &p, const int *cs, int64_t item, int c) {
    if (item >= p.total_items) return;
    int ti, pair;
    decode_item(p, cs, item, ti, pair, c);
    const Tile tile = p.tiles[ti];
    constexpr int per_line = 128 / int(sizeof(T));
    const int b0 = 2 * pair;
    const int nx_arr = b0 + 1 < p.nrhs ? 2 : 1;
    int r0, nr, c0, nc, narr;
    if constexpr (!ADJ) {
        r0 = tile.in_lo[0], nr = tile.in_ext[0], c0 = tile.in_lo[1], nc = tile.in_ext[1];
        narr = nx_arr + 1;   // weights first
    } else {
        r0 = max(tile.out_lo[0], 0);
        nr = min(tile.out_lo[0] + tile.in_ext[0] + tile.kext[0] - 1, p.nx[0]) - r0;
        c0 = max(tile.out_lo[1], 0);
        nc = min(tile.out_lo[1] + tile.in_ext[1] + tile.kext[1] - 1, p.nx[1]) - c0;
        narr = nx_arr;
        if (nr <= 0 || nc <= 0) return;
    }
    const int lines_per_row = (nc + per_line - 1) / per_line + 1;   // +1: rows need not start on a line
    const int total = narr * nr * lines_per_row;
    for (int q = threadIdx.x; q < total; q += blockDim.x) {
        const int arr = q / (nr * lines_per_row);
        const int rem = q - arr * nr * lines_per_row;
        const int i = rem / lines_per_row, l = rem % lines_per_row;
        const int col = min(l * per_line, nc - 1);
        const T *base;
        if (!ADJ && arr == 0)
            base = static_cast<const T *>(p.w) + tile.w_base + int64_t(i) * tile.w_ld[0];
        else
            base = static_cast<const T *>(p.x) + int64_t(b0 + arr - (ADJ ? 0 : 1)) * p.ldx +
                   int64_t(r0 + i) * p.nx[1] + c0;
        prefetch_l2(base + col);
    }
}

// Overlap-add of one output row of a line: value m (< L2) goes to y[g0 + m]
// when 0 <= g0 + m < width.  FP32 stages the row and hands its aligned
// interior to bulk add-reductions (add_row_f32); FP64 adds element by element.
template <typename T, int P, typename C>
__device__ __forceinline__ void add_row(const C *a, int t, unsigned lmask, float *st, T *y0, T *y1, bool has1, int g0,
                                        int L2, int width) {
    constexpr int R1 = FftShape<P>::R1, R2 = FftShape<P>::R2;
    if constexpr (sizeof(T) == 8) {
        (void)st;
        (void)lmask;
#pragma unroll
        for (int j = 0; j < R1; ++j) {
            const int m = t + R2 * j;
            const int ox = g0 + m;
            if (m < L2 && ox >= 0 && ox < width) {
                atomicAdd(y0 + ox, a[j].x);
                if (has1) atomicAdd(y1 + ox, a[j].y);
            }
        }
    } else {
        add_row_f32<P>(a, t, lmask, st, Smem2d<T, P>::IMOFF, y0, y1, has1, g0, L2, width);
    }
}

// MULTI: launches through a descriptor, which may carry a run table (the
// claim order across segments); single-apply launches compile without it.
template <typename T, int P, bool ADJ, bool MULTI>
__global__ void __launch_bounds__(KCfg<T, P>::threads, 1) fft2d_kernel(const LaunchParams lp) {
    using C = typename Cx<T>::type;
    using L = Smem2d<T, P>;
    constexpr int R1 = FftShape<P>::R1, R2 = FftShape<P>::R2;
    constexpr int NT = KCfg<T, P>::threads;
    constexpr int LINES = NT / R2;
    constexpr int H = P / 2 + 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    C *S = reinterpret_cast<C *>(smem_raw);
    T *Sf = reinterpret_cast<T *>(smem_raw);
    C *SP = reinterpret_cast<C *>(smem_raw + L::ws);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw + L::ws + L::sp);
    __shared__ int64_t s_next_buf[2];   // claim of the next item, by item parity
    __shared__ int s_segidx;
    __shared__ int s_run, s_runcol;
    __shared__ int64_t s_runbase;
    __shared__ __align__(16) Segment s_seg;          // the current item's request
    __shared__ int s_cstart_buf[kMaxColorsCached + 1];
    // set once a wait of this launch has given up: the CTA takes no more items
    __shared__ int s_stop;

    const int nseg = lp.desc ? lp.desc->nseg : 1;
    const int nrun = MULTI && lp.desc ? lp.desc->nrun : 0;
    const int64_t total = lp.desc ? lp.desc->total_items : lp.one.p.total_items;
    constexpr int PITCH = L::PITCH;
    const int t = threadIdx.x % R2;
    const int line = threadIdx.x / R2;
    const unsigned lmask = FftShape<P>::line_mask();
    // every operator of a launch shares P, so the twiddle values W_P^k are the same
    const C *twg = static_cast<const C *>(lp.desc ? lp.desc->seg[0].p.tw : lp.one.p.tw);
    C tw[R1];   // W_P^{t m} for this thread's t
#pragma unroll
    for (int m = 0; m < R1; ++m) tw[m] = twg[(t * m) & (P - 1)];
    const C zero{T(0), T(0)};
    uint32_t phase = 0;
    int cur_seg = -1;
    int chint = 0;   // colour of this CTA's last item in the current segment
    const int *s_cstart = s_cstart_buf;
    // the last finished item's flag, published (by thread 0) once its
    // reductions have landed
    bool pend_flag_any = false;   // uniform: some item is awaiting publication
    __shared__ uint32_t *pend_flag, *pend_seg_done;
    __shared__ uint32_t pend_epoch;
    __shared__ int64_t pend_total;
    __shared__ int pend_slot;
    if (threadIdx.x == 0) pend_flag = nullptr;
    auto publish_pending = [&]() {
        if (!pend_flag) return;
        __threadfence();
        st_release_u32(pend_flag, pend_epoch);
        if (pend_seg_done) {
            // the request's last item raises its completion flag in host memory
            const uint32_t before = atomicAdd(pend_seg_done, 1u);
            if (int64_t(before) + 1 == pend_total && pend_slot >= 0 && lp.host_flags) {
                __threadfence_system();
                st_release_sys_u32(lp.host_flags + pend_slot, 1u);
            }
        }
        pend_flag = nullptr;
    };

    // one arrival per spectrum column: each copying thread announces its own bytes
    if (threadIdx.x == 0) {
        mbar_init(mbar, H);
        fence_mbar_init();
    }

    // Items are taken one ahead: while item i runs, item i+1 is already
    // claimed so its input rows can be pulled into L2.  Claims still happen in
    // increasing order, and the lowest unfinished item is always one that a
    // CTA is working on, so every dependency wait ends.
    unsigned long long *counter = lp.counter;
    if (threadIdx.x == 0) {
        s_next_buf[0] = int64_t(atomicAdd(counter, 1ull));
        s_run = 0;
        s_stop = 0;
    }
    __syncthreads();
    for (int par = 0;; par ^= 1) {
        // s_next_buf[par] and s_stop were written before the barrier that ended the previous item
        const int64_t gitem = s_next_buf[par];
        if (gitem >= total || s_stop) break;
        // the request (segment) this item belongs to (a single-apply launch has one)
        int segidx = 0;
        if (lp.desc) {
            if (threadIdx.x == 0) {
                if (MULTI && nrun > 0) {
                    // run table: resume where this CTA's last search ended (its claims increase)
                    int b = s_run;
                    while (b + 1 < nrun && lp.desc->run_begin[b + 1] <= gitem) ++b;
                    s_run = b;
                    s_runbase = lp.desc->run_begin[b];
                    s_segidx = lp.desc->run_segcol[2 * b];
                    s_runcol = lp.desc->run_segcol[2 * b + 1];
                } else {
                    int sx = MULTI && cur_seg > 0 ? cur_seg : 0;
                    while (sx + 1 < nseg && lp.desc->seg[sx + 1].item_begin <= gitem) ++sx;
                    s_segidx = sx;
                }
            }
            __syncthreads();
            segidx = s_segidx;
        }
        if (segidx != cur_seg) {
            cur_seg = segidx;
            chint = 0;
            if (lp.desc) {
                const uint32_t *src = reinterpret_cast<const uint32_t *>(lp.desc->seg + cur_seg);
                for (int q = threadIdx.x; q < int(sizeof(Segment) / 4); q += blockDim.x)
                    reinterpret_cast<uint32_t *>(&s_seg)[q] = src[q];
            } else if (threadIdx.x == 0) {
                s_seg = lp.one;
            }
            __syncthreads();
            // a segment whose input is still being copied in: wait (bounded) for its ready
            // word; if the wait gives up, the launch's result is invalid and the CTA stops
            if (threadIdx.x == 0 && s_seg.ready &&
                !wait_flag_eq<true>(s_seg.ready, s_seg.ready_val, lp.status, wait_limit_ns(s_seg.p.wait_ns), 1, 128))
                s_stop = 1;
            const int nc = s_seg.p.n_colors;
            s_cstart = nc <= kMaxColorsCached ? s_cstart_buf : s_seg.p.color_start;
            for (int c = threadIdx.x; c <= nc && c <= kMaxColorsCached; c += blockDim.x)
                s_cstart_buf[c] = s_seg.p.color_start[c];
            __syncthreads();
            if (s_stop) break;
        }
        const ApplyParams &p = s_seg.p;
        const int64_t item = gitem - s_seg.item_begin;
        const T *x = static_cast<const T *>(p.x);
        T *y = static_cast<T *>(p.y);
        const T *w = static_cast<const T *>(p.w);
        const C *spec = static_cast<const C *>(p.spec);
        int ti, pair;
        if (MULTI && nrun > 0) {
            // within a run: the colour's items in decode_item's order
            const int64_t local = gitem - s_runbase;
            const int c = s_runcol, ntc = s_cstart[c + 1] - s_cstart[c];
            pair = int(local / ntc);
            ti = s_cstart[c] + int(local % ntc);
        } else {
            decode_item(p, s_cstart, item, ti, pair, chint);
        }
        const Tile tile = p.tiles[ti];
        if (threadIdx.x == NT - 1) s_next_buf[par ^ 1] = int64_t(atomicAdd(counter, 1ull));
        const int n1 = tile.in_ext[0], n2 = tile.in_ext[1];
        const int i0 = tile.in_lo[0], j0 = tile.in_lo[1];
        const int L1 = n1 + tile.kext[0] - 1, L2 = n2 + tile.kext[1] - 1;   // <= P
        const int o0 = tile.out_lo[0], o1 = tile.out_lo[1];
        const int b0 = 2 * pair;
        const bool has1 = b0 + 1 < p.nrhs;
        const T *x0 = x + int64_t(b0) * p.ldx;
        const T *x1 = has1 ? x0 + p.ldx : x0;
        const T *wt = w + tile.w_base;

        // ---------------- the patch spectrum streams into shared memory (TMA bulk
        // copies, one per stored column) while phase A runs
        if (threadIdx.x < H) {
            const int col = threadIdx.x;
            const C *src = spec + int64_t(tile.spec) * p.spec_stride + int64_t(col) * P;
            fence_proxy_async_smem();
            mbar_arrive_expect_tx(mbar, uint32_t(P * sizeof(C) + 16));
            bulk_g2s(SP + col * L::SPLD, src, uint32_t(P * sizeof(C)), mbar);
            bulk_g2s(SP + col * L::SPLD + P, src, 16u, mbar);   // value 0 again, at index P
        }

        // ---------------- phase A: stage w, x0, x1 rows (cp.async), weight, row FFTs
        // rows of one warp sit 2P reals apart (same banks): shift each row's staging
        // by (row & 3) * 8 reals when the three arrays leave room
        if constexpr (!ADJ) {
            // staging of row i: the first 2 PITCH reals of the workspace row
            const int shmul = 3 * n2 + 24 <= 2 * PITCH ? 8 : 0;
            for (int i = line; i < n1; i += LINES) {
                T *row = Sf + i * 2 * PITCH + (i & 3) * shmul;
                const int64_t xr = int64_t(i0 + i) * p.nx[1] + j0;
                const T *wr = wt + int64_t(i) * tile.w_ld[0];
#pragma unroll
                for (int j = 0; j < R1; ++j) {
                    const int col = t + R2 * j;
                    if (col < n2) {
                        cp_async<sizeof(T)>(row + col, wr + col);
                        cp_async<sizeof(T)>(row + n2 + col, x0 + xr + col);
                        if (has1) cp_async<sizeof(T)>(row + 2 * n2 + col, x1 + xr + col);
                    }
                }
            }
            cp_async_wait_all();
            __syncwarp(lmask);
            for (int i = line; i < n1; i += LINES) {
                const T *row = Sf + i * 2 * PITCH + (i & 3) * shmul;
                C a[R1];
#pragma unroll
                for (int j = 0; j < R1; ++j) {
                    const int col = t + R2 * j;
                    if (col < n2) {
                        const T wv = row[col];
                        a[j] = C{wv * row[n2 + col], has1 ? wv * row[2 * n2 + col] : T(0)};
                    } else {
                        a[j] = zero;
                    }
                }
                C *Srow = S + i * PITCH + pad_shift(i);
                PadScratch<P, C, false> scr(Srow, t);
                fft_line<P, false>(a, tw, t, scr, lmask);
#pragma unroll
                for (int j = 0; j < R1; ++j) Srow[t + R2 * j] = a[j];
            }
        } else {
            // adjoint: x over the output box (L1 x L2 at (o0, o1)), zero outside
            // the box x lives on, staged as [x0 | x1] per row
            for (int i = line; i < L1; i += LINES) {
                const int gr = o0 + i;
                if (gr < 0 || gr >= p.nx[0]) continue;
                T *row = Sf + i * 2 * PITCH;
                const int64_t xr = int64_t(gr) * p.nx[1] + o1;
#pragma unroll
                for (int j = 0; j < R1; ++j) {
                    const int col = t + R2 * j;
                    const int gc = o1 + col;
                    if (col < L2 && gc >= 0 && gc < p.nx[1]) {
                        cp_async<sizeof(T)>(row + col, x0 + xr + col);
                        if (has1) cp_async<sizeof(T)>(row + L2 + col, x1 + xr + col);
                    }
                }
            }
            cp_async_wait_all();
            __syncwarp(lmask);
            for (int i = line; i < L1; i += LINES) {
                const int gr = o0 + i;
                const bool rin = gr >= 0 && gr < p.nx[0];
                const T *row = Sf + i * 2 * PITCH;
                C a[R1];
#pragma unroll
                for (int j = 0; j < R1; ++j) {
                    const int col = t + R2 * j;
                    const int gc = o1 + col;
                    a[j] = rin && col < L2 && gc >= 0 && gc < p.nx[1] ? C{row[col], has1 ? row[L2 + col] : T(0)}
                                                                    : zero;
                }
                C *Srow = S + i * PITCH + pad_shift(i);
                PadScratch<P, C, false> scr(Srow, t);
                fft_line<P, false>(a, tw, t, scr, lmask);
#pragma unroll
                for (int j = 0; j < R1; ++j) Srow[t + R2 * j] = a[j];
            }
        }
        // the previous item's bulk reductions have landed: it can report done
        if constexpr (sizeof(T) == 4) {
            if (t == 0 && pend_flag_any) {
                bulk_wait_all();
                fence_proxy_async_global();
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) publish_pending();

        if ((!MULTI || nrun == 0) && s_next_buf[par ^ 1] - s_seg.item_begin < p.total_items)
            prefetch_item<T, ADJ>(p, s_cstart, s_next_buf[par ^ 1] - s_seg.item_begin, chint);

        // ---------------- phase B: column FFT, spectral product, inverse column FFT
        // If the spectrum copy does not land within the limit, the item is
        // abandoned: the warp waits once more (the copy writes into this CTA's
        // shared memory) and skips phase B; the CTA then stops before adding.
        const int64_t lim = wait_limit_ns(p.wait_ns);
        bool bad = !mbar_wait_ns(mbar, phase, lim);
        if (bad) {
            atomicCAS(lp.status, 0, 2);
            (void)mbar_wait_ns(mbar, phase, lim);
        }
        bad = __any_sync(0xffffffffu, bad);
        phase ^= 1u;
        for (int rnd = 0; rnd < P / LINES && !bad; ++rnd) {
            const int col = phase_b_col<LINES>(line, rnd);
            C a[R1];
            // rows in: n1 (forward) or L1 (adjoint); rows kept: the other.
            // Row t + R2 j of the column: (t + R2 j) * PITCH + col + pad_shift(t)
            const int rows_in = ADJ ? L1 : n1, rows_out = ADJ ? n1 : L1;
            C *Scol = S + t * PITCH + pad_shift(t) + col;
#pragma unroll
            for (int j = 0; j < R1; ++j) a[j] = t + R2 * j < rows_in ? Scol[j * R2 * PITCH] : zero;
            PadScratch<P, C, true> scr(S + col, t);
            fft_line<P, false>(a, tw, t, scr, lmask);
            // Hermitian half spectrum stored as [k2 <= P/2][k1]; the adjoint
            // multiplies by the conjugate.  Mirrored columns read index
            // P - k1 (index P holds value 0 again).
            if (col <= P / 2) {
                const C *sc = SP + col * L::SPLD + t;
#pragma unroll
                for (int j = 0; j < R1; ++j) a[j] = ADJ ? cmulc(a[j], sc[R2 * j]) : cmul(a[j], sc[R2 * j]);
            } else {
                const C *sc = SP + (P - col) * L::SPLD + (P - t);
#pragma unroll
                for (int j = 0; j < R1; ++j) {
                    const C v = sc[-R2 * j];
                    a[j] = ADJ ? cmul(a[j], v) : cmulc(a[j], v);
                }
            }
            fft_line<P, true>(a, tw, t, scr, lmask);
#pragma unroll
            for (int j = 0; j < R1; ++j)
                if (t + R2 * j < rows_out) Scol[j * R2 * PITCH] = a[j];
        }

        // ---------------- ordered overlap-add: wait for lower colours
        // one thread per dependency flag, all polled concurrently; the barrier
        // after the polls also ends phase B
        {
            const int d0 = p.dep_start[ti], nd = p.dep_start[ti + 1] - d0;
            for (int d = threadIdx.x; d < nd && !bad; d += blockDim.x) {
                const uint32_t *f = p.done + int64_t(p.dep[d0 + d]) * p.done_ld + pair;
                // timeout (or another wait of the launch gave up): result invalid
                bad = !wait_flag_eq<false>(f, p.epoch, lp.status, lim, 1, 64);
                __threadfence();
            }
        }
        // an abandoned item adds nothing and is not reported done; the CTA
        // stops (its earlier, finished item is still published at exit)
        if (__syncthreads_or(bad)) break;

        // ---------------- phase C: inverse row FFTs and overlap-add (fire-and-forget
        // reductions: no two tiles that overlap add at the same time, so each pixel
        // still sums in colour order)
        T *y0 = y + int64_t(b0) * p.ldy;
        T *y1 = has1 ? y0 + p.ldy : y0;
        if (sizeof(T) == 4 && t == 0) fence_proxy_async_global();
        if constexpr (!ADJ) {
            for (int n = line; n < L1; n += LINES) {
                const int oy = o0 + n;
                if (oy < 0 || oy >= p.n[0]) continue;
                C a[R1];
                C *Srow = S + n * PITCH + pad_shift(n);
#pragma unroll
                for (int j = 0; j < R1; ++j) a[j] = Srow[t + R2 * j];
                PadScratch<P, C, false> scr(Srow, t);
                fft_line<P, true>(a, tw, t, scr, lmask);
                add_row<T, P>(a, t, lmask, reinterpret_cast<float *>(SP) + line * L::STAGE,
                              y0 + int64_t(oy) * p.n[1], y1 + int64_t(oy) * p.n[1], has1, o1, L2, p.n[1]);
            }
        } else {
            // adjoint: the n1 x n2 input box, weighted by w_k, added at (i0, j0);
            // in store mode (incremental estimator) stored unweighted to the tile's block
            for (int n = line; n < n1; n += LINES) {
                const T *wr = wt + int64_t(n) * tile.w_ld[0];
                T wv[R1];
#pragma unroll
                for (int j = 0; j < R1; ++j) wv[j] = t + R2 * j < n2 ? __ldg(wr + t + R2 * j) : T(0);
                C a[R1];
                C *Srow = S + n * PITCH + pad_shift(n);
#pragma unroll
                for (int j = 0; j < R1; ++j) a[j] = Srow[t + R2 * j];
                PadScratch<P, C, false> scr(Srow, t);
                fft_line<P, true>(a, tw, t, scr, lmask);
                if (p.store) {
                    const StoreDesc sd = p.store[ti];
                    T *st0 = static_cast<T *>(p.store_base) + sd.off + int64_t(b0) * sd.ld_rhs + int64_t(n) * sd.ld_row;
#pragma unroll
                    for (int j = 0; j < R1; ++j) {
                        const int col = t + R2 * j;
                        if (col < n2) {
                            st0[col] = a[j].x;
                            if (has1) st0[sd.ld_rhs + col] = a[j].y;
                        }
                    }
                    continue;
                }
#pragma unroll
                for (int j = 0; j < R1; ++j) a[j] = C{a[j].x * wv[j], a[j].y * wv[j]};
                const int oy = i0 + n;
                add_row<T, P>(a, t, lmask, reinterpret_cast<float *>(SP) + line * L::STAGE,
                              y0 + int64_t(oy) * p.n[1], y1 + int64_t(oy) * p.n[1], has1, j0, n2, p.n[1]);
            }
        }
        if constexpr (sizeof(T) == 4) {
            // the staging rows are read: the next spectrum may overwrite them.
            // Completion of the reductions is awaited after the next item's
            // phase A (or at exit), and only then is this item reported done.
            if (t == 0) bulk_wait_read();
        }
        pend_flag_any = true;
        if (threadIdx.x == 0) {
            if (ld_volatile_s32(lp.status) != 0) s_stop = 1;
            pend_flag = p.done + int64_t(ti) * p.done_ld + pair;
            pend_epoch = p.epoch;
            pend_seg_done = lp.seg_done ? lp.seg_done + cur_seg : nullptr;
            pend_total = p.total_items;
            pend_slot = s_seg.slot;
        }
        __syncthreads();
    }
    if constexpr (sizeof(T) == 4) {
        if (t == 0 && pend_flag_any) {
            bulk_wait_all();
            fence_proxy_async_global();
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) publish_pending();
}

template <typename T>
__global__ void zero_kernel(T *y, int64_t ldy, int32_t nrhs, int64_t N, unsigned long long *counter) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0ull;
    const int64_t total = int64_t(nrhs) * N;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t b = i / N, e = i - b * N;
        y[b * ldy + e] = T(0);
    }
}

cudaError_t launch_zero(const ApplyParams &p, int64_t N, pc_precision prec, cudaStream_t s) {
    const int64_t total = int64_t(p.nrhs) * N;
    int blocks = int(std::min<int64_t>((total + 255) / 256, 4096));
    if (blocks < 1) blocks = 1;
    auto *ctr = reinterpret_cast<unsigned long long *>(p.ctrl);
    if (prec == PC_FP64)
        zero_kernel<double><<<blocks, 256, 0, s>>>(static_cast<double *>(p.y), p.ldy, p.nrhs, N, ctr);
    else
        zero_kernel<float><<<blocks, 256, 0, s>>>(static_cast<float *>(p.y), p.ldy, p.nrhs, N, ctr);
    return cudaGetLastError();
}

template <typename T, int P>
static cudaError_t configure_one(int *ctas_per_sm, size_t *smem) {
    const size_t bytes = Smem2d<T, P>::bytes;
    cudaError_t e = cudaSuccess;
    const void *fns[4] = {reinterpret_cast<const void *>(fft2d_kernel<T, P, false, false>),
                          reinterpret_cast<const void *>(fft2d_kernel<T, P, true, false>),
                          reinterpret_cast<const void *>(fft2d_kernel<T, P, false, true>),
                          reinterpret_cast<const void *>(fft2d_kernel<T, P, true, true>)};
    for (const void *f : fns)
        if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    if (e != cudaSuccess) return e;
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fft2d_kernel<T, P, false, false>, KCfg<T, P>::threads,
                                                      bytes);
    if (e != cudaSuccess) return e;
    if (ctas_per_sm) *ctas_per_sm = n;
    if (smem) *smem = bytes;
    return cudaSuccess;
}

cudaError_t fft2d_configure(int P, pc_precision prec, int *ctas_per_sm, size_t *smem) {
    if (prec == PC_FP64) {
        if (P == 64) return configure_one<double, 64>(ctas_per_sm, smem);
        return cudaErrorInvalidValue;
    }
    if (P == 64) return configure_one<float, 64>(ctas_per_sm, smem);
    if (P == 128) return configure_one<float, 128>(ctas_per_sm, smem);
    return cudaErrorInvalidValue;
}

template <bool ADJ, bool MULTI>
static void launch_one(const LaunchParams &lp, int P, pc_precision prec, int ctas, size_t smem, cudaStream_t s) {
    if (prec == PC_FP64)
        fft2d_kernel<double, 64, ADJ, MULTI><<<ctas, KCfg<double, 64>::threads, smem, s>>>(lp);
    else if (P == 64)
        fft2d_kernel<float, 64, ADJ, MULTI><<<ctas, KCfg<float, 64>::threads, smem, s>>>(lp);
    else
        fft2d_kernel<float, 128, ADJ, MULTI><<<ctas, KCfg<float, 128>::threads, smem, s>>>(lp);
}

cudaError_t launch_fft2d(const ApplyParams &p, int P, pc_precision prec, int ctas, cudaStream_t s, bool adjoint) {
    size_t smem = 0;
    cudaError_t e = fft2d_configure(P, prec, nullptr, &smem);
    if (e != cudaSuccess) return e;
    LaunchParams lp{};
    lp.desc = nullptr;
    lp.one.p = p;
    lp.one.item_begin = 0;
    lp.one.slot = -1;
    lp.counter = reinterpret_cast<unsigned long long *>(p.ctrl);
    lp.status = p.ctrl + 2;
    if (adjoint)
        launch_one<true, false>(lp, P, prec, ctas, smem, s);
    else
        launch_one<false, false>(lp, P, prec, ctas, smem, s);
    return cudaGetLastError();
}

// Multi-segment launch: every segment's y zeroed, its ordering flags and
// finished-item counter cleared, the claim counter reset.
template <typename T>
__global__ void round_prepare(const LaunchDesc *d, unsigned long long *counter, uint32_t *seg_done) {
    const int nseg = d->nseg;
    if (blockIdx.x == 0 && threadIdx.x == 0) *counter = 0ull;
    if (blockIdx.x == 0)
        for (int q = threadIdx.x; q < nseg; q += blockDim.x) seg_done[q] = 0u;
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    for (int sx = 0; sx < nseg; ++sx) {
        const ApplyParams &p = d->seg[sx].p;
        const int64_t N = int64_t(p.n[0]) * p.n[1] * p.n[2];
        T *y = static_cast<T *>(p.y);
        const int64_t tot = int64_t(p.nrhs) * N;
        for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < tot; q += stride) {
            const int64_t b = q / N, e = q - b * N;
            y[b * p.ldy + e] = T(0);
        }
        const int64_t nf = int64_t(p.color_start[p.n_colors]) * p.done_ld;
        for (int64_t q = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; q < nf; q += stride) p.done[q] = 0u;
    }
}

cudaError_t launch_round(const LaunchDesc *d_desc, unsigned long long *counter, int32_t *status, uint32_t *seg_done,
                         uint32_t *host_flags, int ctas, size_t smem, cudaStream_t s, int P, pc_precision prec,
                         bool adjoint) {
    if (prec == PC_FP64)
        round_prepare<double><<<1024, 256, 0, s>>>(d_desc, counter, seg_done);
    else
        round_prepare<float><<<1024, 256, 0, s>>>(d_desc, counter, seg_done);
    LaunchParams lp{};
    lp.desc = d_desc;
    lp.one.slot = -1;
    lp.counter = counter;
    lp.status = status;
    lp.seg_done = seg_done;
    lp.host_flags = host_flags;
    if (adjoint)
        launch_one<true, true>(lp, P, prec, ctas, smem, s);
    else
        launch_one<false, true>(lp, P, prec, ctas, smem, s);
    return cudaGetLastError();
}

}  // namespace pc
