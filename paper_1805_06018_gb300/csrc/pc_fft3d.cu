// 3D patch path for y = sum_k phi_k^E * (w_k . x)  (Eq. conv_op_approx_main), P = 64.
//
// A 64^3 complex field (2 MB) does not fit in one CTA's shared memory, so a
// work item (tile, pair of right-hand sides) runs in three phases around a
// scratch volume G in global memory, laid out [plane][k2][k1]:
//
//   phase 1  for each of the n0 non-zero input planes: gather w . x, 2D FFT
//            (rows, then columns) in a 64 x 64 shared workspace, store the
//            plane's 2D spectrum to G
//   phase 2  for each (k1, k2) line: FFT along the first axis over the n0
//            non-zero planes, product with the stored spectrum phi^_k,
//            inverse FFT, keeping the L0 = n0 + K0 - 1 needed output planes
//            (in place in G: a line only touches its own column of G)
//   phase 3  for each needed output plane: inverse 2D FFT (columns, then
//            rows) and the overlap-add of its L1 x L2 box into y
//
// In the fused kernel a cluster of CTAs works on one item at a time through
// one scratch volume: each CTA takes every n-th plane or line of phases 1
// and 2 and one contiguous group of the output planes in phase 3, and
// cluster barriers separate the phases.  Shorter items (in time) shorten the
// chain of ordering waits through the colours, which bounds the forward
// apply; the adjoint, whose chain is shorter, runs clusters of one CTA.
//
// Overlap-add order, termination and determinism are those of the 2D kernel:
// colour-ordered tiles, claims in increasing order, bounded waits.  The same
// phases also run as separate kernels over chunks of items (phase 1, then the
// tensor-core first-axis transform of pc_tc3d.cu, then phase 3).  Scratch
// traffic is about 6.7 MB per item; the line FFTs (about 20,000 of length 64
// per item) dominate the time.
#include <algorithm>

#include "pc_fftcore.cuh"
#include "pc_internal.h"
#include "pc_cluster.cuh"
#include "pc_ptx.cuh"

namespace pc {

constexpr int kThreads3d = 256;
constexpr int kP3 = 64;
constexpr int kSmem3 = kP3 * kP3 * int(sizeof(float2));

// One work item: tile `ti` of the schedule and right-hand-side pair `pair`
// (columns 2 pair and 2 pair + 1 packed as the real and imaginary parts).
struct Item3 {
    int ti, pair;
    Tile tile;
};

// `c`: a colour <= the item's to start the search from (a CTA's claims only
// increase, so its previous item's colour); updated to the item's colour
__device__ __forceinline__ Item3 decode_item3(const ApplyParams &p, int64_t item, int &c) {
    while (int64_t(p.color_start[c + 1]) * p.npairs <= item) ++c;
    const int64_t base = int64_t(p.color_start[c]) * p.npairs;
    const int ntc = p.color_start[c + 1] - p.color_start[c];
    Item3 it;
    it.pair = int((item - base) / ntc);
    it.ti = p.color_start[c] + int((item - base) % ntc);
    it.tile = p.tiles[it.ti];
    return it;
}

// Per-thread constants of the line FFTs (R2 = 8 threads per line of 64).
struct Lines3 {
    static constexpr int P = kP3;
    static constexpr int R1 = FftShape<P>::R1, R2 = FftShape<P>::R2;
    static constexpr int LINES = kThreads3d / R2;
    static constexpr int PP = P * P;
    int t, line;
    unsigned lmask;
    float2 tw[R1];
    __device__ __forceinline__ explicit Lines3(const float2 *twg) {
        t = threadIdx.x % R2;
        line = threadIdx.x / R2;
        lmask = FftShape<P>::line_mask();
#pragma unroll
        for (int m = 0; m < R1; ++m) tw[m] = twg[(t * m) & (P - 1)];
    }
};

// phase 1: 2D FFT of each of the n0 non-zero input planes -> G[i0][k2][k1].
// Adjoint: of the L0 planes of the output box, x unweighted and zero outside
// Omega (rows and columns L1 x L2 at out_lo); planes outside Omega are
// skipped here and read as zero by phase 2.
// The planes i0 = first, first + step, ... of the phase: a CTA's share.
template <bool ADJ>
__device__ __forceinline__ void phase1_3d(const ApplyParams &p, const Item3 &it, float2 *G, float2 *S,
                                          const Lines3 &L, int first, int step) {
    using C = float2;
    constexpr int P = Lines3::P, R1 = Lines3::R1, R2 = Lines3::R2, LINES = Lines3::LINES, PP = Lines3::PP;
    const C zero{0.0f, 0.0f};
    const Tile &tile = it.tile;
    const int n0 = tile.in_ext[0], n1 = tile.in_ext[1], n2 = tile.in_ext[2];
    // planes, rows and columns of the gathered box
    const int m0 = ADJ ? n0 + tile.kext[0] - 1 : n0;
    const int m1 = ADJ ? n1 + tile.kext[1] - 1 : n1;
    const int m2 = ADJ ? n2 + tile.kext[2] - 1 : n2;
    const int g0 = ADJ ? tile.out_lo[0] : tile.in_lo[0];
    const int g1 = ADJ ? tile.out_lo[1] : tile.in_lo[1];
    const int g2 = ADJ ? tile.out_lo[2] : tile.in_lo[2];
    const int b0 = 2 * it.pair;
    const bool has1 = b0 + 1 < p.nrhs;
    const float *x0 = static_cast<const float *>(p.x) + int64_t(b0) * p.ldx;
    const float *x1 = has1 ? x0 + p.ldx : x0;
    const float *wt = static_cast<const float *>(p.w) + tile.w_base;
    const int64_t plane_box = int64_t(p.nx[1]) * p.nx[2];   // x lives on the box nx
    for (int i0 = first; i0 < m0; i0 += step) {
        if (ADJ && (g0 + i0 < 0 || g0 + i0 >= p.nx[0])) continue;   // uniform across the CTA
        const float *wp = wt + int64_t(i0) * tile.w_ld[0];
        const int64_t xp = int64_t(g0 + i0) * plane_box;
        for (int r = L.line; r < m1; r += LINES) {
            C a[R1];
            const int gr = g1 + r;
            const bool rin = !ADJ || (gr >= 0 && gr < p.nx[1]);
            const int64_t xr = xp + int64_t(gr) * p.nx[2] + g2;
            const float *wr = wp + int64_t(r) * tile.w_ld[1];
#pragma unroll
            for (int j = 0; j < R1; ++j) {
                const int col = L.t + R2 * j;
                if constexpr (ADJ) {
                    const int gc = g2 + col;
                    a[j] = rin && col < m2 && gc >= 0 && gc < p.nx[2]
                               ? C{__ldg(x0 + xr + col), has1 ? __ldg(x1 + xr + col) : 0.0f}
                               : zero;
                } else if (col < n2) {
                    const float wv = __ldg(wr + col);
                    a[j] = C{wv * __ldg(x0 + xr + col), has1 ? wv * __ldg(x1 + xr + col) : 0.0f};
                } else {
                    a[j] = zero;
                }
            }
            RowScratch<P, C> scr{S, r};
            fft_line<P, false>(a, L.tw, L.t, scr, L.lmask);
#pragma unroll
            for (int j = 0; j < R1; ++j) S[r * P + ((L.t + R2 * j) ^ swz(r))] = a[j];
        }
        __syncthreads();
        for (int k2 = L.line; k2 < P; k2 += LINES) {
            C a[R1];
#pragma unroll
            for (int j = 0; j < R1; ++j) {
                const int row = L.t + R2 * j;
                a[j] = row < m1 ? S[row * P + (k2 ^ swz(row))] : zero;
            }
            ColScratch<P, C> scr{S, k2};
            fft_line<P, false>(a, L.tw, L.t, scr, L.lmask);
            C *g = G + int64_t(i0) * PP + k2 * P;
#pragma unroll
            for (int j = 0; j < R1; ++j) __stcg(g + L.t + R2 * j, a[j]);
        }
        __syncthreads();
    }
}

// phase 2 (FP32 line FFTs): per (k1, k2) line, FFT along the first axis over
// the n0 non-zero planes, product with the stored spectrum, inverse FFT,
// keeping the L0 needed output planes.  Stored spectrum: Hermitian half in
// k2, layout [k2 <= P/2][k1][k0].
// Adjoint: the L0 output-box planes in (those outside Omega read as zero),
// the conjugate spectrum, the n0 input-box planes kept.  The CTA takes the
// lines of the line groups first, first + step, ... (LINES lines a group).
template <bool ADJ>
__device__ __forceinline__ void phase2_3d(const ApplyParams &p, const Item3 &it, float2 *G, float2 *S,
                                          const Lines3 &L, int first, int step) {
    using C = float2;
    constexpr int P = Lines3::P, R1 = Lines3::R1, R2 = Lines3::R2, LINES = Lines3::LINES, PP = Lines3::PP;
    const C zero{0.0f, 0.0f};
    const int n0 = it.tile.in_ext[0], L0 = n0 + it.tile.kext[0] - 1;
    const int rows_in = ADJ ? L0 : n0, rows_out = ADJ ? n0 : L0;
    const int g0 = it.tile.out_lo[0];
    const C *sp = static_cast<const C *>(p.spec) + int64_t(it.tile.spec) * p.spec_stride;
    for (int l = first * LINES + L.line; l < PP; l += step * LINES) {
        const int k2 = l / P, k1 = l % P;
        C a[R1];
        C *g = G + k2 * P + k1;
#pragma unroll
        for (int j = 0; j < R1; ++j) {
            const int i0 = L.t + R2 * j;
            const bool in = i0 < rows_in && (!ADJ || (g0 + i0 >= 0 && g0 + i0 < p.nx[0]));
            a[j] = in ? __ldcg(g + int64_t(i0) * PP) : zero;
        }
        // S is idle in this phase: row `line` is the line's transpose scratch
        RowScratch<P, C> scr{S, L.line};
        fft_line<P, false>(a, L.tw, L.t, scr, L.lmask);
        // the adjoint multiplies by the conjugate spectrum
        if (k2 <= P / 2) {
            const C *sc = sp + (int64_t(k2) * P + k1) * P;
#pragma unroll
            for (int j = 0; j < R1; ++j) {
                const C v = __ldg(sc + L.t + R2 * j);
                a[j] = ADJ ? cmulc(a[j], v) : cmul(a[j], v);
            }
        } else {
            const C *sc = sp + (int64_t(P - k2) * P + ((P - k1) & (P - 1))) * P;
#pragma unroll
            for (int j = 0; j < R1; ++j) {
                const C v = __ldg(sc + ((P - (L.t + R2 * j)) & (P - 1)));
                a[j] = ADJ ? cmul(a[j], v) : cmulc(a[j], v);
            }
        }
        fft_line<P, true>(a, L.tw, L.t, scr, L.lmask);
#pragma unroll
        for (int j = 0; j < R1; ++j) {
            const int o0 = L.t + R2 * j;
            if (o0 < rows_out) __stcg(g + int64_t(o0) * PP, a[j]);
        }
    }
    __syncthreads();
}

// First-axis range [b, e) (in y) of output-plane group g of ng of a tile:
// the planes kept by phase 3 (the L0 of the output box, or the n0 of the
// input box for the adjoint) split into ng contiguous groups.
template <bool ADJ>
__device__ __forceinline__ void group_span(const Tile &t, int g, int ng, int &b, int &e) {
    const int base = ADJ ? t.in_lo[0] : t.out_lo[0];
    const int m0 = ADJ ? t.in_ext[0] : t.in_ext[0] + t.kext[0] - 1;
    b = base + (m0 * g) / ng;
    e = base + (m0 * (g + 1)) / ng;
}

// ordered overlap-add: wait (bounded) until every overlapping tile of a lower
// colour has published, for this pair, each of its `ng` output-plane groups
// whose planes meet [zb, ze), the planes this CTA is about to add.  A tile's
// flags for the pair are `ng` consecutive words (one per group) starting at
// done[tile * done_ld + pair * ng].  Waiting per group, not per tile, lets a
// tile's groups follow the lower colours' groups plane range by plane range.
// Returns false (for the whole CTA) if a wait gave up - a timeout, or
// another wait of the launch gave up first (the status word p.ctrl[2] is
// then non-zero): the item must be abandoned.
template <bool ADJ>
__device__ __forceinline__ bool wait_deps_3d(const ApplyParams &p, const Item3 &it, int ng, int zb, int ze) {
    const int d0 = p.dep_start[it.ti], nd = p.dep_start[it.ti + 1] - d0;
    const int64_t lim = wait_limit_ns(p.wait_ns);
    bool bad = false;
    for (int d = threadIdx.x; d < nd * ng && !bad && zb < ze; d += blockDim.x) {
        const int dt = p.dep[d0 + d / ng], g = d % ng;
        int gb, ge;
        group_span<ADJ>(p.tiles[dt], g, ng, gb, ge);
        if (gb >= ge || ge <= zb || gb >= ze) continue;   // no plane in common
        const uint32_t *f = p.done + int64_t(dt) * p.done_ld + int64_t(it.pair) * ng + g;
        bad = !wait_flag_eq<false>(f, p.epoch, p.ctrl + 2, lim, 1, 64);
        __threadfence();
    }
    return !__syncthreads_or(bad);
}

// phase 3: inverse 2D FFT of the output planes o0 = ob, ob + step, ... < oe
// (of the L0 needed) and the overlap-add of their L1 x L2 boxes into y; then
// publish `flag` (if not null).  Adjoint: the planes are the n0 of the input
// box, each n1 x n2, weighted by w_k and added at the tile's origin.
template <bool ADJ>
__device__ __forceinline__ void phase3_3d(const ApplyParams &p, const Item3 &it, const float2 *G, float2 *S,
                                          const Lines3 &L, int ob, int oe, int step, uint32_t *flag) {
    using C = float2;
    constexpr int P = Lines3::P, R1 = Lines3::R1, R2 = Lines3::R2, LINES = Lines3::LINES, PP = Lines3::PP;
    const Tile &tile = it.tile;
    const int n0 = tile.in_ext[0], n1 = tile.in_ext[1], n2 = tile.in_ext[2];
    // kept box (rows, columns) and its origin in y
    const int m1 = ADJ ? n1 : n1 + tile.kext[1] - 1, m2 = ADJ ? n2 : n2 + tile.kext[2] - 1;
    const int h0 = ADJ ? tile.in_lo[0] : tile.out_lo[0];
    const int h1 = ADJ ? tile.in_lo[1] : tile.out_lo[1];
    const int h2 = ADJ ? tile.in_lo[2] : tile.out_lo[2];
    const int b0 = 2 * it.pair;
    const bool has1 = b0 + 1 < p.nrhs;
    float *y0 = static_cast<float *>(p.y) + int64_t(b0) * p.ldy;
    float *y1 = has1 ? y0 + p.ldy : y0;
    const float *wt = static_cast<const float *>(p.w) + tile.w_base;
    const int n2box = p.n[2];
    const int64_t plane_box = int64_t(p.n[1]) * n2box;
    (void)n0;
    for (int o0 = ob; o0 < oe; o0 += step) {
        const int gy0 = h0 + o0;
        if (gy0 < 0 || gy0 >= p.n[0]) continue;   // uniform across the CTA
        // inverse along k1 for each k2: rows o1 of S
        const C *gp = G + int64_t(o0) * PP;
        for (int k2 = L.line; k2 < P; k2 += LINES) {
            C a[R1];
#pragma unroll
            for (int j = 0; j < R1; ++j) a[j] = __ldcg(gp + k2 * P + L.t + R2 * j);
            ColScratch<P, C> scr{S, k2};
            fft_line<P, true>(a, L.tw, L.t, scr, L.lmask);
#pragma unroll
            for (int j = 0; j < R1; ++j) {
                const int o1 = L.t + R2 * j;
                if (o1 < m1) S[o1 * P + (k2 ^ swz(o1))] = a[j];
            }
        }
        __syncthreads();
        for (int o1 = L.line; o1 < m1; o1 += LINES) {
            const int gy1 = h1 + o1;
            if (gy1 < 0 || gy1 >= p.n[1]) continue;
            C a[R1];
#pragma unroll
            for (int j = 0; j < R1; ++j) a[j] = S[o1 * P + ((L.t + R2 * j) ^ swz(o1))];
            RowScratch<P, C> scr{S, o1};
            fft_line<P, true>(a, L.tw, L.t, scr, L.lmask);
            if constexpr (ADJ) {
                const float *wr = wt + int64_t(o0) * tile.w_ld[0] + int64_t(o1) * tile.w_ld[1];
#pragma unroll
                for (int j = 0; j < R1; ++j) {
                    const int o2 = L.t + R2 * j;
                    const float wv = o2 < n2 ? __ldg(wr + o2) : 0.0f;
                    a[j] = C{a[j].x * wv, a[j].y * wv};
                }
            }
            const int64_t yr = int64_t(gy0) * plane_box + int64_t(gy1) * n2box;
            // a warp's atomics land in 32-byte sectors of four output rows;
            // staging the row for vector or bulk reductions measured slower
#pragma unroll
            for (int j = 0; j < R1; ++j) {
                const int o2 = L.t + R2 * j;
                const int gy2 = h2 + o2;
                if (o2 < m2 && gy2 >= 0 && gy2 < n2box) {
                    atomicAdd(y0 + yr + gy2, a[j].x);
                    if (has1) atomicAdd(y1 + yr + gy2, a[j].y);
                }
            }
        }
        __syncthreads();
    }
    if (flag && threadIdx.x == 0) {
        __threadfence();
        st_release_u32(flag, p.epoch);
    }
}

// The fused FP32 kernel: persistent clusters of NR CTAs claim items in
// increasing order and run the three phases through the cluster's scratch
// volume, each CTA on its share of every phase.  In phase 3 CTA r adds the
// r-th contiguous group of the item's output planes and publishes that
// group's ordering flag.  NR = 1 is the one-CTA form (no cluster barriers).
template <bool ADJ, int NR>
__global__ void __launch_bounds__(kThreads3d, 3) fft3d_kernel(const ApplyParams p, float2 *scratch) {
    extern __shared__ __align__(16) unsigned char smem3[];
    float2 *S = reinterpret_cast<float2 *>(smem3);
    __shared__ int64_t s_claim;   // rank 0: the cluster's next item
    __shared__ int64_t s_item;
    const int rank = NR > 1 ? int(cluster_ctarank()) : 0;
    const Lines3 L(static_cast<const float2 *>(p.tw));
    float2 *G = scratch + int64_t(blockIdx.x / NR) * kP3 * kP3 * kP3;
    auto sync = [] {
        if constexpr (NR > 1) cluster_sync();
        else __syncthreads();
    };
    int chint = 0;
    for (;;) {
        // a launch whose waits have given up (status word set) takes no more items
        if (rank == 0 && threadIdx.x == 0)
            s_claim = ld_volatile_s32(p.ctrl + 2) != 0
                          ? p.total_items
                          : int64_t(atomicAdd(reinterpret_cast<unsigned long long *>(p.ctrl), 1ull));
        // every CTA is done with the previous item's scratch volume, and the
        // claim is visible
        sync();
        if (threadIdx.x == 0) s_item = NR > 1 ? ld_cluster_s64(&s_claim, 0) : s_claim;
        __syncthreads();
        const int64_t item = s_item;
        if (item >= p.total_items) break;
        const Item3 it = decode_item3(p, item, chint);
        phase1_3d<ADJ>(p, it, G, S, L, rank, NR);
        sync();
        phase2_3d<ADJ>(p, it, G, S, L, rank, NR);
        sync();
        // this CTA's planes; a failed wait abandons them (the status word is
        // then set, so the next claim ends the launch) and the CTA still
        // takes part in the cluster barriers
        int zb, ze;
        group_span<ADJ>(it.tile, rank, NR, zb, ze);
        const int base = ADJ ? it.tile.in_lo[0] : it.tile.out_lo[0];
        if (wait_deps_3d<ADJ>(p, it, NR, zb, ze))
            phase3_3d<ADJ>(p, it, G, S, L, zb - base, ze - base, 1,
                           p.done + int64_t(it.ti) * p.done_ld + int64_t(it.pair) * NR + rank);
    }
    // no CTA leaves while another may still read its shared memory
    if constexpr (NR > 1) cluster_sync();
}

// Split form used with the tensor-core first-axis transform: items
// [c0, c1) of one chunk, each with its own scratch volume G[item - c0].
// Phase 1 needs no ordering.
template <bool ADJ>
__global__ void __launch_bounds__(kThreads3d, 3) fft3d_phase1_kernel(const ApplyParams p, float2 *scratch,
                                                                     int64_t c0, int64_t c1) {
    __shared__ __align__(16) float2 S[kP3 * kP3];
    const Lines3 L(static_cast<const float2 *>(p.tw));
    int chint = 0;
    if constexpr (ADJ) {
        // the adjoint gathers the L0 output-box planes (up to P): tasks of one
        // item's planes g, g + 16, ... balance better than whole items
        constexpr int kTasks = 16;
        for (int64_t task = c0 * kTasks + blockIdx.x; task < c1 * kTasks; task += gridDim.x) {
            const int64_t item = task / kTasks;
            const int g = int(task % kTasks);
            const Item3 it = decode_item3(p, item, chint);
            if (g >= it.tile.in_ext[0] + it.tile.kext[0] - 1) continue;   // uniform across the CTA
            phase1_3d<ADJ>(p, it, scratch + (item - c0) * kP3 * kP3 * kP3, S, L, g, kTasks);
        }
    } else {
        for (int64_t item = c0 + blockIdx.x; item < c1; item += gridDim.x) {
            const Item3 it = decode_item3(p, item, chint);
            phase1_3d<ADJ>(p, it, scratch + (item - c0) * kP3 * kP3 * kP3, S, L, 0, 1);
        }
    }
}

// Phase 3 of the split form works on (item, output-plane group) pieces,
// kPhase3Groups per item, claimed in increasing order (claim counter reset to
// 0 before the launch).  A piece waits for every group of each overlapping
// lower-colour tile, so each voxel still sums its contributions in colour
// order (the groups of one tile write disjoint planes); the pieces shorten
// the chain of waits through the colours by the group count.
template <bool ADJ>
__global__ void __launch_bounds__(kThreads3d, 3) fft3d_phase3_kernel(const ApplyParams p, const float2 *scratch,
                                                                     int64_t c0, int64_t c1) {
    extern __shared__ __align__(16) unsigned char smem3[];
    float2 *S = reinterpret_cast<float2 *>(smem3);
    __shared__ int64_t s_piece;
    constexpr int NG = kPhase3Groups;
    const Lines3 L(static_cast<const float2 *>(p.tw));
    int chint = 0;
    for (;;) {
        if (threadIdx.x == 0)
            s_piece = ld_volatile_s32(p.ctrl + 2) != 0
                          ? c1 * NG
                          : c0 * NG + int64_t(atomicAdd(reinterpret_cast<unsigned long long *>(p.ctrl), 1ull));
        __syncthreads();
        const int64_t piece = s_piece;
        if (piece >= c1 * NG) break;
        const int64_t item = piece / NG;
        const int g = int(piece % NG);
        const Item3 it = decode_item3(p, item, chint);
        int zb, ze;
        group_span<ADJ>(it.tile, g, NG, zb, ze);
        if (!wait_deps_3d<ADJ>(p, it, NG, zb, ze)) break;
        const int base = ADJ ? it.tile.in_lo[0] : it.tile.out_lo[0];
        phase3_3d<ADJ>(p, it, scratch + (item - c0) * kP3 * kP3 * kP3, S, L, zb - base, ze - base, 1,
                       p.done + int64_t(it.ti) * p.done_ld + int64_t(it.pair) * NG + g);
    }
}

// Clusters of the fused kernel (forward, adjoint) that fit on the device at
// once, per device (set by fft3d_configure).
static int g_fft3d_clusters[64][2];

static cudaLaunchConfig_t fft3d_config(cudaLaunchAttribute *attr, int cluster, int64_t clusters, cudaStream_t s) {
    attr->id = cudaLaunchAttributeClusterDimension;
    attr->val.clusterDim.x = unsigned(cluster);
    attr->val.clusterDim.y = 1;
    attr->val.clusterDim.z = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(unsigned(clusters * cluster));
    cfg.blockDim = dim3(kThreads3d);
    cfg.dynamicSmemBytes = kSmem3;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

cudaError_t fft3d_configure(int *ctas_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(fft3d_kernel<false, kCluster3dFwd>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem3);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fft3d_kernel<true, kCluster3dAdj>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem3);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fft3d_phase3_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem3);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fft3d_phase3_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem3);
    static_assert(kCluster3dMax <= 8, "portable cluster sizes only");
    int n = 0, na = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fft3d_kernel<false, kCluster3dFwd>, kThreads3d, kSmem3);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&na, fft3d_kernel<true, kCluster3dAdj>, kThreads3d, kSmem3);
    // one CTA count serves both directions (the scratch volumes are sized by it)
    if (ctas_per_sm) *ctas_per_sm = std::min(n, na);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess && dev >= 0 && dev < 64) {
        const int per_sm = std::max(1, std::min(n, na));
        cudaLaunchAttribute af{}, aa{};
        cudaLaunchConfig_t cf = fft3d_config(&af, kCluster3dFwd, int64_t(sms) * per_sm, nullptr);
        cudaLaunchConfig_t ca = fft3d_config(&aa, kCluster3dAdj, int64_t(sms) * per_sm, nullptr);
        int c0 = 0, c1 = 0;
        e = cudaOccupancyMaxActiveClusters(&c0, fft3d_kernel<false, kCluster3dFwd>, &cf);
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveClusters(&c1, fft3d_kernel<true, kCluster3dAdj>, &ca);
        g_fft3d_clusters[dev][0] = c0;
        g_fft3d_clusters[dev][1] = c1;
        if (e == cudaSuccess && (c0 < 1 || c1 < 1) && ctas_per_sm) *ctas_per_sm = 0;
    }
    return e;
}

// `ctas`: the operator's CTA budget; the launch runs min(ctas / cluster,
// items, resident clusters) clusters, each on its own scratch volume.
cudaError_t launch_fft3d(const ApplyParams &p, int ctas, void *scratch, cudaStream_t s, bool adjoint) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const int cluster = adjoint ? kCluster3dAdj : kCluster3dFwd;
    int64_t clusters = std::min<int64_t>(ctas / cluster, p.total_items);
    if (dev >= 0 && dev < 64 && g_fft3d_clusters[dev][adjoint ? 1 : 0] > 0)
        clusters = std::min<int64_t>(clusters, g_fft3d_clusters[dev][adjoint ? 1 : 0]);
    if (clusters < 1) return cudaErrorInvalidConfiguration;
    cudaLaunchAttribute attr{};
    const cudaLaunchConfig_t cfg = fft3d_config(&attr, cluster, clusters, s);
    float2 *g = static_cast<float2 *>(scratch);
    return adjoint ? cudaLaunchKernelEx(&cfg, fft3d_kernel<true, kCluster3dAdj>, p, g) : cudaLaunchKernelEx(&cfg, fft3d_kernel<false, kCluster3dFwd>, p, g);
}

size_t fft3d_volume_bytes() { return size_t(kP3) * kP3 * kP3 * sizeof(float2); }
size_t fft3d_scratch_bytes(int ctas) { return size_t(std::max(1, ctas / kCluster3dMin)) * fft3d_volume_bytes(); }

cudaError_t launch_fft3d_phase1(const ApplyParams &p, int ctas, void *scratch, int64_t c0, int64_t c1,
                                cudaStream_t s, bool adjoint) {
    if (adjoint)
        fft3d_phase1_kernel<true><<<ctas, kThreads3d, 0, s>>>(p, static_cast<float2 *>(scratch), c0, c1);
    else
        fft3d_phase1_kernel<false><<<ctas, kThreads3d, 0, s>>>(p, static_cast<float2 *>(scratch), c0, c1);
    return cudaGetLastError();
}

cudaError_t launch_fft3d_phase3(const ApplyParams &p, int ctas, const void *scratch, int64_t c0, int64_t c1,
                                cudaStream_t s, bool adjoint) {
    // claim counter of this chunk
    cudaError_t e = cudaMemsetAsync(p.ctrl, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    if (adjoint)
        fft3d_phase3_kernel<true><<<ctas, kThreads3d, kSmem3, s>>>(p, static_cast<const float2 *>(scratch), c0, c1);
    else
        fft3d_phase3_kernel<false><<<ctas, kThreads3d, kSmem3, s>>>(p, static_cast<const float2 *>(scratch), c0, c1);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64 3D spectra: windows psi [nspec][W][W][W] at [0, W)^3, stored Hermitian
// half in k2 with layout [k2 <= P/2][k1][k0], scaled by 1/P^3.
__global__ void spectra3d_stage1(const double *psi, int r0, int nr, int W, int P, const double2 *tw, double2 *T1) {
    // T1[k][a0][a1][c2] = sum_a2 psi[k][a0][a1][a2] W^{a2 c2}
    const int H = P / 2 + 1;
    const int64_t total = int64_t(nr) * W * W * H;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int c2 = int(i % H);
        const int64_t rest = i / H;
        const int a1 = int(rest % W), a0 = int((rest / W) % W);
        const int k = int(rest / (int64_t(W) * W));
        const double *row = psi + ((int64_t(r0 + k) * W + a0) * W + a1) * W;
        double re = 0.0, im = 0.0;
        for (int a2 = 0; a2 < W; ++a2) {
            const double2 wv = tw[(int64_t(a2) * c2) % P];
            re += row[a2] * wv.x;
            im += row[a2] * wv.y;
        }
        T1[i] = make_double2(re, im);
    }
}

__global__ void spectra3d_stage2(const double2 *T1, int nr, int W, int P, const double2 *tw, double2 *T2) {
    // T2[k][a0][c1][c2] = sum_a1 T1[k][a0][a1][c2] W^{a1 c1}
    const int H = P / 2 + 1;
    const int64_t total = int64_t(nr) * W * P * H;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int c2 = int(i % H);
        const int c1 = int((i / H) % P);
        const int64_t rest = i / (int64_t(H) * P);
        const int a0 = int(rest % W);
        const int k = int(rest / W);
        double re = 0.0, im = 0.0;
        for (int a1 = 0; a1 < W; ++a1) {
            const double2 v = T1[((int64_t(k) * W + a0) * W + a1) * H + c2];
            const double2 wv = tw[(int64_t(a1) * c1) % P];
            re += v.x * wv.x - v.y * wv.y;
            im += v.x * wv.y + v.y * wv.x;
        }
        T2[i] = make_double2(re, im);
    }
}

__global__ void spectra3d_stage3(const double2 *T2, int r0, int nr, int W, int P, const double2 *tw, float2 *spec) {
    // spec[k][c2][c1][k0] = (1/P^3) sum_a0 T2[k][a0][c1][c2] W^{a0 k0}
    const int H = P / 2 + 1;
    const double scale = 1.0 / (double(P) * P * P);
    const int64_t total = int64_t(nr) * H * P * P;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int k0 = int(i % P);
        const int c1 = int((i / P) % P);
        const int c2 = int((i / (int64_t(P) * P)) % H);
        const int k = int(i / (int64_t(P) * P * H));
        double re = 0.0, im = 0.0;
        for (int a0 = 0; a0 < W; ++a0) {
            const double2 v = T2[((int64_t(k) * W + a0) * P + c1) * H + c2];
            const double2 wv = tw[(int64_t(a0) * k0) % P];
            re += v.x * wv.x - v.y * wv.y;
            im += v.x * wv.y + v.y * wv.x;
        }
        spec[((int64_t(r0 + k) * H + c2) * P + c1) * P + k0] = make_float2(float(re * scale), float(im * scale));
    }
}

cudaError_t build_spectra_3d(const double *d_psi, int nspec, int W, int P, void *d_spec, const double2 *d_tw64,
                             cudaStream_t s) {
    const int H = P / 2 + 1;
    const int chunk = 32;
    double2 *T1 = nullptr, *T2 = nullptr;
    cudaError_t e = cudaMalloc(&T1, sizeof(double2) * size_t(chunk) * W * W * H);
    if (e == cudaSuccess) e = cudaMalloc(&T2, sizeof(double2) * size_t(chunk) * W * P * H);
    for (int r0 = 0; r0 < nspec && e == cudaSuccess; r0 += chunk) {
        const int nr = std::min(chunk, nspec - r0);
        const int64_t n1 = int64_t(nr) * W * W * H, n2 = int64_t(nr) * W * P * H, n3 = int64_t(nr) * H * P * P;
        auto blocks = [](int64_t n) { return int(std::min<int64_t>((n + 255) / 256, 16384)); };
        spectra3d_stage1<<<blocks(n1), 256, 0, s>>>(d_psi, r0, nr, W, P, d_tw64, T1);
        spectra3d_stage2<<<blocks(n2), 256, 0, s>>>(T1, nr, W, P, d_tw64, T2);
        spectra3d_stage3<<<blocks(n3), 256, 0, s>>>(T2, r0, nr, W, P, d_tw64, static_cast<float2 *>(d_spec));
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(T1);
    cudaFree(T2);
    return e != cudaSuccess ? e : e2;
}

}  // namespace pc
