// 2D patch kernel with 256 x 256 FFTs (FP32), for the large patches of a
// per-patch operator (Section 3.2's FFT convolution of one input tile with
// one kernel sub-window, as in the fused kernel of pc_fft2d.cu).
//
// A 256^2 complex field (512 KB) does not fit in one SM's shared memory, so
// an item (tile, pair of right-hand sides) runs its three phases around a
// per-CTA scratch field G in global memory (L2-resident: 512 KB per CTA),
// laid out column-major, G[k2][row], so that a column is contiguous:
//
//   phase A  rows of the input, 32 at a time: gather (w_k . x), row FFT in a
//            shared-memory tile, then the tile's columns written to G
//   phase B  per column k2: FFT over the rows, product with the stored half
//            spectrum (conjugate for the adjoint), inverse FFT, back to G
//   phase C  output rows, 32 at a time: the tile read from G's columns,
//            inverse row FFT, overlap-add into y
//
// Items are claimed in colour-major order and each tile adds only after the
// overlapping tiles of lower colour (same pair) have added, exactly as in
// the fused kernel, so every output sums its contributions in a fixed order.
// A line FFT of 256 points runs on 16 threads holding 16 values each
// (radix-16 in registers, a transpose through the line's own tile row, then
// radix-16 again).  With 16 threads and 8-byte values, both transpose walks
// of a contiguous 256-slot row are free of bank conflicts.
#include "pc_fftcore.cuh"
#include "pc_internal.h"
#include "pc_overlap.cuh"
#include "pc_ptx.cuh"

namespace pc {

namespace {

constexpr int kBP = 256;                  // FFT extent
constexpr int kBThreads = 512;
constexpr int kBR = FftShape<kBP>::R2;    // 16 threads per line
constexpr int kBLines = kBThreads / kBR;  // 32 lines
constexpr int kBPitch = kBP + 1;          // tile row pitch (complex): columns walk 32 rows conflict-free
constexpr int kBStage = 2 * kBP + 24;     // per-line overlap-add staging (floats)
constexpr int kBImOff = kBP + 12;
constexpr size_t kBTileBytes = size_t(kBLines) * kBPitch * sizeof(float2);
constexpr size_t kBSmem = kBTileBytes + size_t(kBLines) * kBStage * sizeof(float);

// The line's scratch: one contiguous tile row of 256 slots.
struct LinScratch {
    float2 *b;
    __device__ __forceinline__ void st_m(int m, int t, float2 v) const { b[m * kBR + (t ^ m)] = v; }
    __device__ __forceinline__ float2 ld_e(int e, int t2, int t) const { return b[(t + kBR * e) * kBR + (t2 ^ t)]; }
};

__device__ __forceinline__ void decode_big(const ApplyParams &p, int64_t item, int &ti, int &pair, int &c) {
    while (int64_t(p.color_start[c + 1]) * p.npairs <= item) ++c;
    const int64_t base = int64_t(p.color_start[c]) * p.npairs;
    const int ntc = p.color_start[c + 1] - p.color_start[c];
    pair = int((item - base) / ntc);
    ti = p.color_start[c] + int((item - base) % ntc);
}

template <bool ADJ>
__global__ void __launch_bounds__(kBThreads, 1) fft2d_big_kernel(const ApplyParams p, float2 *scratch) {
    constexpr int P = kBP, R1 = FftShape<P>::R1, R2 = kBR, LINES = kBLines;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float2 *Sb = reinterpret_cast<float2 *>(smem_raw);                       // [LINES][kBPitch]
    float *stage = reinterpret_cast<float *>(smem_raw + kBTileBytes);        // [LINES][kBStage]
    __shared__ int64_t s_item;
    __shared__ int s_stop;
    const int t = threadIdx.x % R2, line = threadIdx.x / R2;
    const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
    const unsigned lmask = FftShape<P>::line_mask();
    const float2 *twg = static_cast<const float2 *>(p.tw);
    float2 tw[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) tw[m] = twg[(t * m) & (P - 1)];
    const float2 zero{0.0f, 0.0f};
    float2 *G = scratch + int64_t(blockIdx.x) * P * P;   // G[k2 * P + row]
    const float *x = static_cast<const float *>(p.x);
    float *y = static_cast<float *>(p.y);
    const float *w = static_cast<const float *>(p.w);
    const float2 *spec = static_cast<const float2 *>(p.spec);
    const int64_t lim = wait_limit_ns(p.wait_ns);
    int chint = 0;
    bool pend = false;   // this CTA's previous item: reductions issued, flag not yet published
    uint32_t *pend_flag = nullptr;
    if (threadIdx.x == 0) s_stop = 0;
    for (;;) {
        if (threadIdx.x == 0)
            s_item = ld_volatile_s32(p.ctrl + 2) != 0
                         ? p.total_items
                         : int64_t(atomicAdd(reinterpret_cast<unsigned long long *>(p.ctrl), 1ull));
        __syncthreads();
        const int64_t item = s_item;
        if (item >= p.total_items) break;
        int ti, pair;
        decode_big(p, item, ti, pair, chint);
        const Tile tile = p.tiles[ti];
        const int n1 = tile.in_ext[0], n2 = tile.in_ext[1];
        const int i0 = tile.in_lo[0], j0 = tile.in_lo[1];
        const int L1 = n1 + tile.kext[0] - 1, L2 = n2 + tile.kext[1] - 1;   // <= P
        const int o0 = tile.out_lo[0], o1 = tile.out_lo[1];
        const int b0 = 2 * pair;
        const bool has1 = b0 + 1 < p.nrhs;
        const float *x0 = x + int64_t(b0) * p.ldx;
        const float *x1 = has1 ? x0 + p.ldx : x0;
        const float *wt = w + tile.w_base;
        const int rows_in = ADJ ? L1 : n1, rows_out = ADJ ? n1 : L1;

        // ---------------- phase A: input rows (forward: w . x over the input
        // box; adjoint: x over the output box, zero outside the box x lives
        // on), row FFTs, columns to G
        for (int r0 = 0; r0 < rows_in; r0 += LINES) {
            const int i = r0 + line;
            float2 a[R1];
            if (i < rows_in) {
                if constexpr (!ADJ) {
                    const int64_t xr = int64_t(i0 + i) * p.nx[1] + j0;
                    const float *wr = wt + int64_t(i) * tile.w_ld[0];
#pragma unroll
                    for (int j = 0; j < R1; ++j) {
                        const int col = t + R2 * j;
                        if (col < n2) {
                            const float wv = __ldg(wr + col);
                            a[j] = float2{wv * __ldg(x0 + xr + col), has1 ? wv * __ldg(x1 + xr + col) : 0.0f};
                        } else {
                            a[j] = zero;
                        }
                    }
                } else {
                    const int gr = o0 + i;
                    const bool rin = gr >= 0 && gr < p.nx[0];
                    const int64_t xr = int64_t(gr) * p.nx[1] + o1;
#pragma unroll
                    for (int j = 0; j < R1; ++j) {
                        const int col = t + R2 * j;
                        const int gc = o1 + col;
                        a[j] = rin && col < L2 && gc >= 0 && gc < p.nx[1]
                                   ? float2{__ldg(x0 + xr + col), has1 ? __ldg(x1 + xr + col) : 0.0f}
                                   : zero;
                    }
                }
                float2 *row = Sb + line * kBPitch;
                LinScratch scr{row};
                fft_line<P, false>(a, tw, t, scr, lmask);
#pragma unroll
                for (int j = 0; j < R1; ++j) row[t + R2 * j] = a[j];
            }
            __syncthreads();
            // the tile's columns to G: warp w writes columns w, w + 16, ...; lane = row
            const int nr = min(LINES, rows_in - r0);
            if (lane < nr)
                for (int k = warp; k < P; k += kBThreads / 32) __stcg(G + int64_t(k) * P + r0 + lane, Sb[lane * kBPitch + k]);
            __syncthreads();
        }
        __threadfence_block();

        // ---------------- phase B: per column, FFT, spectral product, inverse FFT (in G)
        for (int k = line; k < P; k += LINES) {
            float2 a[R1];
            float2 *gc = G + int64_t(k) * P + t;
#pragma unroll
            for (int j = 0; j < R1; ++j) a[j] = t + R2 * j < rows_in ? __ldcg(gc + R2 * j) : zero;
            LinScratch scr{Sb + line * kBPitch};
            fft_line<P, false>(a, tw, t, scr, lmask);
            // Hermitian half spectrum [k2 <= P/2][k1]; mirrored columns read index P - k1
            if (k <= P / 2) {
                const float2 *sc = spec + int64_t(tile.spec) * p.spec_stride + int64_t(k) * P + t;
#pragma unroll
                for (int j = 0; j < R1; ++j) {
                    const float2 v = __ldg(sc + R2 * j);
                    a[j] = ADJ ? cmulc(a[j], v) : cmul(a[j], v);
                }
            } else {
                const float2 *sc = spec + int64_t(tile.spec) * p.spec_stride + int64_t(P - k) * P;
#pragma unroll
                for (int j = 0; j < R1; ++j) {
                    const float2 v = __ldg(sc + ((P - (t + R2 * j)) & (P - 1)));
                    a[j] = ADJ ? cmul(a[j], v) : cmulc(a[j], v);
                }
            }
            fft_line<P, true>(a, tw, t, scr, lmask);
#pragma unroll
            for (int j = 0; j < R1; ++j)
                if (t + R2 * j < rows_out) __stcg(gc + R2 * j, a[j]);
        }

        // ---------------- the previous item's reductions have landed: publish it
        if (t == 0 && pend) {
            bulk_wait_all();
            fence_proxy_async_global();
        }
        __syncthreads();
        if (threadIdx.x == 0 && pend) {
            __threadfence();
            st_release_u32(pend_flag, p.epoch);
        }
        pend = false;

        // ---------------- ordered overlap-add: wait for lower colours
        bool bad = false;
        {
            const int d0 = p.dep_start[ti], nd = p.dep_start[ti + 1] - d0;
            for (int d = threadIdx.x; d < nd && !bad; d += blockDim.x) {
                const uint32_t *f = p.done + int64_t(p.dep[d0 + d]) * p.done_ld + pair;
                bad = !wait_flag_eq<false>(f, p.epoch, p.ctrl + 2, lim, 1, 64);
                __threadfence();
            }
        }
        if (__syncthreads_or(bad)) break;

        // ---------------- phase C: output rows, 32 at a time: tile from G's
        // columns, inverse row FFTs, overlap-add
        float *y0 = y + int64_t(b0) * p.ldy;
        float *y1 = has1 ? y0 + p.ldy : y0;
        if (t == 0) fence_proxy_async_global();
        for (int r0 = 0; r0 < rows_out; r0 += LINES) {
            const int nr = min(LINES, rows_out - r0);
            if (lane < nr)
                for (int k = warp; k < P; k += kBThreads / 32) Sb[lane * kBPitch + k] = __ldcg(G + int64_t(k) * P + r0 + lane);
            __syncthreads();
            const int n = r0 + line;
            if (n < rows_out) {
                float2 *row = Sb + line * kBPitch;
                float2 a[R1];
#pragma unroll
                for (int j = 0; j < R1; ++j) a[j] = row[t + R2 * j];
                LinScratch scr{row};
                fft_line<P, true>(a, tw, t, scr, lmask);
                float *st = stage + line * kBStage;
                if constexpr (!ADJ) {
                    const int oy = o0 + n;
                    if (oy >= 0 && oy < p.n[0])
                        add_row_f32<P>(a, t, lmask, st, kBImOff, y0 + int64_t(oy) * p.n[1], y1 + int64_t(oy) * p.n[1],
                                       has1, o1, L2, p.n[1]);
                } else {
                    const float *wr = wt + int64_t(n) * tile.w_ld[0];
#pragma unroll
                    for (int j = 0; j < R1; ++j) {
                        const float wv = t + R2 * j < n2 ? __ldg(wr + t + R2 * j) : 0.0f;
                        a[j] = float2{a[j].x * wv, a[j].y * wv};
                    }
                    const int oy = i0 + n;
                    add_row_f32<P>(a, t, lmask, st, kBImOff, y0 + int64_t(oy) * p.n[1], y1 + int64_t(oy) * p.n[1],
                                   has1, j0, n2, p.n[1]);
                }
            }
            // the staging rows must have been read before the next round's rows overwrite the tile
            if (t == 0) bulk_wait_read();
            __syncthreads();
        }
        pend = true;
        pend_flag = p.done + int64_t(ti) * p.done_ld + pair;
    }
    if (t == 0 && pend) {
        bulk_wait_all();
        fence_proxy_async_global();
    }
    __syncthreads();
    if (threadIdx.x == 0 && pend) {
        __threadfence();
        st_release_u32(pend_flag, p.epoch);
    }
}

}  // namespace

cudaError_t fft2d_big_configure(int *ctas_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(fft2d_big_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         int(kBSmem));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(fft2d_big_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(kBSmem));
    int n = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fft2d_big_kernel<false>, kBThreads, kBSmem);
    if (ctas_per_sm) *ctas_per_sm = n;
    return e;
}

size_t fft2d_big_scratch_bytes(int ctas) { return size_t(ctas) * kBP * kBP * sizeof(float2); }

cudaError_t launch_fft2d_big(const ApplyParams &p, int ctas, void *scratch, cudaStream_t s, bool adjoint) {
    if (adjoint)
        fft2d_big_kernel<true><<<ctas, kBThreads, kBSmem, s>>>(p, static_cast<float2 *>(scratch));
    else
        fft2d_big_kernel<false><<<ctas, kBThreads, kBSmem, s>>>(p, static_cast<float2 *>(scratch));
    return cudaGetLastError();
}

}  // namespace pc
