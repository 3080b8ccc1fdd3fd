// 3D patch path for y = sum_k phi_k^E * (w_k . x)  (Eq. conv_op_approx_main), P = 64.
//
// A 64^3 complex field (2 MB) does not fit in one CTA's shared memory, so a
// work item (tile, pair of right-hand sides) runs in three phases around a
// per-CTA scratch volume G in global memory, laid out [plane][k2][k1]:
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
// Overlap-add order, termination and determinism are those of the 2D kernel:
// colour-ordered tiles, claims in increasing order, bounded waits.  Scratch
// traffic is about 6.7 MB per item; the line FFTs (about 20,000 of length 64
// per item) dominate the time.
#include "pc_fftcore.cuh"
#include "pc_internal.h"
#include "pc_ptx.cuh"

namespace pc {

constexpr int kThreads3d = 256;
constexpr int kP3 = 64;
constexpr long long kSpinLimit3 = 1ll << 24;

__global__ void __launch_bounds__(kThreads3d, 3) fft3d_kernel(const ApplyParams p, float2 *scratch) {
    using C = float2;
    constexpr int P = kP3;
    constexpr int R1 = FftShape<P>::R1, R2 = FftShape<P>::R2;
    constexpr int LINES = kThreads3d / R2;
    constexpr int PP = P * P;
    __shared__ __align__(16) C S[P * P];
    __shared__ int64_t s_item;

    const int t = threadIdx.x % R2;
    const int line = threadIdx.x / R2;
    const unsigned lmask = FftShape<P>::line_mask();
    const C *twg = static_cast<const C *>(p.tw);
    C tw[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) tw[m] = twg[(t * m) & (P - 1)];
    const float *x = static_cast<const float *>(p.x);
    float *y = static_cast<float *>(p.y);
    const float *w = static_cast<const float *>(p.w);
    const C *spec = static_cast<const C *>(p.spec);
    C *G = scratch + int64_t(blockIdx.x) * P * PP;
    const C zero{0.0f, 0.0f};
    const int n1box = p.n[1], n2box = p.n[2];
    const int64_t plane_box = int64_t(n1box) * n2box;

    for (;;) {
        if (threadIdx.x == 0) s_item = int64_t(atomicAdd(reinterpret_cast<unsigned long long *>(p.ctrl), 1ull));
        __syncthreads();
        const int64_t item = s_item;
        if (item >= p.total_items) break;
        int c = 0;
        while (int64_t(p.color_start[c + 1]) * p.npairs <= item) ++c;
        const int64_t base = int64_t(p.color_start[c]) * p.npairs;
        const int ntc = p.color_start[c + 1] - p.color_start[c];
        const int pair = int((item - base) / ntc);
        const int ti = p.color_start[c] + int((item - base) % ntc);
        const Tile tile = p.tiles[ti];
        const int n0 = tile.in_ext[0], n1 = tile.in_ext[1], n2 = tile.in_ext[2];
        const int L0 = n0 + tile.kext[0] - 1, L1 = n1 + tile.kext[1] - 1, L2 = n2 + tile.kext[2] - 1;
        const int b0 = 2 * pair;
        const bool has1 = b0 + 1 < p.nrhs;
        const float *x0 = x + int64_t(b0) * p.ldx;
        const float *x1 = has1 ? x0 + p.ldx : x0;
        const float *wt = w + tile.w_base;
        const C *sp = spec + int64_t(tile.spec) * p.spec_stride;

        // ---------------- phase 1: 2D FFT of each non-zero input plane -> G[i0][k2][k1]
        for (int i0 = 0; i0 < n0; ++i0) {
            const float *wp = wt + int64_t(i0) * tile.w_ld[0];
            const int64_t xp = int64_t(tile.in_lo[0] + i0) * plane_box;
            for (int r = line; r < n1; r += LINES) {
                C a[R1];
                const int64_t xr = xp + int64_t(tile.in_lo[1] + r) * n2box + tile.in_lo[2];
                const float *wr = wp + int64_t(r) * tile.w_ld[1];
#pragma unroll
                for (int j = 0; j < R1; ++j) {
                    const int col = t + R2 * j;
                    if (col < n2) {
                        const float wv = __ldg(wr + col);
                        a[j] = C{wv * __ldg(x0 + xr + col), has1 ? wv * __ldg(x1 + xr + col) : 0.0f};
                    } else {
                        a[j] = zero;
                    }
                }
                RowScratch<P, C> scr{S, r};
                fft_line<P, false>(a, tw, t, scr, lmask);
#pragma unroll
                for (int j = 0; j < R1; ++j) S[r * P + ((t + R2 * j) ^ swz(r))] = a[j];
            }
            __syncthreads();
            for (int k2 = line; k2 < P; k2 += LINES) {
                C a[R1];
#pragma unroll
                for (int j = 0; j < R1; ++j) {
                    const int row = t + R2 * j;
                    a[j] = row < n1 ? S[row * P + (k2 ^ swz(row))] : zero;
                }
                ColScratch<P, C> scr{S, k2};
                fft_line<P, false>(a, tw, t, scr, lmask);
                C *g = G + int64_t(i0) * PP + k2 * P;
#pragma unroll
                for (int j = 0; j < R1; ++j) __stcg(g + t + R2 * j, a[j]);
            }
            __syncthreads();
        }

        // ---------------- phase 2: first-axis FFT, spectral product, inverse, per (k1, k2)
        // stored spectrum: Hermitian half in k2, layout [k2 <= P/2][k1][k0]
        for (int l = line; l < PP; l += LINES) {
            const int k2 = l / P, k1 = l % P;
            C a[R1];
            C *g = G + k2 * P + k1;
#pragma unroll
            for (int j = 0; j < R1; ++j) {
                const int i0 = t + R2 * j;
                a[j] = i0 < n0 ? __ldcg(g + int64_t(i0) * PP) : zero;
            }
            // S is idle in this phase: row `line` is the line's transpose scratch
            RowScratch<P, C> scr{S, line};
            fft_line<P, false>(a, tw, t, scr, lmask);
            if (k2 <= P / 2) {
                const C *sc = sp + (int64_t(k2) * P + k1) * P;
#pragma unroll
                for (int j = 0; j < R1; ++j) a[j] = cmul(a[j], __ldg(sc + t + R2 * j));
            } else {
                const C *sc = sp + (int64_t(P - k2) * P + ((P - k1) & (P - 1))) * P;
#pragma unroll
                for (int j = 0; j < R1; ++j) a[j] = cmulc(a[j], __ldg(sc + ((P - (t + R2 * j)) & (P - 1))));
            }
            fft_line<P, true>(a, tw, t, scr, lmask);
#pragma unroll
            for (int j = 0; j < R1; ++j) {
                const int o0 = t + R2 * j;
                if (o0 < L0) __stcg(g + int64_t(o0) * PP, a[j]);
            }
        }
        __syncthreads();

        // ---------------- ordered overlap-add: wait for lower colours
        {
            const int d0 = p.dep_start[ti], nd = p.dep_start[ti + 1] - d0;
            for (int d = threadIdx.x; d < nd; d += blockDim.x) {
                const uint32_t *f = p.done + int64_t(p.dep[d0 + d]) * p.done_ld + pair;
                long long spins = 0;
                while (ld_acquire_u32(f) != p.epoch) {
                    if (++spins > kSpinLimit3) {
                        atomicExch(p.ctrl + 2, 1);
                        break;
                    }
                    __nanosleep(64);
                }
                __threadfence();
            }
        }
        __syncthreads();

        // ---------------- phase 3: inverse 2D FFT of each output plane, overlap-add
        float *y0 = y + int64_t(b0) * p.ldy;
        float *y1 = has1 ? y0 + p.ldy : y0;
        for (int o0 = 0; o0 < L0; ++o0) {
            const int gy0 = tile.out_lo[0] + o0;
            if (gy0 < 0 || gy0 >= p.n[0]) continue;   // uniform across the CTA
            // inverse along k1 for each k2: rows o1 of S
            const C *gp = G + int64_t(o0) * PP;
            for (int k2 = line; k2 < P; k2 += LINES) {
                C a[R1];
#pragma unroll
                for (int j = 0; j < R1; ++j) a[j] = __ldcg(gp + k2 * P + t + R2 * j);
                ColScratch<P, C> scr{S, k2};
                fft_line<P, true>(a, tw, t, scr, lmask);
#pragma unroll
                for (int j = 0; j < R1; ++j) {
                    const int o1 = t + R2 * j;
                    if (o1 < L1) S[o1 * P + (k2 ^ swz(o1))] = a[j];
                }
            }
            __syncthreads();
            for (int o1 = line; o1 < L1; o1 += LINES) {
                const int gy1 = tile.out_lo[1] + o1;
                if (gy1 < 0 || gy1 >= p.n[1]) continue;
                C a[R1];
#pragma unroll
                for (int j = 0; j < R1; ++j) a[j] = S[o1 * P + ((t + R2 * j) ^ swz(o1))];
                RowScratch<P, C> scr{S, o1};
                fft_line<P, true>(a, tw, t, scr, lmask);
                const int64_t yr = int64_t(gy0) * plane_box + int64_t(gy1) * n2box;
#pragma unroll
                for (int j = 0; j < R1; ++j) {
                    const int o2 = t + R2 * j;
                    const int gy2 = tile.out_lo[2] + o2;
                    if (o2 < L2 && gy2 >= 0 && gy2 < n2box) {
                        atomicAdd(y0 + yr + gy2, a[j].x);
                        if (has1) atomicAdd(y1 + yr + gy2, a[j].y);
                    }
                }
            }
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            __threadfence();
            st_release_u32(p.done + int64_t(ti) * p.done_ld + pair, p.epoch);
        }
    }
}

cudaError_t fft3d_configure(int *ctas_per_sm) {
    int n = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fft3d_kernel, kThreads3d, 0);
    if (ctas_per_sm) *ctas_per_sm = n;
    return e;
}

cudaError_t launch_fft3d(const ApplyParams &p, int ctas, void *scratch, cudaStream_t s) {
    fft3d_kernel<<<ctas, kThreads3d, 0, s>>>(p, static_cast<float2 *>(scratch));
    return cudaGetLastError();
}

size_t fft3d_scratch_bytes(int ctas) { return size_t(ctas) * kP3 * kP3 * kP3 * sizeof(float2); }

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
