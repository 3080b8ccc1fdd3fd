// One-time FP64 construction of the patch spectra phi^_k = DFT_P(psi_k) / P^d,
// psi[a] = a window (phi_k^E or one sub-window of it) placed at [0, W)^d,
// zero elsewhere in [0, P)^d.
//
// With this placement the linear convolution of a tile u (extent n per axis,
// n + 2R <= P) with phi_k^E comes out of the circular product at output index
// o = (x - tile origin) + z + R, i.e. at y = tile origin - R + o (Section 3.3's
// translation of a block to a small convolution).  The 1/P^d of the inverse
// transform is folded in here.  The stored layout is the Hermitian half in k2:
// 2D [k2 in 0..P/2][k1 in 0..P-1].  Twiddles W_P^j come from a host table in
// FP64 indexed by (a * k) mod P, so no twiddle is ever accumulated.
#include "pc_internal.h"

namespace pc {

// T1[k][a][c] = sum_b psi[k][a][b] W_P^{b c},  a in [0, 2R], c in [0, P/2]
__global__ void spectra2d_stage1(const double *psi, int r0, int nr, int W, int P, const double2 *tw, double2 *T1) {
    const int H = P / 2 + 1;
    const int64_t total = int64_t(nr) * W * H;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int c = int(i % H);
        const int a = int((i / H) % W);
        const int k = int(i / (int64_t(H) * W));
        const double *row = psi + (int64_t(r0 + k) * W + a) * W;
        double re = 0.0, im = 0.0;
        for (int b = 0; b < W; ++b) {
            const double2 wv = tw[(int64_t(b) * c) % P];
            re += row[b] * wv.x;
            im += row[b] * wv.y;
        }
        T1[i] = make_double2(re, im);
    }
}

// spec[k][c][k1] = (1/P^2) sum_a T1[k][a][c] W_P^{a k1}
template <typename C>
__global__ void spectra2d_stage2(const double2 *T1, int r0, int nr, int W, int P, const double2 *tw, C *spec) {
    const int H = P / 2 + 1;
    const double scale = 1.0 / (double(P) * double(P));
    const int64_t total = int64_t(nr) * H * P;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int k1 = int(i % P);
        const int c = int((i / P) % H);
        const int k = int(i / (int64_t(P) * H));
        double re = 0.0, im = 0.0;
        for (int a = 0; a < W; ++a) {
            const double2 t = T1[(int64_t(k) * W + a) * H + c];
            const double2 wv = tw[(int64_t(a) * k1) % P];
            re += t.x * wv.x - t.y * wv.y;
            im += t.x * wv.y + t.y * wv.x;
        }
        C out;
        out.x = decltype(out.x)(re * scale);
        out.y = decltype(out.y)(im * scale);
        spec[(int64_t(r0 + k) * H + c) * P + k1] = out;
    }
}

cudaError_t build_spectra_2d(const double *d_psi, int r, int W, int P, pc_precision prec, void *d_spec,
                             const double2 *d_tw64, cudaStream_t s) {
    const int H = P / 2 + 1;
    const int chunk = 256;
    double2 *T1 = nullptr;
    cudaError_t e = cudaMalloc(&T1, sizeof(double2) * size_t(chunk) * W * H);
    if (e != cudaSuccess) return e;
    for (int r0 = 0; r0 < r && e == cudaSuccess; r0 += chunk) {
        const int nr = std::min(chunk, r - r0);
        const int64_t n1 = int64_t(nr) * W * H, n2 = int64_t(nr) * H * P;
        spectra2d_stage1<<<int(std::min<int64_t>((n1 + 255) / 256, 8192)), 256, 0, s>>>(d_psi, r0, nr, W, P, d_tw64, T1);
        if (prec == PC_FP64)
            spectra2d_stage2<double2><<<int(std::min<int64_t>((n2 + 255) / 256, 8192)), 256, 0, s>>>(
                T1, r0, nr, W, P, d_tw64, static_cast<double2 *>(d_spec));
        else
            spectra2d_stage2<float2><<<int(std::min<int64_t>((n2 + 255) / 256, 8192)), 256, 0, s>>>(
                T1, r0, nr, W, P, d_tw64, static_cast<float2 *>(d_spec));
        e = cudaGetLastError();
    }
    cudaError_t e2 = cudaStreamSynchronize(s);
    cudaFree(T1);
    return e != cudaSuccess ? e : e2;
}

}  // namespace pc
