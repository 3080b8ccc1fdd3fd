// Matrix entries of the approximation (Section 3.1):
//
//   A~[y, x] = sum_{k : x in U_k} w_k[x] phi_k^E[y - x]          (Eq. conv_matrix_entries)
//
// w_k vanishes outside U_k, and a point x in a leaf cell C lies in U_k only
// for the sample points p_k of C (corners and hanging nodes on its facets),
// so an entry costs O(points per cell): the operator keeps, per pixel, one
// leaf cell that contains it and, per cell, its sample points.  phi_k^E is
// kept in FP64 on its window [-R, R]^d; w_k in the operator's precision.
#include "pc_internal.h"

namespace pc {
namespace {

template <typename T>
__global__ void entries_kernel(int64_t n, const int64_t *rows, const int64_t *cols, double *out, EntryData e,
                               const T *w) {
    const int64_t N = int64_t(e.n[0]) * e.n[1] * e.n[2];
    const int W = 2 * e.R + 1;
    const int W1 = e.d >= 2 ? W : 1, W2 = e.d == 3 ? W : 1;
    const int64_t wsz = int64_t(W) * W1 * W2;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t y = rows[i], x = cols[i];
        if (y < 0 || y >= N || x < 0 || x >= N) {   // invalid index: NaN, no access
            out[i] = __longlong_as_double(0x7ff8000000000000ll);
            continue;
        }
        const int64_t x2 = x % e.n[2], x1 = (x / e.n[2]) % e.n[1], x0 = x / (int64_t(e.n[1]) * e.n[2]);
        const int64_t y2 = y % e.n[2], y1 = (y / e.n[2]) % e.n[1], y0 = y / (int64_t(e.n[1]) * e.n[2]);
        // window offsets (axes beyond d have extent 1 and offset 0)
        const int64_t z0 = y0 - x0, z1 = y1 - x1, z2 = y2 - x2;
        const int64_t h1 = (W1 - 1) / 2, h2 = (W2 - 1) / 2;
        double acc = 0.0;
        if (z0 >= -e.R && z0 <= e.R && z1 >= -h1 && z1 <= h1 && z2 >= -h2 && z2 <= h2) {
            const int64_t widx = ((z0 + e.R) * W1 + (z1 + h1)) * W2 + (z2 + h2);
            const int c = e.cell_of[x];
            for (int j = e.cpts_start[c]; j < e.cpts_start[c + 1]; ++j) {
                const int k = e.cpts[j];
                const int32_t *lo = e.bb_lo + 3 * k, *ext = e.bb_ext + 3 * k;
                const int64_t widx_w = ((x0 - lo[0]) * ext[1] + (x1 - lo[1])) * ext[2] + (x2 - lo[2]);
                acc += double(w[e.w_off[k] + widx_w]) * e.phiE[int64_t(k) * wsz + widx];
            }
        }
        out[i] = acc;
    }
}

}  // namespace

cudaError_t launch_entries(pc_precision prec, int64_t n, const int64_t *rows, const int64_t *cols, double *out,
                           const EntryData &e, const void *w, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    const int blocks = int(std::min<int64_t>((n + 255) / 256, 8192));
    if (prec == PC_FP64)
        entries_kernel<double><<<blocks, 256, 0, s>>>(n, rows, cols, out, e, static_cast<const double *>(w));
    else
        entries_kernel<float><<<blocks, 256, 0, s>>>(n, rows, cols, out, e, static_cast<const float *>(w));
    return cudaGetLastError();
}

}  // namespace pc
