// Randomized a-posteriori error estimator (Section 2.6).  For every leaf cell
// C of the operator's grid (closed box, grid order):
//
//   eta_C = (1/sqrt(q)) || Y~[C, .] - Y[C, .] ||_F        (Eq. randomized_estimator_ec)
//
// with Y~ = A~* Z from the adjoint apply and Y = A* Z supplied by the caller
// (the paper's matrix-free access to A*).  The squares are summed in FP64,
// one CTA per cell: each warp walks whole rows of the cell (lanes along the
// fastest axis, so loads are coalesced), and the CTA combines its per-thread
// sums in one fixed tree order, so the result is bitwise reproducible.
#include <cmath>
#include <vector>

#include "pc_internal.h"

namespace pc {
namespace {

constexpr int kThreadsEst = 256;

// cells: [nc][6] = lo0 lo1 lo2 hi0 hi1 hi2 on a box of extents (n0, n1, n2)
// whose last axis is the fastest (2D grids are passed as (1, n0, n1))
template <typename T>
__global__ void __launch_bounds__(kThreadsEst) cell_sqdiff_kernel(const T *yt, int64_t ldyt, const T *y, int64_t ldy,
                                                                  int32_t q, const int32_t *cells, int64_t n1,
                                                                  int64_t n2, double *out) {
    const int32_t *b = cells + 6 * int64_t(blockIdx.x);
    const int64_t e0 = b[3] - b[0] + 1, e1 = b[4] - b[1] + 1, e2 = b[5] - b[2] + 1;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
    const int64_t rows = int64_t(q) * e0 * e1;
    double acc = 0.0;
    for (int64_t row = warp; row < rows; row += nwarps) {
        const int64_t probe = row / (e0 * e1), rr = row - probe * e0 * e1;
        const int64_t a0 = rr / e1, a1 = rr - a0 * e1;
        const int64_t base = ((b[0] + a0) * n1 + (b[1] + a1)) * n2 + b[2];
        const T *pt = yt + probe * ldyt + base, *py = y + probe * ldy + base;
        for (int64_t a2 = lane; a2 < e2; a2 += 32) {
            const double d = double(pt[a2]) - double(py[a2]);
            acc += d * d;
        }
    }
    __shared__ double red[kThreadsEst];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = kThreadsEst / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

}  // namespace

cudaError_t launch_cell_sqdiff(pc_precision prec, const void *yt, int64_t ldyt, const void *y, int64_t ldy, int32_t q,
                               const int32_t *cells, int32_t ncells, int64_t n1, int64_t n2, double *out,
                               cudaStream_t s) {
    if (prec == PC_FP64)
        cell_sqdiff_kernel<double><<<ncells, kThreadsEst, 0, s>>>(static_cast<const double *>(yt), ldyt,
                                                                  static_cast<const double *>(y), ldy, q, cells, n1,
                                                                  n2, out);
    else
        cell_sqdiff_kernel<float><<<ncells, kThreadsEst, 0, s>>>(static_cast<const float *>(yt), ldyt,
                                                                 static_cast<const float *>(y), ldy, q, cells, n1, n2,
                                                                 out);
    return cudaGetLastError();
}

}  // namespace pc
