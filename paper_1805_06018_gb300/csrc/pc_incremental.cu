// Incremental update of Y~ = A~* Z for the adaptive construction
// (Algorithm 1; Section 2.8, construction cost):
//
//   A~* z = sum_k w_k . c_k,   c_k = flip(phi_k^E) * z on bbox(U_k)      (Eq. adjoint_random_z)
//
// c_k depends only on phi_k^E and bbox(U_k), so after a refinement it is
// recomputed only for sample points that are new or whose extension changed
// (a new neighbour); the others are kept.  Two kernels here:
//   block_copy_kernel    moves the kept correlation blocks into the new arena
//   corr_combine_kernel  Y~[b][x] = sum_{k : x in U_k} w_k[x] sum_s c_{k,s}[b][x - lo_k]
// The points k with x in U_k and w_k[x] != 0 are the sample points of a leaf
// cell containing x (corners and facet hanging nodes), the same tables the
// O(1) entries use; each output sums them in the cell's fixed point order, so
// Y~ is bitwise reproducible.
#include "pc_internal.h"

namespace pc {
namespace {

// copies[3 i + 0..2] = source offset, destination offset, length (elements)
template <typename T>
__global__ void block_copy_kernel(const int64_t *copies, const T *src, T *dst) {
    const int64_t so = copies[3 * blockIdx.x], dof = copies[3 * blockIdx.x + 1], len = copies[3 * blockIdx.x + 2];
    for (int64_t i = threadIdx.x; i < len; i += blockDim.x) dst[dof + i] = src[so + i];
}

// Correlation blocks of point k: [nsub2][q][e0][e1] at c + blk_off[k].
template <typename T>
__global__ void corr_combine_kernel(EntryData e, const T *w, const T *c, const int64_t *blk_off, int32_t nsub2,
                                    int32_t q, T *yt, int64_t N) {
    const int64_t total = int64_t(q) * N;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
        const int64_t b = i / N, x = i - b * N;
        const int64_t x1 = x % e.n[1], x0 = x / e.n[1];
        const int cell = e.cell_of[x];
        T acc = T(0);
        for (int j = e.cpts_start[cell]; j < e.cpts_start[cell + 1]; ++j) {
            const int k = e.cpts[j];
            const int32_t *lo = e.bb_lo + 3 * k, *ext = e.bb_ext + 3 * k;
            const int64_t E = int64_t(ext[0]) * ext[1];
            const int64_t local = (x0 - lo[0]) * ext[1] + (x1 - lo[1]);
            const T *ck = c + blk_off[k] + b * E + local;
            T sum = T(0);
            for (int sw = 0; sw < nsub2; ++sw) sum += ck[int64_t(sw) * q * E];
            acc += w[e.w_off[k] + local] * sum;
        }
        yt[b * N + x] = acc;
    }
}

}  // namespace

cudaError_t launch_block_copies(pc_precision prec, const int64_t *copies, int32_t n, const void *src, void *dst,
                                cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    if (prec == PC_FP64)
        block_copy_kernel<double><<<n, 256, 0, s>>>(copies, static_cast<const double *>(src),
                                                     static_cast<double *>(dst));
    else
        block_copy_kernel<float><<<n, 256, 0, s>>>(copies, static_cast<const float *>(src), static_cast<float *>(dst));
    return cudaGetLastError();
}

cudaError_t launch_corr_combine(pc_precision prec, const EntryData &e, const void *w, const void *c,
                                const int64_t *blk_off, int32_t nsub2, int32_t q, void *yt, int64_t N, cudaStream_t s) {
    const int64_t total = int64_t(q) * N;
    if (total <= 0) return cudaSuccess;
    const int blocks = int(std::min<int64_t>((total + 255) / 256, 16384));
    if (prec == PC_FP64)
        corr_combine_kernel<double><<<blocks, 256, 0, s>>>(e, static_cast<const double *>(w),
                                                           static_cast<const double *>(c), blk_off, nsub2, q,
                                                           static_cast<double *>(yt), N);
    else
        corr_combine_kernel<float><<<blocks, 256, 0, s>>>(e, static_cast<const float *>(w),
                                                          static_cast<const float *>(c), blk_off, nsub2, q,
                                                          static_cast<float *>(yt), N);
    return cudaGetLastError();
}

}  // namespace pc
