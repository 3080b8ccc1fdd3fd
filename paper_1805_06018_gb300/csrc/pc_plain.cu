// Plain single-vector path: the reference point the fused kernels are
// measured against.  For each right-hand side separately:
//   1. gather   u_t = w_k . x on every tile t, zero-padded to P^d (HBM buffer)
//   2. cuFFT    batched R2C of all tiles (2D P x P, or 3D P x P x P)
//   3. product  U_t . phi^_k (half spectrum)
//   4. cuFFT    batched C2R
//   5. add      output-stationary overlap-add: every pixel sums the tiles that
//               cover it in ascending tile order (deterministic, no atomics)
// cuFFT is used here as a black-box library FFT.
#include <cufft.h>

#include "pc_internal.h"

namespace pc {

struct PlainState {
    cufftHandle fwd = 0, inv = 0;
    bool have_plans = false;
    float *real = nullptr;       // [n_tiles][P^d]
    float2 *freq = nullptr;      // [n_tiles][P^(d-1)][P/2+1]
    int32_t *blk_start = nullptr;  // CSR over output blocks (2D 32x32, 3D 8x8x8)
    int32_t *blk_tiles = nullptr;
    int nb0 = 0, nb1 = 0, nb2 = 1;
};

// 3D: u_t[a][b][c] = w_k . x over the tile's input box, zero elsewhere in P^3
__global__ void plain_gather3(const float *x, const Tile *tiles, const float *w, int n1, int n2, int P, float *real) {
    const Tile t = tiles[blockIdx.y];
    float *u = real + int64_t(blockIdx.y) * P * P * P;
    const int64_t PPP = int64_t(P) * P * P;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < PPP; i += int64_t(gridDim.x) * blockDim.x) {
        const int a = int(i / (P * P)), b = int((i / P) % P), c = int(i % P);
        float v = 0.0f;
        if (a < t.in_ext[0] && b < t.in_ext[1] && c < t.in_ext[2])
            v = w[t.w_base + int64_t(a) * t.w_ld[0] + int64_t(b) * t.w_ld[1] + c] *
                x[(int64_t(t.in_lo[0] + a) * n1 + t.in_lo[1] + b) * n2 + t.in_lo[2] + c];
        u[i] = v;
    }
}

// 3D: cuFFT's [k0][k1][k2 <= P/2] times the stored [k2][k1][k0] half spectrum
__global__ void plain_product3(float2 *freq, const Tile *tiles, const float2 *spec, int64_t spec_stride, int P) {
    const int H = P / 2 + 1;
    const Tile t = tiles[blockIdx.y];
    float2 *f = freq + int64_t(blockIdx.y) * P * P * H;
    const float2 *sp = spec + int64_t(t.spec) * spec_stride;
    const int64_t n = int64_t(P) * P * H;
    for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
        const int k2 = int(i % H), k1 = int((i / H) % P), k0 = int(i / (int64_t(H) * P));
        const float2 a = f[i], sv = sp[(int64_t(k2) * P + k1) * P + k0];
        f[i] = make_float2(a.x * sv.x - a.y * sv.y, a.x * sv.y + a.y * sv.x);
    }
}

// 3D output-stationary overlap-add over 8 x 8 x 8 blocks
__global__ void plain_add3(float *y, const float *real, const Tile *tiles, const int32_t *blk_start,
                           const int32_t *blk_tiles, int nb1, int nb2, int n0, int n1, int n2, int P) {
    const int i = blockIdx.z * 8 + threadIdx.z, j = blockIdx.y * 8 + threadIdx.y, l = blockIdx.x * 8 + threadIdx.x;
    if (i >= n0 || j >= n1 || l >= n2) return;
    const int blk = (blockIdx.z * nb1 + blockIdx.y) * nb2 + blockIdx.x;
    float acc = 0.0f;
    for (int q = blk_start[blk]; q < blk_start[blk + 1]; ++q) {
        const int ti = blk_tiles[q];
        const Tile t = tiles[ti];
        const int o0 = i - t.out_lo[0], o1 = j - t.out_lo[1], o2 = l - t.out_lo[2];
        if (o0 >= 0 && o0 < t.in_ext[0] + t.kext[0] - 1 && o1 >= 0 && o1 < t.in_ext[1] + t.kext[1] - 1 && o2 >= 0 &&
            o2 < t.in_ext[2] + t.kext[2] - 1)
            acc += real[((int64_t(ti) * P + o0) * P + o1) * P + o2];
    }
    y[(int64_t(i) * n1 + j) * n2 + l] = acc;
}

__global__ void plain_gather(const float *x, const Tile *tiles, const float *w, int n1box, int P, float *real) {
    const Tile t = tiles[blockIdx.x];
    float *u = real + int64_t(blockIdx.x) * P * P;
    for (int i = threadIdx.x; i < P * P; i += blockDim.x) {
        const int a = i / P, b = i % P;
        float v = 0.0f;
        if (a < t.in_ext[0] && b < t.in_ext[1])
            v = w[t.w_base + int64_t(a) * t.w_ld[0] + b] * x[int64_t(t.in_lo[0] + a) * n1box + t.in_lo[1] + b];
        u[i] = v;
    }
}

__global__ void plain_product(float2 *freq, const Tile *tiles, const float2 *spec, int64_t spec_stride, int P) {
    const int H = P / 2 + 1;
    const Tile t = tiles[blockIdx.x];
    float2 *f = freq + int64_t(blockIdx.x) * P * H;
    const float2 *sp = spec + int64_t(t.spec) * spec_stride;
    for (int i = threadIdx.x; i < P * H; i += blockDim.x) {
        const int k1 = i / H, k2 = i % H;
        const float2 a = f[i], s = sp[int64_t(k2) * P + k1];
        f[i] = make_float2(a.x * s.x - a.y * s.y, a.x * s.y + a.y * s.x);
    }
}

__global__ void plain_add(float *y, const float *real, const Tile *tiles, const int32_t *blk_start,
                          const int32_t *blk_tiles, int nb1, int n0, int n1, int P) {
    const int i = blockIdx.y * 32 + threadIdx.y;
    const int j = blockIdx.x * 32 + threadIdx.x;
    if (i >= n0 || j >= n1) return;
    const int blk = blockIdx.y * nb1 + blockIdx.x;
    float acc = 0.0f;
    for (int q = blk_start[blk]; q < blk_start[blk + 1]; ++q) {
        const int ti = blk_tiles[q];
        const Tile t = tiles[ti];
        const int o0 = i - t.out_lo[0], o1 = j - t.out_lo[1];
        if (o0 >= 0 && o0 < t.in_ext[0] + t.kext[0] - 1 && o1 >= 0 && o1 < t.in_ext[1] + t.kext[1] - 1)
            acc += real[(int64_t(ti) * P + o0) * P + o1];
    }
    y[int64_t(i) * n1 + j] = acc;
}

static void destroy_state(PlainState *st) {
    if (!st) return;
    if (st->have_plans) {
        cufftDestroy(st->fwd);
        cufftDestroy(st->inv);
    }
    cudaFree(st->real);
    cudaFree(st->freq);
    cudaFree(st->blk_start);
    cudaFree(st->blk_tiles);
    delete st;
}

void plain_free(pc_operator *op) {
    destroy_state(static_cast<PlainState *>(op->plain));
    op->plain = nullptr;
}

static pc_status plain_init(pc_operator *op, std::string &err) {
    auto *st = new PlainState;
    const bool three = op->d == 3;
    const int P = op->P, H = P / 2 + 1, nt = op->n_tiles;
    const int64_t vol = three ? int64_t(P) * P * P : int64_t(P) * P;
    const int64_t hvol = three ? int64_t(P) * P * H : int64_t(P) * H;
    int dims[3] = {P, P, P};
    cudaError_t e = cudaMalloc(&st->real, sizeof(float) * size_t(nt) * size_t(vol));
    if (e == cudaSuccess) e = cudaMalloc(&st->freq, sizeof(float2) * size_t(nt) * size_t(hvol));
    if (e != cudaSuccess) {
        destroy_state(st);
        err = std::string("plain path scratch: ") + cudaGetErrorString(e);
        return PC_ERR_NOMEM;
    }
    const int rank = three ? 3 : 2;
    if (cufftPlanMany(&st->fwd, rank, dims, nullptr, 1, int(vol), nullptr, 1, int(hvol), CUFFT_R2C, nt) !=
            CUFFT_SUCCESS ||
        cufftPlanMany(&st->inv, rank, dims, nullptr, 1, int(hvol), nullptr, 1, int(vol), CUFFT_C2R, nt) !=
            CUFFT_SUCCESS) {
        destroy_state(st);
        err = "cuFFT plan creation failed";
        return PC_ERR_CUDA;
    }
    st->have_plans = true;
    // tiles covering each output block (2D 32 x 32, 3D 8 x 8 x 8)
    const int blk = three ? 8 : 32;
    const int n0 = int(op->shape[0]), n1 = int(op->shape[1]), n2 = int(op->shape[2]);
    st->nb0 = (n0 + blk - 1) / blk;
    st->nb1 = (n1 + blk - 1) / blk;
    st->nb2 = three ? (n2 + blk - 1) / blk : 1;
    std::vector<std::vector<int32_t>> lists(size_t(st->nb0) * st->nb1 * st->nb2);
    for (int ti = 0; ti < nt; ++ti) {
        const Tile &t = op->tiles_h[ti];
        int lo[3], hi[3];
        for (int a = 0; a < 3; ++a) {
            const int n = int(op->shape[a]);
            lo[a] = std::max(0, t.out_lo[a]);
            hi[a] = std::min(n - 1, t.out_lo[a] + t.in_ext[a] + t.kext[a] - 2);
        }
        if (!three) lo[2] = hi[2] = 0;
        for (int bi = lo[0] / blk; bi <= hi[0] / blk; ++bi)
            for (int bj = lo[1] / blk; bj <= hi[1] / blk; ++bj)
                for (int bk = lo[2] / blk; bk <= hi[2] / blk; ++bk)
                    lists[(size_t(bi) * st->nb1 + bj) * st->nb2 + bk].push_back(ti);
    }
    std::vector<int32_t> start(1, 0), flat;
    for (auto &l : lists) {
        flat.insert(flat.end(), l.begin(), l.end());
        start.push_back(int32_t(flat.size()));
    }
    if (flat.empty()) flat.push_back(0);
    e = cudaMalloc(&st->blk_start, sizeof(int32_t) * start.size());
    if (e == cudaSuccess) e = cudaMalloc(&st->blk_tiles, sizeof(int32_t) * flat.size());
    if (e == cudaSuccess) e = cudaMemcpy(st->blk_start, start.data(), sizeof(int32_t) * start.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(st->blk_tiles, flat.data(), sizeof(int32_t) * flat.size(), cudaMemcpyHostToDevice);
    // the copies have landed before any apply on a caller's stream reads them
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        destroy_state(st);
        err = std::string("plain path tables: ") + cudaGetErrorString(e);
        return PC_ERR_CUDA;
    }
    op->plain = st;
    return PC_OK;
}

pc_status plain_apply(pc_operator *op, int32_t nrhs, const void *x, int64_t ldx, void *y, int64_t ldy,
                      cudaStream_t s, std::string &err) {
    if (!op->plain) {
        pc_status st = plain_init(op, err);
        if (st != PC_OK) return st;
    }
    auto *st = static_cast<PlainState *>(op->plain);
    if (cufftSetStream(st->fwd, s) != CUFFT_SUCCESS || cufftSetStream(st->inv, s) != CUFFT_SUCCESS) {
        err = "cufftSetStream failed";
        return PC_ERR_CUDA;
    }
    const int P = op->P, nt = op->n_tiles;
    const int n0 = int(op->shape[0]), n1 = int(op->shape[1]), n2 = int(op->shape[2]);
    const bool three = op->d == 3;
    int64_t launches = 0;
    for (int b = 0; b < nrhs; ++b) {
        const float *xb = static_cast<const float *>(x) + int64_t(b) * ldx;
        float *yb = static_cast<float *>(y) + int64_t(b) * ldy;
        if (three)
            plain_gather3<<<dim3(64, nt), 256, 0, s>>>(xb, op->d_tiles, static_cast<const float *>(op->d_w), n1, n2, P,
                                                       st->real);
        else
            plain_gather<<<nt, 256, 0, s>>>(xb, op->d_tiles, static_cast<const float *>(op->d_w), n1, P, st->real);
        if (cufftExecR2C(st->fwd, st->real, reinterpret_cast<cufftComplex *>(st->freq)) != CUFFT_SUCCESS) {
            err = "cufftExecR2C failed";
            return PC_ERR_CUDA;
        }
        if (three)
            plain_product3<<<dim3(64, nt), 256, 0, s>>>(st->freq, op->d_tiles, static_cast<const float2 *>(op->d_spec),
                                                        op->spec_stride, P);
        else
            plain_product<<<nt, 256, 0, s>>>(st->freq, op->d_tiles, static_cast<const float2 *>(op->d_spec),
                                             op->spec_stride, P);
        if (cufftExecC2R(st->inv, reinterpret_cast<cufftComplex *>(st->freq), st->real) != CUFFT_SUCCESS) {
            err = "cufftExecC2R failed";
            return PC_ERR_CUDA;
        }
        if (three)
            plain_add3<<<dim3(st->nb2, st->nb1, st->nb0), dim3(8, 8, 8), 0, s>>>(
                yb, st->real, op->d_tiles, st->blk_start, st->blk_tiles, st->nb1, st->nb2, n0, n1, n2, P);
        else
            plain_add<<<dim3(st->nb1, st->nb0), dim3(32, 32), 0, s>>>(yb, st->real, op->d_tiles, st->blk_start,
                                                                    st->blk_tiles, st->nb1, n0, n1, P);
        launches += 3;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        err = std::string("plain path launch: ") + cudaGetErrorString(e);
        return PC_ERR_CUDA;
    }
    op->launches_last = launches;
    return PC_OK;
}

}  // namespace pc
