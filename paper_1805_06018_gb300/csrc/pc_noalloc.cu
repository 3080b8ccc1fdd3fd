// pc_apply_batched_noalloc: the fused batched apply with its scratch in a
// file-scope device array, for callers that must not allocate device memory
// while they run.
//
// The fused patch kernel needs, beyond x, y and the operator's own data,
// a small scratch area: one ordering flag per (tile, right-hand-side pair)
// and a control block (work counter, timeout flag).  pc_apply_batched keeps
// it in memory the operator allocates on demand (it grows when a larger
// batch arrives).  Here it lives in g_noalloc_scratch instead, a statically
// sized __device__ array that every GPU which loads libpc holds until the
// process exits.
#include <mutex>

#include "pc_internal.h"

namespace {

// 1 MiB: the control block (16 words) plus up to kNoAllocFlagWords flags,
// i.e. tiles x ceil(nrhs/2) <= 262128.
constexpr int64_t kNoAllocWords = int64_t(1) << 18;
constexpr int64_t kNoAllocCtrlWords = 16;
constexpr int64_t kNoAllocFlagWords = kNoAllocWords - kNoAllocCtrlWords;

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNoAllocWords];

// y = 0 for the batch, flags of this call cleared, work counter reset.
template <typename T>
__global__ void noalloc_prepare(T *y, int64_t ldy, int32_t nrhs, int64_t N, uint32_t *scratch, int64_t nflags) {
    const int64_t stride = int64_t(gridDim.x) * blockDim.x;
    const int64_t i0 = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (i0 == 0) {
        scratch[0] = 0u;   // 64-bit work counter, low word
        scratch[1] = 0u;   // high word
        scratch[2] = 0u;   // timeout flag
    }
    for (int64_t i = i0; i < nflags; i += stride) scratch[kNoAllocCtrlWords + i] = 0u;
    const int64_t total = int64_t(nrhs) * N;
    for (int64_t i = i0; i < total; i += stride) {
        const int64_t b = i / N, e = i - b * N;
        y[b * ldy + e] = T(0);
    }
}

// Device address of g_noalloc_scratch, looked up once per device.  In host
// code the symbol itself is only a host-side handle; kernels must be given the
// address cudaGetSymbolAddress returns with the device current.  The same
// set-up loads this path's kernels (under lazy module loading a kernel's
// module is otherwise loaded, and its device memory taken, at its first
// launch), so that later calls take no device memory at all.
std::mutex g_mu;
uint32_t *g_addr[64] = {};

cudaError_t scratch_address(int device, uint32_t **out) {
    if (device < 0 || device >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[device]) {
        void *ptr = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        cudaFuncAttributes fa;
        if ((e = cudaFuncGetAttributes(&fa, noalloc_prepare<float>)) != cudaSuccess ||
            (e = cudaFuncGetAttributes(&fa, noalloc_prepare<double>)) != cudaSuccess)
            return e;
        g_addr[device] = static_cast<uint32_t *>(ptr);
    }
    *out = g_addr[device];
    return cudaSuccess;
}

// Select `device` for the lifetime of the guard (restored afterwards).
struct DeviceSel {
    int prev = -1;
    bool ok = false;
    explicit DeviceSel(int device) {
        if (cudaGetDevice(&prev) != cudaSuccess) return;
        ok = prev == device || cudaSetDevice(device) == cudaSuccess;
    }
    ~DeviceSel() {
        if (ok && prev >= 0) cudaSetDevice(prev);
    }
};

}  // namespace

extern "C" pc_status pc_noalloc_check(pc_context *ctx, pc_stream stream) {
    if (!ctx) return PC_ERR_ARG;
    DeviceSel sel(ctx->device);
    if (!sel.ok) {
        ctx->last_error = "cannot select the context's device";
        return PC_ERR_CUDA;
    }
    uint32_t *scratch = nullptr;
    cudaError_t e = scratch_address(ctx->device, &scratch);
    if (e == cudaSuccess) e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
    uint32_t flag = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&flag, scratch + 2, sizeof(flag), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && flag != 0) {
        e = cudaMemset(scratch + 2, 0, sizeof(flag));
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        ctx->last_error = std::string("reading the allocation-free apply's status: ") + cudaGetErrorString(e);
        return PC_ERR_CUDA;
    }
    if (flag != 0) {
        ctx->last_error = "a device-side wait of the last allocation-free apply ran out";
        return PC_ERR_TIMEOUT;
    }
    return PC_OK;
}

extern "C" pc_status pc_apply_batched_noalloc(pc_operator *op, int32_t nrhs, const void *x, int64_t ldx, void *y,
                                              int64_t ldy, pc_stream stream) {
    if (!op) return PC_ERR_ARG;
    pc_context *ctx = op->ctx;
    auto fail = [&](pc_status st, const std::string &msg) {
        ctx->last_error = msg;
        return st;
    };
    if (nrhs < 0) return fail(PC_ERR_ARG, "nrhs < 0");
    if (op->d != 2) return fail(PC_ERR_UNSUPPORTED, "the allocation-free apply covers 2D operators");
    DeviceSel sel(ctx->device);
    if (!sel.ok) return fail(PC_ERR_CUDA, "cannot select the context's device");
    // set-up first, so that a call with nrhs == 0 serves as the warm-up call
    uint32_t *scratch = nullptr;
    cudaError_t e = scratch_address(ctx->device, &scratch);
    if (e != cudaSuccess) return fail(PC_ERR_CUDA, std::string("setting up the static scratch: ") + cudaGetErrorString(e));
    if (nrhs == 0) return PC_OK;
    if (!x || !y) return fail(PC_ERR_ARG, "null x or y");
    if (ldx < op->N || ldy < op->N) return fail(PC_ERR_ARG, "ldx and ldy must be >= N");
    const uintptr_t xa = reinterpret_cast<uintptr_t>(x), ya = reinterpret_cast<uintptr_t>(y);
    if (xa % op->elem || ya % op->elem) return fail(PC_ERR_ARG, "x and y must be aligned to the element size");
    const uintptr_t xe = xa + uintptr_t((int64_t(nrhs - 1) * ldx + op->N) * op->elem);
    const uintptr_t ye = ya + uintptr_t((int64_t(nrhs - 1) * ldy + op->N) * op->elem);
    if (xa < ye && ya < xe) return fail(PC_ERR_ARG, "x and y overlap");
    const int32_t npairs = (nrhs + 1) / 2;
    const int64_t nflags = int64_t(op->n_tiles) * npairs;
    if (nflags > kNoAllocFlagWords)
        return fail(PC_ERR_ARG, "tiles x ceil(nrhs/2) = " + std::to_string(nflags) +
                                    " exceeds the static scratch of pc_apply_batched_noalloc (" +
                                    std::to_string(kNoAllocFlagWords) + " flags); split the batch");
    pc_status st = PC_OK;
    {
        cudaStream_t s = static_cast<cudaStream_t>(stream);
        const int64_t total = std::max<int64_t>(nflags, int64_t(nrhs) * op->N);
        const int blocks = int(std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 4096)));
        if (op->prec == PC_FP64)
            noalloc_prepare<double><<<blocks, 256, 0, s>>>(static_cast<double *>(y), ldy, nrhs, op->N, scratch, nflags);
        else
            noalloc_prepare<float><<<blocks, 256, 0, s>>>(static_cast<float *>(y), ldy, nrhs, op->N, scratch, nflags);
        e = cudaGetLastError();
        if (e == cudaSuccess) {
            pc::ApplyParams p{};
            p.x = x;
            p.y = y;
            p.ldx = ldx;
            p.ldy = ldy;
            p.nrhs = nrhs;
            p.npairs = npairs;
            p.n[0] = int32_t(op->shape[0]);
            p.n[1] = int32_t(op->shape[1]);
            p.n[2] = int32_t(op->shape[2]);
            p.nx[0] = p.n[0];
            p.nx[1] = p.n[1];
            p.nx[2] = p.n[2];
            p.R = op->R;
            p.tiles = op->d_tiles;
            p.color_start = op->d_color_start;
            p.n_colors = op->n_colors;
            p.dep_start = op->d_dep_start;
            p.dep = op->d_dep;
            p.done = scratch + kNoAllocCtrlWords;
            p.done_ld = npairs;
            p.epoch = 1u;   // flags were just cleared to 0
            p.ctrl = reinterpret_cast<int32_t *>(scratch);
            p.spec = op->d_spec;
            p.spec_stride = op->spec_stride;
            p.w = op->d_w;
            p.tw = op->d_tw;
            p.wait_ns = op->wait_ns;
            p.total_items = int64_t(op->n_tiles) * npairs;
            if (op->parts.empty()) {
                const int ctas = int(std::min<int64_t>(op->ctas, p.total_items));
                e = pc::launch_fft2d(p, op->P, op->prec, ctas, s);
            }
            // a per_patch operator: its parts one after another, the claim
            // counter reset between them (noalloc_prepare reset it for the first)
            for (size_t q = 0; q < op->parts.size() && e == cudaSuccess; ++q) {
                const pc::ApplyParams pq = pc::part_params(op, op->parts[q], p);
                if (q > 0) e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), s);
                const int ctas = int(std::min<int64_t>(op->ctas, pq.total_items));
                if (e == cudaSuccess && ctas > 0)
                    e = op->parts[q].P == pc::kBigFft ? pc::launch_fft2d_big(pq, ctas, op->d_big_scratch, s, false)
                                                      : pc::launch_fft2d(pq, op->parts[q].P, op->prec, ctas, s);
            }
        }
        if (e != cudaSuccess) st = fail(PC_ERR_CUDA, std::string("launching the apply: ") + cudaGetErrorString(e));
    }
    return st;
}
