// Helpers shared by the translation units of the C ABI (pc_api.cpp,
// pc_block.cpp, pc_estimator.cpp): error recording, a device guard and
// host-to-device uploads.
#pragma once

#include <string>

#include "pc_internal.h"

namespace pc {

// Record msg as ctx's last error (the context-free last error when ctx is
// null) and return st.
pc_status fail(pc_context *ctx, pc_status st, const std::string &msg);
// A failed CUDA call: PC_ERR_NOMEM for an allocation failure, else PC_ERR_CUDA.
pc_status cuda_fail(pc_context *ctx, cudaError_t e, const char *what);

// Make ctx's device current for the duration of a call, then restore.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// Zero n device bytes at p and wait until the zeros have landed.  The
// synchronous cudaMemset (like cudaMemcpy from pageable host memory) may still
// be in flight on the legacy default stream when it returns, and kernels on
// non-blocking streams are not ordered after that stream.
inline cudaError_t zero_now(void *p, size_t n) {
    const cudaError_t e = cudaMemset(p, 0, n);
    return e == cudaSuccess ? cudaDeviceSynchronize() : e;
}

// cudaMalloc n elements at *dst, copy src there, count the bytes in acct.  The
// copy may still be in flight when this returns (see zero_now): callers
// synchronise the device before work on a caller's stream reads *dst.
template <typename T>
cudaError_t upload(T **dst, const T *src, size_t n, size_t &acct) {
    *dst = nullptr;
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), sizeof(T) * n);
    if (e != cudaSuccess) return e;
    acct += sizeof(T) * n;
    return cudaMemcpy(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice);
}

// upload, with the copy ordered on stream s instead (src must stay valid until
// the copy has run on s).
template <typename T>
cudaError_t upload_on(T **dst, const T *src, size_t n, size_t &acct, cudaStream_t s) {
    *dst = nullptr;
    if (n == 0) return cudaSuccess;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(dst), sizeof(T) * n);
    if (e != cudaSuccess) return e;
    acct += sizeof(T) * n;
    return cudaMemcpyAsync(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice, s);
}

}  // namespace pc
