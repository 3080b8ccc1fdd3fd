// Overlap-add of one output row of a line FFT into y (FP32), shared by the 2D
// and 3D patch kernels.
#pragma once

#include "pc_fftcore.cuh"
#include "pc_ptx.cuh"

namespace pc {

// The line's R2 threads hold values m = t + R2 j of one output row; value m
// (< L2) goes to y[g0 + m] when 0 <= g0 + m < width (y0, y1: the row's base in
// the two right-hand sides of the pair; y1 only when has1).
//
// The values are laid out in the line's staging row `st` (re part at 0, im
// part at `imoff`, each shifted so that a 16-byte aligned y address meets a
// 16-byte aligned staging address), then lane 0 of the line hands the aligned
// interior of each part to the TMA unit as one bulk add-reduction; the at most
// three ragged values at either end are added by single atomics.  The
// reductions stay asynchronous: before the staging row is reused the line's
// lane 0 waits for them to have read it, and the caller waits for their
// completion (bulk_wait_all) before it publishes the tile as done.
template <int P, typename C>
__device__ __forceinline__ void add_row_f32(const C *a, int t, unsigned lmask, float *st, int imoff, float *y0,
                                            float *y1, bool has1, int g0, int L2, int width) {
    constexpr int R1 = FftShape<P>::R1, R2 = FftShape<P>::R2;
    const int lo = max(g0, 0), hi = min(g0 + L2, width);   // [lo, hi) in y coordinates
    // y row alignment (in elements, mod 4) and the aligned origin q <= lo of each part
    const int off0 = int((reinterpret_cast<uintptr_t>(y0) >> 2) & 3);
    const int off1 = int((reinterpret_cast<uintptr_t>(y1) >> 2) & 3);
    const int q0 = ((lo + off0) & ~3) - off0, q1 = ((lo + off1) & ~3) - off1;
    // the previous row's bulk reductions have finished reading `st`
    if (t == 0) bulk_wait_read();
    __syncwarp(lmask);
#pragma unroll
    for (int j = 0; j < R1; ++j) {
        const int gx = g0 + t + R2 * j;
        if (gx >= lo && gx < hi) {
            st[gx - q0] = a[j].x;
            st[imoff + gx - q1] = a[j].y;
        }
    }
    fence_proxy_async_smem();   // these generic writes are read by the bulk (async-proxy) reductions
    __syncwarp(lmask);
    // aligned interior [a, b) of each part; ragged ends by atomics
    const int a0 = lo == q0 ? q0 : q0 + 4, b0 = q0 + ((hi - q0) & ~3);
    const int a1 = lo == q1 ? q1 : q1 + 4, b1 = q1 + ((hi - q1) & ~3);
    if (t == 0) {
        if (b0 > a0) bulk_reduce_add_f32(y0 + a0, st + (a0 - q0), uint32_t(b0 - a0) * 4u);
        if (has1 && b1 > a1) bulk_reduce_add_f32(y1 + a1, st + imoff + (a1 - q1), uint32_t(b1 - a1) * 4u);
        bulk_commit();
    }
    if (b0 > a0) {
        for (int gx = lo + t; gx < a0; gx += R2) atomicAdd(y0 + gx, st[gx - q0]);
        for (int gx = b0 + t; gx < hi; gx += R2) atomicAdd(y0 + gx, st[gx - q0]);
    } else {
        for (int gx = lo + t; gx < hi; gx += R2) atomicAdd(y0 + gx, st[gx - q0]);
    }
    if (has1) {
        if (b1 > a1) {
            for (int gx = lo + t; gx < a1; gx += R2) atomicAdd(y1 + gx, st[imoff + gx - q1]);
            for (int gx = b1 + t; gx < hi; gx += R2) atomicAdd(y1 + gx, st[imoff + gx - q1]);
        } else {
            for (int gx = lo + t; gx < hi; gx += R2) atomicAdd(y1 + gx, st[imoff + gx - q1]);
        }
    }
}

}  // namespace pc

