// Tensor-core form of the 3D patch path's first-axis transform (BF16x3).
//
// Between phase 1 (2D FFTs of the input planes) and phase 3 (inverse 2D FFTs
// and the overlap-add) a 3D item needs, for each of its 64 x 64 (k2, k1)
// lines, the length-64 DFT along the first axis of the n0 non-zero planes,
// the product with the stored spectrum phi^_k (Section 3.2) and the inverse
// DFT restricted to the L0 = n0 + K0 - 1 output planes of the linear
// convolution.  Here both DFTs are dense GEMMs on the tcgen05 tensor cores,
// 128 lines at a time (one "unit"):
//
//   GEMM 1   D1[line][(k0, re|im)] = sum_(i0, re|im) U[line][(i0, re|im)] F1[(k0, re|im)][(i0, re|im)]
//   product  V^[line][k0] = D1[line][k0] * phi^[line][k0]          (CUDA cores)
//   GEMM 2   D2[line][(o0, re|im)] = sum_(k0, re|im) V^[line][(k0, re|im)] F2[(o0, re|im)][(k0, re|im)]
//
// F1 and F2 are the real 128 x 128 block forms of the complex DFT matrices
// W^(i0 k0) and W^(-o0 k0), W = exp(-2 pi i / 64).  Every operand a is split
// as a = a_hi + a_lo with a_hi = bf16(a), a_lo = bf16(a - a_hi), and a product
// is taken as a_lo b_hi + a_hi b_lo + a_hi b_hi with FP32 accumulation in
// tensor memory (the a_lo b_lo term, ~2^-16 relative, is dropped).
//
// F1 and F2 (hi and lo, 128 KB) are copied into shared memory once per CTA by
// the bulk-copy (TMA) engine; the data tile is split and written by the
// threads; D1 and D2 live in 128 columns of tensor memory.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "pc_internal.h"
#include "pc_ptx.cuh"
#include "pc_tc.cuh"

namespace pc {
namespace {

constexpr int kP = 64;
constexpr int kPlane = kP * kP;                     // (k2, k1) lines per item
constexpr int kBlock = 128;                         // lines per unit = MMA M
constexpr int kUnitsPerItem = kPlane / kBlock;      // 32
constexpr int kK = 2 * kP;                          // (index, re|im) = MMA K and N
constexpr int kTile = kBlock * kK * 2;              // one BF16 128 x 128 operand tile: 32 KB
constexpr int kThreads = 256;
constexpr uint32_t kLBO = 128u;                     // core matrices adjacent along K
constexpr uint32_t kSBO = uint32_t(kK * 2 / 16) * 128u;   // 8-row groups: 2048 B
constexpr int kSmem = 6 * kTile + 64;
constexpr long long kSpin = 1ll << 24;
constexpr uint32_t kIdesc = tc::idesc_bf16(kBlock, kK);

static_assert(kSmem <= 227 * 1024, "shared memory");
static_assert(tc::kmajor_offset(kBlock - 1, kK - 1, kK, 2) == kTile - 2, "tile layout");

// shared layout: [F1 hi | F1 lo | F2 hi | F2 lo | A hi | A lo | mbarriers, TMEM slot]

// 8 consecutive K values of one row -> hi and lo 16-byte core-matrix rows
__device__ __forceinline__ void split8_store(uint8_t *hi_tile, uint32_t off, const float *v) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
        const float2 hf = __bfloat1622float2(hb);
        const __nv_bfloat162 lb = __floats2bfloat162_rn(v[2 * i] - hf.x, v[2 * i + 1] - hf.y);
        h[i] = *reinterpret_cast<const uint32_t *>(&hb);
        l[i] = *reinterpret_cast<const uint32_t *>(&lb);
    }
    *reinterpret_cast<uint4 *>(hi_tile + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4 *>(hi_tile + kTile + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// D (tensor memory) = A * B^T over `steps` K steps of 16, three split products each
__device__ __forceinline__ void issue_gemm(uint32_t d_tmem, const uint8_t *a_tile, const uint8_t *b_tile, int steps) {
    const uint32_t a = smem_u32(a_tile), b = smem_u32(b_tile);
    for (int s = 0; s < steps; ++s) {
        const uint32_t o = 256u * uint32_t(s);
        const uint64_t ah = tc::smem_desc(a + o, kLBO, kSBO), al = tc::smem_desc(a + kTile + o, kLBO, kSBO);
        const uint64_t bh = tc::smem_desc(b + o, kLBO, kSBO), bl = tc::smem_desc(b + kTile + o, kLBO, kSBO);
        tc::mma<false>(d_tmem, al, bh, kIdesc, s > 0 ? 1u : 0u);
        tc::mma<false>(d_tmem, ah, bl, kIdesc, 1u);
        tc::mma<false>(d_tmem, ah, bh, kIdesc, 1u);
    }
}

// One unit: 128 consecutive (k2, k1) lines of one work item.
struct Unit {
    int line0, n0, L0, steps1, spec;
    float2 *G;   // the item's scratch volume [plane][k2][k1]
};

__device__ __forceinline__ Unit unit_of(const ApplyParams &p, float2 *scratch, int64_t c0, int64_t nitems,
                                        int64_t u) {
    // block index major, so that the items of one tile (all pairs) read the
    // same 64 KB spectrum block close together in time
    const int blk = int(u / nitems);
    const int64_t item = c0 + (u - int64_t(blk) * nitems);
    int c = 0;
    while (int64_t(p.color_start[c + 1]) * p.npairs <= item) ++c;
    const int64_t cbase = int64_t(p.color_start[c]) * p.npairs;
    const int ntc = p.color_start[c + 1] - p.color_start[c];
    const Tile &tile = p.tiles[p.color_start[c] + int((item - cbase) % ntc)];
    Unit x;
    x.n0 = tile.in_ext[0];
    x.L0 = x.n0 + tile.kext[0] - 1;
    x.steps1 = (2 * x.n0 + 15) / 16;
    x.spec = tile.spec;
    x.G = scratch + (item - c0) * int64_t(kP) * kPlane;
    x.line0 = blk * kBlock;
    return x;
}

// The GEMM-1 input of a unit: thread (m = tid % 128, h = tid / 128) holds
// groups g = h + 2 e of 4 planes (8 K values) of line line0 + m.  All loads
// are issued before any is used.
__device__ __forceinline__ void stage_load(const Unit &x, int tid, float2 (&z)[32]) {
    const int m = tid & (kBlock - 1), h = tid >> 7;
#pragma unroll
    for (int e = 0; e < 8; ++e)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i0 = 4 * (h + 2 * e) + q;
            z[4 * e + q] = i0 < x.n0 ? __ldcg(x.G + int64_t(i0) * kPlane + x.line0 + m) : make_float2(0.f, 0.f);
        }
}

__device__ __forceinline__ void stage_store(const Unit &x, int tid, const float2 (&z)[32], uint8_t *sA) {
    const int m = tid & (kBlock - 1), h = tid >> 7;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const int g = h + 2 * e;
        if (g < 2 * x.steps1) {
            float v[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                v[2 * q] = z[4 * e + q].x;
                v[2 * q + 1] = z[4 * e + q].y;
            }
            split8_store(sA, tc::kmajor_offset(m, 8 * g, kK, 2), v);
        }
    }
}

__global__ void __launch_bounds__(kThreads, 1)
    tc3d_axis0_kernel(const ApplyParams p, float2 *scratch, int64_t c0, int64_t c1, const uint8_t *ops) {
    extern __shared__ __align__(1024) uint8_t sm[];
    uint8_t *sF1 = sm, *sF2 = sm + 2 * kTile, *sA = sm + 4 * kTile;
    uint64_t *bar_ld = reinterpret_cast<uint64_t *>(sm + 6 * kTile);
    uint64_t *bar_mma = bar_ld + 1;
    uint32_t *slot = reinterpret_cast<uint32_t *>(bar_ld + 2);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t nitems = c1 - c0;
    const int64_t nunits = nitems * kUnitsPerItem;

    if (tid == 0) {
        mbar_init(bar_ld, 1);
        mbar_init(bar_mma, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(slot, 128);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    if (tid == 0) {
        mbar_arrive_expect_tx(bar_ld, 4 * kTile);
        for (int i = 0; i < 4; ++i) bulk_g2s(sm + i * kTile, ops + i * kTile, kTile, bar_ld);
    }
    bool ok = __syncthreads_and(mbar_wait_bounded(bar_ld, 0, kSpin));
    bool mma_pending = false;
    uint32_t phase = 0;

    // epilogue roles: warp w reads tensor-memory lanes 32 (w % 4) ... (its 32
    // lines) and the column half w / 4
    const int quarter = warp & 3, half = warp >> 2;
    const int erow = 32 * quarter + lane;
    const float2 *spec_all = static_cast<const float2 *>(p.spec);

    // software pipeline: the next unit's input is loaded while GEMM 2 runs,
    // the spectrum while GEMM 1 runs
    float2 z[32];
    int64_t u = blockIdx.x;
    Unit cur{};
    if (ok && u < nunits) {
        cur = unit_of(p, scratch, c0, nitems, u);
        stage_load(cur, tid, z);
    }
    for (; ok && u < nunits; u += gridDim.x) {
        // ---- A = split(U): rows = lines, K = (i0, re|im)
        stage_store(cur, tid, z, sA);
        fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            issue_gemm(tmem, sA, sF1, cur.steps1);
            tc::mma_commit(bar_mma);
        }
        mma_pending = true;
        // spectrum of this thread's line, k0 = 32 half ... 32 half + 31
        // (Hermitian mirror for k2 > P/2)
        float2 f[32];
        {
            const int line = cur.line0 + erow, k2 = line / kP, k1 = line % kP;
            const bool mirror = k2 > kP / 2;
            const float2 *sp = spec_all + int64_t(cur.spec) * p.spec_stride +
                               (mirror ? (int64_t(kP - k2) * kP + ((kP - k1) & (kP - 1))) * kP
                                       : (int64_t(k2) * kP + k1) * kP);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int k0 = 32 * half + j;
                f[j] = __ldg(sp + (mirror ? ((kP - k0) & (kP - 1)) : k0));
                if (mirror) f[j].y = -f[j].y;
            }
        }
        ok = __syncthreads_and(mbar_wait_bounded(bar_mma, phase, kSpin));
        if (!ok) break;
        mma_pending = false;
        phase ^= 1u;
        tc::fence_after_sync();

        // ---- V^ = D1 * phi^, split into A (K = (k0, re|im))
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
            float v[32];
            tc::tmem_ld32(tmem + (uint32_t(32 * quarter) << 16) + uint32_t(64 * half + 32 * cc), v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float2 w = f[16 * cc + j];
                const float re = v[2 * j] * w.x - v[2 * j + 1] * w.y;
                const float im = v[2 * j] * w.y + v[2 * j + 1] * w.x;
                v[2 * j] = re;
                v[2 * j + 1] = im;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
                split8_store(sA, tc::kmajor_offset(erow, 64 * half + 32 * cc + 8 * r, kK, 2), v + 8 * r);
        }
        fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            issue_gemm(tmem, sA, sF2, kK / 16);
            tc::mma_commit(bar_mma);
        }
        mma_pending = true;
        Unit nxt = cur;
        if (u + gridDim.x < nunits) {
            nxt = unit_of(p, scratch, c0, nitems, u + gridDim.x);
            stage_load(nxt, tid, z);
        }
        ok = __syncthreads_and(mbar_wait_bounded(bar_mma, phase, kSpin));
        if (!ok) break;
        mma_pending = false;
        phase ^= 1u;
        tc::fence_after_sync();

        // ---- output planes o0 < L0 back into G (in place: this unit's lines only)
        {
            float2 *g = cur.G + cur.line0 + erow;
#pragma unroll
            for (int cc = 0; cc < 2; ++cc) {
                float v[32];
                tc::tmem_ld32(tmem + (uint32_t(32 * quarter) << 16) + uint32_t(64 * half + 32 * cc), v);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int o0 = 32 * half + 16 * cc + j;
                    if (o0 < cur.L0) __stcg(g + int64_t(o0) * kPlane, make_float2(v[2 * j], v[2 * j + 1]));
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        cur = nxt;
    }
    if (!ok) {
        if (tid == 0) atomicExch(p.ctrl + 2, 1);
        // give an MMA still in flight a bounded chance to finish before the
        // tensor memory is released
        if (mma_pending) (void)__syncthreads_and(mbar_wait_bounded(bar_mma, phase, kSpin));
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 128);
}

uint16_t bf16_rn(float f) {
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return uint16_t(u >> 16);
}
float bf16_to_float(uint16_t h) {
    const uint32_t u = uint32_t(h) << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return f;
}

}  // namespace

// F1 hi, F1 lo, F2 hi, F2 lo in the shared-memory operand layout (128 KB)
cudaError_t tc3d_build_operands(void **d_ops) {
    std::vector<uint8_t> h(size_t(4) * kTile, 0);
    const long double two_pi = 6.283185307179586476925286766559005768L;
    auto put = [&](int mat, int n, int k, double v) {
        const uint16_t hi = bf16_rn(float(v));
        const uint16_t lo = bf16_rn(float(v - double(bf16_to_float(hi))));
        const uint32_t off = tc::kmajor_offset(n, k, kK, 2);
        std::memcpy(&h[size_t(2 * mat) * kTile + off], &hi, 2);
        std::memcpy(&h[size_t(2 * mat + 1) * kTile + off], &lo, 2);
    };
    for (int a = 0; a < kP; ++a)
        for (int b = 0; b < kP; ++b) {
            const int e = (a * b) % kP;
            const double cs = double(cosl(two_pi * e / kP)), sn = double(sinl(two_pi * e / kP));
            // F1: rows (k0 = a, re|im), columns (i0 = b, re|im): W^(i0 k0)
            put(0, 2 * a, 2 * b, cs);
            put(0, 2 * a, 2 * b + 1, sn);
            put(0, 2 * a + 1, 2 * b, -sn);
            put(0, 2 * a + 1, 2 * b + 1, cs);
            // F2: rows (o0 = a, re|im), columns (k0 = b, re|im): W^(-o0 k0)
            put(1, 2 * a, 2 * b, cs);
            put(1, 2 * a, 2 * b + 1, -sn);
            put(1, 2 * a + 1, 2 * b, sn);
            put(1, 2 * a + 1, 2 * b + 1, cs);
        }
    cudaError_t e = cudaMalloc(d_ops, h.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*d_ops, h.data(), h.size(), cudaMemcpyHostToDevice);
}

cudaError_t tc3d_configure() {
    return cudaFuncSetAttribute(tc3d_axis0_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
}

cudaError_t launch_tc3d_axis0(const ApplyParams &p, int ctas, void *scratch, int64_t c0, int64_t c1,
                              const void *ops, cudaStream_t s) {
    const int64_t units = (c1 - c0) * kUnitsPerItem;
    const int grid = int(std::min<int64_t>(ctas, units));
    tc3d_axis0_kernel<<<grid, kThreads, kSmem, s>>>(p, static_cast<float2 *>(scratch), c0, c1,
                                                    static_cast<const uint8_t *>(ops));
    return cudaGetLastError();
}

}  // namespace pc
