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
// F1 (K limited to k1cap = 16 ceil(2 T / 16) columns, T <= 48 the tile
// extent) and F2 are copied into shared memory once per CTA by the bulk-copy
// (TMA) engine; the data tiles are split and written by the threads; two D1
// accumulators and D2 live in 128-column blocks of tensor memory.  Two units
// are in flight: GEMM 1 of unit u+1 is issued as soon as GEMM 1 of unit u is
// done, so it runs while the threads do unit u's epilogue 1 (into the other
// D1); then GEMM 2 of unit u runs while they load unit u+2.
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
constexpr int kK = 2 * kP;                          // (index, re|im): K of GEMM 2, N of both
constexpr int kTile = kBlock * kK * 2;              // one BF16 128 x 128 operand tile: 32 KB
constexpr int kThreads = 512;
constexpr int kQuads = kThreads / kBlock;          // threads per line in staging, warps per lane quarter
constexpr uint32_t kLBO = 128u;                     // core matrices adjacent along K
constexpr uint32_t kSBO2 = uint32_t(kK * 2 / 16) * 128u;   // 8-row groups of a K = 128 tile: 2048 B
constexpr long long kSpin = 1ll << 24;
constexpr uint32_t kIdesc = tc::idesc_bf16(kBlock, kK);

// bytes of one BF16 128 x k operand tile (hi or lo)
__host__ __device__ constexpr int tile_bytes(int k) { return kBlock * k * 2; }
// shared layout: [F1 hi|lo (k1cap) | F2 hi|lo | A2 hi|lo | A1 hi|lo (k1cap) | 3 mbarriers, TMEM slot]
__host__ __device__ constexpr int smem_bytes(int k1cap) { return 4 * tile_bytes(k1cap) + 4 * kTile + 64; }

static_assert(smem_bytes(kTc3dMaxK1) <= 227 * 1024, "shared memory");
static_assert(tc::kmajor_offset(kBlock - 1, kK - 1, kK, 2) == kTile - 2, "tile layout");

// 8 consecutive K values of one row -> hi and lo 16-byte core-matrix rows
// (the lo tile follows the hi tile at `lo_off` bytes)
__device__ __forceinline__ void split8_store(uint8_t *hi_tile, int lo_off, uint32_t off, const float *v) {
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
    *reinterpret_cast<uint4 *>(hi_tile + lo_off + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// D (tensor memory) = A * B^T over `steps` K steps of 16, three split products
// each; A and B tiles have K_total = sbo / 16 columns (lo tile at lo_off)
__device__ __forceinline__ void issue_gemm(uint32_t d_tmem, const uint8_t *a_tile, const uint8_t *b_tile, int lo_off,
                                           uint32_t sbo, int steps) {
    const uint32_t a = smem_u32(a_tile), b = smem_u32(b_tile), lo = uint32_t(lo_off);
    for (int s = 0; s < steps; ++s) {
        const uint32_t o = 256u * uint32_t(s);
        const uint64_t ah = tc::smem_desc(a + o, kLBO, sbo), al = tc::smem_desc(a + lo + o, kLBO, sbo);
        const uint64_t bh = tc::smem_desc(b + o, kLBO, sbo), bl = tc::smem_desc(b + lo + o, kLBO, sbo);
        tc::mma<false>(d_tmem, al, bh, kIdesc, s > 0 ? 1u : 0u);
        tc::mma<false>(d_tmem, ah, bl, kIdesc, 1u);
        tc::mma<false>(d_tmem, ah, bh, kIdesc, 1u);
    }
}

// One unit: 128 consecutive (k2, k1) lines of one work item.  GEMM 1 reads
// rows_in planes (the n0 input planes; adjoint: the L0 output-box planes,
// those outside Omega read as zero), GEMM 2 keeps rows_out (L0; adjoint n0).
struct Unit {
    int line0, n0, L0, steps1, spec;
    int rows_in, rows_out, g0;   // g0: first-axis origin of the rows_in planes
    float2 *G;   // the item's scratch volume [plane][k2][k1]
};

// Units of a chunk: u -> block index blk = u / nitems, then the chunk's items
// in the host-built order order[c0 + r] (sorted by tile, then pair), so that
// consecutive units share the tile and block and with them the spectrum block.
// order[total_items + i] is the tile of item order[i], so that no unit walks
// the colour table.
template <bool ADJ = false>
__device__ __forceinline__ Unit unit_of(const ApplyParams &p, float2 *scratch, const int32_t *order, int64_t c0,
                                        int64_t nitems, int64_t u) {
    const int blk = int(u / nitems);
    const int64_t r = c0 + (u - int64_t(blk) * nitems);
    const int64_t item = order[r];
    const Tile &tile = p.tiles[order[p.total_items + r]];
    Unit x;
    x.n0 = tile.in_ext[0];
    x.L0 = x.n0 + tile.kext[0] - 1;
    x.rows_in = ADJ ? x.L0 : x.n0;
    x.rows_out = ADJ ? x.n0 : x.L0;
    x.g0 = tile.out_lo[0];
    x.steps1 = (2 * x.rows_in + 15) / 16;
    x.spec = tile.spec;
    x.G = scratch + (item - c0) * int64_t(kP) * kPlane;
    x.line0 = blk * kBlock;
    return x;
}

// GEMM-1 input of a unit: thread (m = tid % 128, h = tid / 128) holds groups
// g = h + 4 e (e < GROUPS, g < k1cap / 8) of 4 planes (8 K values) of line
// line0 + m.  All loads are issued before any is used.  CLIP: planes outside
// Omega along the first axis read as zero (the adjoint's phase 1 skips them).
constexpr int kGroups = kTc3dMaxK1 / 8 / kQuads;   // groups per thread (forward)
constexpr int kGroupsAdj = 2 * kP / 8 / kQuads;    // adjoint: K up to 2 P
static_assert(kGroups * kQuads * 8 == kTc3dMaxK1, "staging groups");
template <int GROUPS, bool CLIP>
__device__ __forceinline__ void stage_load(const ApplyParams &p, const Unit &x, int tid, float2 (&z)[4 * GROUPS]) {
    const int m = tid & (kBlock - 1), h = tid >> 7;
#pragma unroll
    for (int e = 0; e < GROUPS; ++e)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i0 = 4 * (h + kQuads * e) + q;
            const bool in = i0 < x.rows_in && (!CLIP || (x.g0 + i0 >= 0 && x.g0 + i0 < p.nx[0]));
            z[4 * e + q] = in ? __ldcg(x.G + int64_t(i0) * kPlane + x.line0 + m) : make_float2(0.f, 0.f);
        }
}

template <int GROUPS>
__device__ __forceinline__ void stage_store(const Unit &x, int tid, const float2 (&z)[4 * GROUPS], uint8_t *sA1,
                                            int k1cap) {
    const int m = tid & (kBlock - 1), h = tid >> 7;
#pragma unroll
    for (int e = 0; e < GROUPS; ++e) {
        const int g = h + kQuads * e;
        if (g < 2 * x.steps1) {
            float v[8];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                v[2 * q] = z[4 * e + q].x;
                v[2 * q + 1] = z[4 * e + q].y;
            }
            split8_store(sA1, tile_bytes(k1cap), tc::kmajor_offset(m, 8 * g, k1cap, 2), v);
        }
    }
}

// spectrum of the thread's line, k0 = 16 part ... 16 part + 15 (Hermitian
// mirror for k2 > P/2); conjugated for the adjoint
template <bool ADJ = false>
__device__ __forceinline__ void spectrum_load(const ApplyParams &p, const Unit &x, int erow, int part,
                                              float2 (&f)[16]) {
    const int line = x.line0 + erow, k2 = line / kP, k1 = line % kP;
    const bool mirror = k2 > kP / 2;
    const float2 *sp = static_cast<const float2 *>(p.spec) + int64_t(x.spec) * p.spec_stride +
                       (mirror ? (int64_t(kP - k2) * kP + ((kP - k1) & (kP - 1))) * kP : (int64_t(k2) * kP + k1) * kP);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int k0 = 16 * part + j;
        f[j] = __ldg(sp + (mirror ? ((kP - k0) & (kP - 1)) : k0));
        if (mirror != ADJ) f[j].y = -f[j].y;
    }
}

__global__ void __launch_bounds__(kThreads, 1) tc3d_axis0_kernel(const ApplyParams p, float2 *scratch,
                                                                 const int32_t *order, int64_t c0, int64_t c1,
                                                                 const uint8_t *ops, int k1cap) {
    extern __shared__ __align__(1024) uint8_t sm[];
    const int t1 = tile_bytes(k1cap);
    uint8_t *sF1 = sm, *sF2 = sm + 2 * t1, *sA2 = sF2 + 2 * kTile, *sA1 = sA2 + 2 * kTile;
    uint64_t *bar_ld = reinterpret_cast<uint64_t *>(sA1 + 2 * t1);
    uint64_t *bar_g1 = bar_ld + 1, *bar_g2 = bar_ld + 2;
    uint32_t *slot = reinterpret_cast<uint32_t *>(bar_ld + 3);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t nitems = c1 - c0;
    // this CTA's contiguous range of units
    const int64_t u_begin = nitems * kUnitsPerItem * blockIdx.x / gridDim.x;
    const int64_t nunits = nitems * kUnitsPerItem * (blockIdx.x + 1) / gridDim.x;
    const int64_t stride = 1;
    const uint32_t sbo1 = uint32_t(k1cap) * 16u;
    const int steps2 = kK / 16;

    if (tid == 0) {
        mbar_init(bar_ld, 1);
        mbar_init(bar_g1, 1);
        mbar_init(bar_g2, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(slot, 512);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    // two D1 accumulators (GEMM 1 of the next unit runs while this unit's
    // epilogue 1 reads its own), one D2
    const uint32_t d2 = tmem + 256u;
    if (tid == 0) {
        mbar_arrive_expect_tx(bar_ld, uint32_t(2 * t1 + 2 * kTile));
        bulk_g2s(sF1, ops, uint32_t(2 * t1), bar_ld);
        bulk_g2s(sF2, ops + 2 * t1, uint32_t(2 * kTile), bar_ld);
    }
    // epilogue roles: warp w reads tensor-memory lanes 32 (w % 4) ... (its 32
    // lines) and the column quarter w / 4 (frequencies 16 (w / 4) ...)
    const int quarter = warp & 3, part = warp >> 2;
    const int erow = 32 * quarter + lane;
    const uint32_t lane_base = uint32_t(32 * quarter) << 16;

    float2 z[4 * kGroups];   // GEMM-1 input of the next unit to be staged
    float2 f[16];            // spectrum of the unit whose epilogue 1 is next
    int64_t u = u_begin;
    Unit cur{}, nxt{};
    if (u < nunits) {
        cur = unit_of(p, scratch, order, c0, nitems, u);
        stage_load<kGroups, false>(p, cur, tid, z);
    }
    bool ok = __syncthreads_and(mbar_wait_bounded(bar_ld, 0, kSpin));
    bool pend1 = false, pend2 = false;
    uint32_t ph1 = 0, ph2 = 0;
    int kb = 0;   // D1 buffer of `cur`
    if (ok && u < nunits) {
        stage_store<kGroups>(cur, tid, z, sA1, k1cap);
        fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            issue_gemm(tmem, sA1, sF1, t1, sbo1, cur.steps1);
            tc::mma_commit(bar_g1);
        }
        pend1 = true;
        if (u + stride < nunits) {
            nxt = unit_of(p, scratch, order, c0, nitems, u + stride);
            stage_load<kGroups, false>(p, nxt, tid, z);
        }
        spectrum_load(p, cur, erow, part, f);
    }
    for (; ok && u < nunits; u += stride) {
        // the unit after the next one: its table entries load meanwhile
        Unit nn = nxt;
        const bool has_next = u + stride < nunits, has_nn = u + 2 * stride < nunits;
        if (has_nn) nn = unit_of(p, scratch, order, c0, nitems, u + 2 * stride);
        const uint32_t d1 = tmem + 128u * uint32_t(kb);
        ok = __syncthreads_and(mbar_wait_bounded(bar_g1, ph1, kSpin));
        if (!ok) break;
        pend1 = false;
        ph1 ^= 1u;
        tc::fence_after_sync();
        // ---- GEMM 1 of the next unit first (A1 is free: GEMM 1 of `cur` is
        // done; it writes the other D1), so it runs during epilogue 1
        if (has_next) {
            stage_store<kGroups>(nxt, tid, z, sA1, k1cap);
            fence_proxy_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            if (tid == 0) {
                tc::fence_after_sync();
                issue_gemm(tmem + 128u * uint32_t(kb ^ 1), sA1, sF1, t1, sbo1, nxt.steps1);
                tc::mma_commit(bar_g1);
            }
            pend1 = true;
        }
        // ---- epilogue 1 of `cur`: V^ = D1 * phi^, split into A2 (free: GEMM 2
        // of the previous unit is done)
        {
            float v[32];
            tc::tmem_ld32(d1 + lane_base + uint32_t(32 * part), v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float2 w = f[j];
                const float re = v[2 * j] * w.x - v[2 * j + 1] * w.y;
                const float im = v[2 * j] * w.y + v[2 * j + 1] * w.x;
                v[2 * j] = re;
                v[2 * j + 1] = im;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
                split8_store(sA2, kTile, tc::kmajor_offset(erow, 32 * part + 8 * r, kK, 2), v + 8 * r);
        }
        fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            issue_gemm(d2, sA2, sF2, kTile, kSBO2, steps2);
            tc::mma_commit(bar_g2);
        }
        pend2 = true;
        if (has_nn) stage_load<kGroups, false>(p, nn, tid, z);
        // the spectrum registers stay valid while the tile and block repeat
        if (has_next && (nxt.spec != cur.spec || nxt.line0 != cur.line0)) spectrum_load(p, nxt, erow, part, f);

        // ---- epilogue 2 of `cur`: output planes o0 < L0 back into G (in
        // place: this unit's lines only)
        ok = __syncthreads_and(mbar_wait_bounded(bar_g2, ph2, kSpin));
        if (!ok) break;
        pend2 = false;
        ph2 ^= 1u;
        tc::fence_after_sync();
        {
            float2 *g = cur.G + cur.line0 + erow;
            float v[32];
            tc::tmem_ld32(d2 + lane_base + uint32_t(32 * part), v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int o0 = 16 * part + j;
                if (o0 < cur.rows_out) __stcg(g + int64_t(o0) * kPlane, make_float2(v[2 * j], v[2 * j + 1]));
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        cur = nxt;
        nxt = nn;
        kb ^= 1;
    }
    if (!ok) {
        if (tid == 0) atomicExch(p.ctrl + 2, 1);
        // give MMAs still in flight a bounded chance to finish before the
        // tensor memory is released
        if (pend1) (void)__syncthreads_and(mbar_wait_bounded(bar_g1, ph1, kSpin));
        if (pend2) (void)__syncthreads_and(mbar_wait_bounded(bar_g2, ph2, kSpin));
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// The adjoint (Eq. adjoint_random_z): GEMM 1 takes the L0 output-box planes
// (K = 2 L0 <= 2 P, so F1 is the whole DFT matrix), the product takes the
// conjugate spectrum, and GEMM 2 keeps the n0 input-box planes.  With F1 of
// K = 128 the two data tiles no longer fit beside F1 and F2, so GEMM 1 and
// GEMM 2 share one data tile and a unit runs its steps one after another:
// stage, GEMM 1, epilogue 1 (into the same tile, which GEMM 1 has finished
// reading), GEMM 2, epilogue 2.  The next unit's loads are in flight meanwhile.
__host__ __device__ constexpr int smem_bytes_adj() { return 2 * tile_bytes(2 * kP) + 2 * kTile + 2 * kTile + 64; }
static_assert(smem_bytes_adj() <= 227 * 1024, "shared memory");

__global__ void __launch_bounds__(kThreads, 1) tc3d_axis0_adj_kernel(const ApplyParams p, float2 *scratch,
                                                                     const int32_t *order, int64_t c0, int64_t c1,
                                                                     const uint8_t *ops) {
    extern __shared__ __align__(1024) uint8_t sm[];
    constexpr int K1 = 2 * kP;
    constexpr int t1 = tile_bytes(K1);
    uint8_t *sF1 = sm, *sF2 = sm + 2 * t1, *sA = sF2 + 2 * kTile;
    uint64_t *bar_ld = reinterpret_cast<uint64_t *>(sA + 2 * kTile);
    uint64_t *bar_g1 = bar_ld + 1, *bar_g2 = bar_ld + 2;
    uint32_t *slot = reinterpret_cast<uint32_t *>(bar_ld + 3);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t nitems = c1 - c0;
    const int64_t u_begin = nitems * kUnitsPerItem * blockIdx.x / gridDim.x;
    const int64_t nunits = nitems * kUnitsPerItem * (blockIdx.x + 1) / gridDim.x;
    const uint32_t sbo1 = uint32_t(K1) * 16u;
    const int steps2 = kK / 16;

    if (tid == 0) {
        mbar_init(bar_ld, 1);
        mbar_init(bar_g1, 1);
        mbar_init(bar_g2, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(slot, 256);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *slot;
    const uint32_t d1 = tmem, d2 = tmem + 128u;
    if (tid == 0) {
        mbar_arrive_expect_tx(bar_ld, uint32_t(2 * t1 + 2 * kTile));
        bulk_g2s(sF1, ops, uint32_t(2 * t1), bar_ld);
        bulk_g2s(sF2, ops + 2 * t1, uint32_t(2 * kTile), bar_ld);
    }
    const int quarter = warp & 3, part = warp >> 2;
    const int erow = 32 * quarter + lane;
    const uint32_t lane_base = uint32_t(32 * quarter) << 16;

    float2 z[4 * kGroupsAdj];   // GEMM-1 input of the next unit to be staged
    float2 f[16];               // spectrum of the current unit
    Unit cur{};
    int spec_of_f = -1, line_of_f = -1;
    if (u_begin < nunits) {
        cur = unit_of<true>(p, scratch, order, c0, nitems, u_begin);
        stage_load<kGroupsAdj, true>(p, cur, tid, z);
    }
    bool ok = __syncthreads_and(mbar_wait_bounded(bar_ld, 0, kSpin));
    bool pend1 = false, pend2 = false;
    uint32_t ph1 = 0, ph2 = 0;
    for (int64_t u = u_begin; ok && u < nunits; ++u) {
        // ---- stage (the data tile is free: the previous GEMM 2 has completed)
        stage_store<kGroupsAdj>(cur, tid, z, sA, K1);
        fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            issue_gemm(d1, sA, sF1, t1, sbo1, cur.steps1);
            tc::mma_commit(bar_g1);
        }
        pend1 = true;
        // the next unit's loads and this unit's spectrum while GEMM 1 runs
        Unit nxt = cur;
        if (u + 1 < nunits) {
            nxt = unit_of<true>(p, scratch, order, c0, nitems, u + 1);
            stage_load<kGroupsAdj, true>(p, nxt, tid, z);
        }
        if (cur.spec != spec_of_f || cur.line0 != line_of_f) {
            spectrum_load<true>(p, cur, erow, part, f);
            spec_of_f = cur.spec;
            line_of_f = cur.line0;
        }
        // ---- epilogue 1: V^ = D1 * conj(phi^), split into the data tile
        ok = __syncthreads_and(mbar_wait_bounded(bar_g1, ph1, kSpin));
        if (!ok) break;
        pend1 = false;
        ph1 ^= 1u;
        tc::fence_after_sync();
        {
            float v[32];
            tc::tmem_ld32(d1 + lane_base + uint32_t(32 * part), v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float2 w = f[j];
                const float re = v[2 * j] * w.x - v[2 * j + 1] * w.y;
                const float im = v[2 * j] * w.y + v[2 * j + 1] * w.x;
                v[2 * j] = re;
                v[2 * j + 1] = im;
            }
#pragma unroll
            for (int r = 0; r < 4; ++r)
                split8_store(sA, kTile, tc::kmajor_offset(erow, 32 * part + 8 * r, kK, 2), v + 8 * r);
        }
        fence_proxy_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            issue_gemm(d2, sA, sF2, kTile, kSBO2, steps2);
            tc::mma_commit(bar_g2);
        }
        pend2 = true;
        // ---- epilogue 2: the n0 input-box planes back into G (in place)
        ok = __syncthreads_and(mbar_wait_bounded(bar_g2, ph2, kSpin));
        if (!ok) break;
        pend2 = false;
        ph2 ^= 1u;
        tc::fence_after_sync();
        {
            float2 *g = cur.G + cur.line0 + erow;
            float v[32];
            tc::tmem_ld32(d2 + lane_base + uint32_t(32 * part), v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int o0 = 16 * part + j;
                if (o0 < cur.rows_out) __stcg(g + int64_t(o0) * kPlane, make_float2(v[2 * j], v[2 * j + 1]));
            }
        }
        tc::fence_before_sync();
        __syncthreads();
        cur = nxt;
    }
    if (!ok) {
        if (tid == 0) atomicExch(p.ctrl + 2, 1);
        if (pend1) (void)__syncthreads_and(mbar_wait_bounded(bar_g1, ph1, kSpin));
        if (pend2) (void)__syncthreads_and(mbar_wait_bounded(bar_g2, ph2, kSpin));
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 256);
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

int tc3d_k1cap(int tile) { return 16 * ((2 * tile + 15) / 16); }

// F1 hi, F1 lo (K = k1cap), F2 hi, F2 lo in the shared-memory operand layout
cudaError_t tc3d_build_operands(int k1cap, void **d_ops) {
    if (k1cap < 16 || k1cap > 2 * kP || k1cap % 16) return cudaErrorInvalidValue;
    const int t1 = tile_bytes(k1cap);
    std::vector<uint8_t> h(size_t(2 * t1 + 2 * kTile), 0);
    const long double two_pi = 6.283185307179586476925286766559005768L;
    auto put = [&](size_t base, int tb, int ktot, int n, int k, double v) {
        const uint16_t hi = bf16_rn(float(v));
        const uint16_t lo = bf16_rn(float(v - double(bf16_to_float(hi))));
        const uint32_t off = tc::kmajor_offset(n, k, ktot, 2);
        std::memcpy(&h[base + off], &hi, 2);
        std::memcpy(&h[base + size_t(tb) + off], &lo, 2);
    };
    for (int a = 0; a < kP; ++a)
        for (int b = 0; b < kP; ++b) {
            const int e = (a * b) % kP;
            const double cs = double(cosl(two_pi * e / kP)), sn = double(sinl(two_pi * e / kP));
            // F1: rows (k0 = a, re|im), columns (i0 = b, re|im): W^(i0 k0)
            if (2 * b + 1 < k1cap) {
                put(0, t1, k1cap, 2 * a, 2 * b, cs);
                put(0, t1, k1cap, 2 * a, 2 * b + 1, sn);
                put(0, t1, k1cap, 2 * a + 1, 2 * b, -sn);
                put(0, t1, k1cap, 2 * a + 1, 2 * b + 1, cs);
            }
            // F2: rows (o0 = a, re|im), columns (k0 = b, re|im): W^(-o0 k0)
            const size_t f2 = size_t(2 * t1);
            put(f2, kTile, kK, 2 * a, 2 * b, cs);
            put(f2, kTile, kK, 2 * a, 2 * b + 1, -sn);
            put(f2, kTile, kK, 2 * a + 1, 2 * b, sn);
            put(f2, kTile, kK, 2 * a + 1, 2 * b + 1, cs);
        }
    cudaError_t e = cudaMalloc(d_ops, h.size());
    if (e != cudaSuccess) return e;
    return cudaMemcpy(*d_ops, h.data(), h.size(), cudaMemcpyHostToDevice);
}

cudaError_t tc3d_configure() {
    cudaError_t e =
        cudaFuncSetAttribute(tc3d_axis0_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes(kTc3dMaxK1));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(tc3d_axis0_adj_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes_adj());
    return e;
}

cudaError_t launch_tc3d_axis0(const ApplyParams &p, int ctas, void *scratch, const int32_t *order, int64_t c0,
                              int64_t c1, const void *ops, int k1cap, cudaStream_t s) {
    if (k1cap < 16 || k1cap > kTc3dMaxK1 || k1cap % 16) return cudaErrorInvalidValue;
    const int64_t units = (c1 - c0) * kUnitsPerItem;
    const int grid = int(std::min<int64_t>(ctas, units));
    tc3d_axis0_kernel<<<grid, kThreads, smem_bytes(k1cap), s>>>(p, static_cast<float2 *>(scratch), order, c0, c1,
                                                                static_cast<const uint8_t *>(ops), k1cap);
    return cudaGetLastError();
}

cudaError_t launch_tc3d_axis0_adjoint(const ApplyParams &p, int ctas, void *scratch, const int32_t *order, int64_t c0,
                                      int64_t c1, const void *ops_full, cudaStream_t s) {
    const int64_t units = (c1 - c0) * kUnitsPerItem;
    const int grid = int(std::min<int64_t>(ctas, units));
    tc3d_axis0_adj_kernel<<<grid, kThreads, smem_bytes_adj(), s>>>(p, static_cast<float2 *>(scratch), order, c0, c1,
                                                                   static_cast<const uint8_t *>(ops_full));
    return cudaGetLastError();
}

}  // namespace pc
