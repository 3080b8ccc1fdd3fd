// Register/shared-memory FFT building blocks for the fused patch kernels.
//
// A line FFT of length P = R1 * R2 is computed by R2 cooperating threads
// ("a line"), thread t holding the R1 values x[t + R2*j], j < R1:
//
//   X[m + R1*q] = sum_t W_R2^{t q} ( W_P^{t m} sum_j x[t + R2 j] W_R1^{j m} )
//
// step 1: a length-R1 DFT in registers over j, step 2: the twiddle W_P^{t m},
// step 3: a transpose through shared memory so that thread t owns the
// R1/R2 residues m = t + R2*e, step 4: length-R2 DFTs in registers over t.
// The result X[k] lands in thread t, register j', with k = t + R2*j', i.e.
// the same strided layout as the input, so forward and inverse transforms
// chain without extra data movement.  The inverse transform uses conjugate
// twiddles and no scaling (1/P^d is folded into the stored spectra).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace pc {

template <typename T> struct Cx;
template <> struct Cx<float> { using type = float2; };
template <> struct Cx<double> { using type = double2; };

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return C{a.x + b.x, a.y + b.y}; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return C{a.x - b.x, a.y - b.y}; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {  // a * conj(b)
    return C{a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}

// Butterfly sum and difference.  For FP32 both components go through one
// packed two-lane instruction (add/sub.rn.f32x2, round-to-nearest per lane,
// the same result as two scalar operations); FP64 stays scalar.
template <typename C> __device__ __forceinline__ C badd(C a, C b) { return cadd(a, b); }
template <typename C> __device__ __forceinline__ C bsub(C a, C b) { return csub(a, b); }
template <> __device__ __forceinline__ float2 badd<float2>(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "add.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}
template <> __device__ __forceinline__ float2 bsub<float2>(float2 a, float2 b) {
    float2 r;
    asm("{\n\t.reg .b64 pa, pb, pr;\n\tmov.b64 pa, {%2, %3};\n\tmov.b64 pb, {%4, %5};\n\t"
        "sub.rn.f32x2 pr, pa, pb;\n\tmov.b64 {%0, %1}, pr;\n\t}"
        : "=f"(r.x), "=f"(r.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return r;
}

// cos and sin of 2*pi*e/16 for e = 0..15 (exact values of the regular
// 16-gon: cos(pi/8) = sqrt(2 + sqrt 2)/2, sin(pi/8) = sqrt(2 - sqrt 2)/2).
__host__ __device__ constexpr double kC16(int e) {
    return e == 0 ? 1.0 : e == 1 ? 0.92387953251128675613 : e == 2 ? 0.70710678118654752440
         : e == 3 ? 0.38268343236508977173 : e == 4 ? 0.0 : e == 5 ? -0.38268343236508977173
         : e == 6 ? -0.70710678118654752440 : e == 7 ? -0.92387953251128675613 : e == 8 ? -1.0
         : e == 9 ? -0.92387953251128675613 : e == 10 ? -0.70710678118654752440
         : e == 11 ? -0.38268343236508977173 : e == 12 ? 0.0 : e == 13 ? 0.38268343236508977173
         : e == 14 ? 0.70710678118654752440 : 0.92387953251128675613;
}
__host__ __device__ constexpr double kS16(int e) { return kC16((e + 12) & 15); }  // sin x = cos(x - pi/2)

// v * W_16^e (forward: W = exp(-2 pi i e / 16)) or v * conj(W_16^e) (inverse)
template <int E, bool INV, typename C>
__device__ __forceinline__ C tw16(C v) {
    using T = decltype(v.x);
    constexpr int e = E & 15;
    if constexpr (e == 0) {
        return v;
    } else if constexpr (e == 8) {
        return C{-v.x, -v.y};
    } else if constexpr (e == 4) {
        return INV ? C{-v.y, v.x} : C{v.y, -v.x};
    } else if constexpr (e == 12) {
        return INV ? C{v.y, -v.x} : C{-v.y, v.x};
    } else {
        constexpr T c = T(kC16(e));
        constexpr T s = INV ? T(-kS16(e)) : T(kS16(e));
        // (x + i y)(c - i s) = (x c + y s) + i (y c - x s)
        return C{v.x * c + v.y * s, v.y * c - v.x * s};
    }
}

__host__ __device__ constexpr int bitrev(int i, int n) {
    int r = 0;
    for (int b = 1; b < n; b <<= 1) r = (r << 1) | ((i & b) ? 1 : 0);
    return r;
}

// In-register radix-2 DIT DFT of length N (N = 2, 4, 8, 16), natural order
// in and out.  Every register index is a template constant, so the arrays
// stay in registers.
template <int N, int I, typename C>
__device__ __forceinline__ void bitrev_perm(C *a) {
    if constexpr (I < N) {
        constexpr int J = bitrev(I, N);
        if constexpr (J > I) {
            C t = a[I];
            a[I] = a[J];
            a[J] = t;
        }
        bitrev_perm<N, I + 1>(a);
    }
}

// butterfly B (< N/2) of the stage that merges blocks of length LEN/2
template <int N, bool INV, int LEN, int B, typename C>
__device__ __forceinline__ void dit_stage(C *a) {
    if constexpr (B < N / 2) {
        constexpr int half = LEN / 2, blk = B / half, k = B % half;
        constexpr int i0 = blk * LEN + k, i1 = i0 + half;
        constexpr int e = (k * (16 / LEN)) & 15;   // W_LEN^k = W_16^(16k/LEN)
        const C u = a[i0];
        if constexpr (e == 4 || e == 12) {
            // +-i: a swap of components, cheaper as scalar operations
            const C v = tw16<e, INV>(a[i1]);
            a[i0] = cadd(u, v);
            a[i1] = csub(u, v);
        } else {
            const C v = tw16<e, INV>(a[i1]);
            a[i0] = badd(u, v);
            a[i1] = bsub(u, v);
        }
        dit_stage<N, INV, LEN, B + 1>(a);
    }
}

template <int N, bool INV, int LEN, typename C>
__device__ __forceinline__ void dit_stages(C *a) {
    if constexpr (LEN <= N) {
        dit_stage<N, INV, LEN, 0>(a);
        dit_stages<N, INV, 2 * LEN>(a);
    }
}

template <int N, bool INV, typename C>
__device__ __forceinline__ void dft_reg(C *a) {
    static_assert(N >= 2 && N <= 16 && (N & (N - 1)) == 0, "register DFT length");
    bitrev_perm<N, 0>(a);
    dit_stages<N, INV, 2>(a);
}

// Swizzle of the column index inside a shared-memory row so that strided
// column walks, row walks and the line transposes are free of bank conflicts
// for 8-byte elements with 8 threads per line.
__device__ __forceinline__ int swz(int row) {
    const int u = row & 7;
    return 2 * (u ^ ((u & 1) << 2));
}

template <int P> struct FftShape {
    static constexpr int R2 = (P >= 256) ? 16 : 8;   // threads per line
    static constexpr int R1 = P / R2;                 // values per thread
    static_assert(R1 >= R2 && R1 % R2 == 0, "unsupported line FFT shape");
    // lanes of the calling thread's line within its warp
    static __device__ __forceinline__ unsigned line_mask() {
        return ((1u << R2) - 1u) << ((threadIdx.x & 31) & ~(R2 - 1));
    }
};

// One line FFT.  `a` holds x[t + R2 j]; `tw` holds W_P^{t m} for m < R1;
// Scratch holds P slots private to the line: st_m(m, t, v) stores register m
// of thread t at slot m R2 + (t ^ (m mod R2)) and ld_e(e, t2, t) loads slot
// (t + R2 e) R2 + (t2 ^ t), the value thread t2 stored as register t + R2 e
// (the transpose of step 3).  `mask` names the line's lanes (lines of one
// warp may diverge).  On return a[j'] = X[t + R2 j'].
template <int P, bool INV, typename C, typename Scratch>
__device__ __forceinline__ void fft_line(C *a, const C *tw, int t, Scratch &scr, unsigned mask) {
    constexpr int R1 = FftShape<P>::R1, R2 = FftShape<P>::R2, E = R1 / R2;
    dft_reg<R1, INV>(a);
#pragma unroll
    for (int m = 1; m < R1; ++m) a[m] = INV ? cmulc(a[m], tw[m]) : cmul(a[m], tw[m]);
    // the scratch may be the storage the line just read its input from
    __syncwarp(mask);
#pragma unroll
    for (int m = 0; m < R1; ++m) scr.st_m(m, t, a[m]);
    __syncwarp(mask);
#pragma unroll
    for (int e = 0; e < E; ++e)
#pragma unroll
        for (int t2 = 0; t2 < R2; ++t2) a[e * R2 + t2] = scr.ld_e(e, t2, t);
    __syncwarp(mask);
    C b[R1];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        dft_reg<R2, INV>(a + e * R2);
#pragma unroll
        for (int q = 0; q < R2; ++q) b[e + E * q] = a[e * R2 + q];
    }
#pragma unroll
    for (int j = 0; j < R1; ++j) a[j] = b[j];
}

// Line scratch inside a P x P shared workspace laid out row * P + (col ^ swz(row)):
// a row, or a column (positions are then row indices).
template <int P, typename C> struct RowScratch {
    static constexpr int R2 = FftShape<P>::R2;
    C *S;
    int row;
    __device__ __forceinline__ C ld(int s) const { return S[row * P + (s ^ swz(row))]; }
    __device__ __forceinline__ void st(int s, C v) const { S[row * P + (s ^ swz(row))] = v; }
    __device__ __forceinline__ void st_m(int m, int t, C v) const { st(m * R2 + (t ^ (m & (R2 - 1))), v); }
    __device__ __forceinline__ C ld_e(int e, int t2, int t) const { return ld((t + R2 * e) * R2 + (t2 ^ t)); }
};
template <int P, typename C> struct ColScratch {
    static constexpr int R2 = FftShape<P>::R2;
    C *S;
    int col;
    __device__ __forceinline__ C ld(int s) const { return S[s * P + (col ^ swz(s))]; }
    __device__ __forceinline__ void st(int s, C v) const { S[s * P + (col ^ swz(s))] = v; }
    __device__ __forceinline__ void st_m(int m, int t, C v) const { st(m * R2 + (t ^ (m & (R2 - 1))), v); }
    __device__ __forceinline__ C ld_e(int e, int t2, int t) const { return ld((t + R2 * e) * R2 + (t2 ^ t)); }
};

// Padded workspace of the 2D patch kernel: element (r, c) of a P x P complex
// field sits at r * pitch + c + pad_shift(r), pitch = P + 8.  A pitch of 8
// mod 16 eight-byte units puts consecutive rows in opposite halves of the
// banks, and the shift (r mod 8) / 2 spreads the 8 rows r = 8u + x (x < 8)
// that a column walk or a column transpose touches at once over distinct
// banks.  Unlike a swizzle, every address is a per-thread base plus a
// compile-time offset.
template <int P> struct PadLayout {
    static constexpr int pitch = P + 8;
};
__device__ __forceinline__ int pad_shift(int r) { return (r & 7) >> 1; }

// Line scratch in the padded workspace, for R2 = 8 threads per line: slot
// s = 8 u + x lives at base + u * A + x * B (+ pad_shift(x) for a column,
// whose slots are rows).  q[c] is the address of slot x = t ^ c of group 0, so
// the transpose's stores and loads are q[c] plus compile-time offsets.
//   row r:     base = &ws[r * pitch + pad_shift(r)], A = 8,         B = 1
//   column c:  base = &ws[c],                        A = 8 * pitch, B = pitch
template <int P, typename C, bool COL> struct PadScratch {
    static constexpr int R2 = FftShape<P>::R2;
    static_assert(R2 == 8, "padded line scratch assumes 8 threads per line");
    static constexpr int A = COL ? 8 * PadLayout<P>::pitch : 8;
    static constexpr int B = COL ? PadLayout<P>::pitch : 1;
    C *q[8];
    int tA;
    __device__ __forceinline__ PadScratch(C *base, int t) : tA(t * A) {
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            const int x = t ^ c;
            q[c] = base + x * B + (COL ? (x >> 1) : 0);
        }
    }
    // slot m * 8 + (t ^ (m mod 8)): group m, x = t ^ (m mod 8)
    __device__ __forceinline__ void st_m(int m, int, C v) const { q[m & 7][m * A] = v; }
    // slot (t + 8 e) * 8 + (t2 ^ t): group t + 8 e, x = t ^ t2
    __device__ __forceinline__ C ld_e(int e, int t2, int) const { return q[t2][tA + 8 * e * A]; }
};

}  // namespace pc
