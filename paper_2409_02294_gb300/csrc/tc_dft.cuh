// Radix-16 DFT stages on tensor cores with split-precision operands.
//
// A 16-point DFT applied to 8 lines at once is the complex matrix product
// Y = F X with F[k][r] = W_16^{kr} (16 x 16) and X (16 x 8).  In real form,
//   Yr = Fr Xr - Fi Xi,   Yi = Fi Xr + Fr Xi,
// i.e. four real m16n8k16 products.  Each FP32 operand v is split into
// v = hi + lo with hi = round16(v) and lo = round16(v - hi) (FP16 or BF16), and
// every real product is evaluated as Ahi Bhi + Ahi Blo + Alo Bhi (the lo*lo term
// is below the FP32 rounding of the result for FP16, ~2^-16 for BF16),
// accumulated in FP32: 12 mma.sync per group of 8 lines.  The DFT matrix's
// hi/lo fragments are fixed per lane and kept in registers.
//
// Each group's operands are scaled by a power of two (exact) that brings the
// largest magnitude to ~2^14 before the split, and the results are scaled
// back.  FP16 needs it for its narrow exponent range; BF16 shares FP32's
// range, but without it the lo parts of small values (and their products)
// fall below FP32's normal range and are lost when the whole field is tiny
// (a field scaled by 1e-30 lost 1e-4 of max|Phi| that way).
//
// Fragment layouts (PTX m16n8k16, g = lane / 4, c = lane % 4):
//   A (16x16, row):  a0 = A[g][2c..2c+1]   a1 = A[g+8][2c..2c+1]
//                    a2 = A[g][2c+8..9]    a3 = A[g+8][2c+8..9]
//   B (16x8, col):   b0 = B[2c..2c+1][g]   b1 = B[2c+8..9][g]
//   D (16x8, f32):   d0 = D[g][2c] d1 = D[g][2c+1] d2 = D[g+8][2c] d3 = D[g+8][2c+1]
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "fft_core.cuh"

namespace pgb {

// cos(2 pi e / 16), e = 0..15, from the exact constant table
__constant__ float c_cos16[16] = {
    1.0f, (float)cos96(6), (float)cos96(12), (float)cos96(18), 0.0f, -(float)cos96(18),
    -(float)cos96(12), -(float)cos96(6), -1.0f, -(float)cos96(6), -(float)cos96(12), -(float)cos96(18),
    0.0f, (float)cos96(18), (float)cos96(12), (float)cos96(6)};
__device__ __forceinline__ float cos16_tab(int e) { return c_cos16[e & 15]; }
__device__ __forceinline__ float sin16_tab(int e) { return c_cos16[(e - 4) & 15]; }

template <bool BF16> __device__ __forceinline__ uint32_t pack2(float x, float y) {
    if constexpr (BF16) {
        __nv_bfloat162 h = __floats2bfloat162_rn(x, y);
        return *reinterpret_cast<uint32_t*>(&h);
    } else {
        __half2 h = __floats2half2_rn(x, y);
        return *reinterpret_cast<uint32_t*>(&h);
    }
}
template <bool BF16> __device__ __forceinline__ float2 unpack2(uint32_t v) {
    if constexpr (BF16) {
        return __bfloat1622float2(*reinterpret_cast<__nv_bfloat162*>(&v));
    } else {
        return __half22float2(*reinterpret_cast<__half2*>(&v));
    }
}
// (x, y) -> hi, lo with x = hi.x + lo.x etc. to 2 x 11 (FP16) or 2 x 8 (BF16) bits
template <bool BF16> __device__ __forceinline__ void split2(float x, float y, uint32_t& hi, uint32_t& lo) {
    hi = pack2<BF16>(x, y);
    const float2 h = unpack2<BF16>(hi);
    lo = pack2<BF16>(x - h.x, y - h.y);
}

template <bool BF16>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    if constexpr (BF16) {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
            "{%8,%9}, {%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    } else {
        asm volatile(
            "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
            "{%8,%9}, {%0,%1,%2,%3};\n"
            : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
            : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
    }
}

// Per-lane fragments of the 16-point DFT matrix: real part C, imaginary part
// S (forward sign: W = C + i S with S = -sin) and -S, each as hi and lo.
template <bool BF16> struct Dft16Frags {
    uint32_t c_hi[4], c_lo[4], s_hi[4], s_lo[4], ns_hi[4], ns_lo[4];
    __device__ __forceinline__ void init(int lane) {
        const int g = lane >> 2, c = lane & 3;
        const int rows[4] = {g, g + 8, g, g + 8};
        const int cols[4] = {2 * c, 2 * c, 2 * c + 8, 2 * c + 8};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int e0 = rows[i] * cols[i], e1 = rows[i] * (cols[i] + 1);
            const float c0 = cos16_tab(e0), c1 = cos16_tab(e1);
            const float s0 = -sin16_tab(e0), s1 = -sin16_tab(e1);
            split2<BF16>(c0, c1, c_hi[i], c_lo[i]);
            split2<BF16>(s0, s1, s_hi[i], s_lo[i]);
            split2<BF16>(-s0, -s1, ns_hi[i], ns_lo[i]);
        }
    }
};

// One radix-16 DFT of 8 lines on tensor cores.  Input: this lane's B
// fragment values br[0..3] / bi[0..3] = X[r][g] for r = 2c, 2c+1, 2c+8, 2c+9
// (FP32).  Output: dr/di = Y[k][n] for (k, n) = (g, 2c), (g, 2c+1),
// (g+8, 2c), (g+8, 2c+1).  INV uses conj(F) (F is symmetric).
template <bool BF16, bool INV>
__device__ __forceinline__ void dft16_tc(const Dft16Frags<BF16>& F, const float (&br)[4], const float (&bi)[4],
                                         float (&dr)[4], float (&di)[4]) {
    // scale the group so that its largest magnitude is about 2^14
    float s = 1.0f, inv_s = 1.0f;
    {
        float m = 0.0f;
#pragma unroll
        for (int i = 0; i < 4; ++i) m = fmaxf(m, fmaxf(fabsf(br[i]), fabsf(bi[i])));
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, off));
        if (m > 0.0f) {
            const int e = (int)((__float_as_uint(m) >> 23) & 0xff) - 127;  // m in [2^e, 2^(e+1))
            const int k = max(-120, min(120, 13 - e));
            s = __uint_as_float((uint32_t)(127 + k) << 23);
            inv_s = __uint_as_float((uint32_t)(127 - k) << 23);
        }
    }
    uint32_t xr_hi0, xr_lo0, xr_hi1, xr_lo1, xi_hi0, xi_lo0, xi_hi1, xi_lo1;
    split2<BF16>(br[0] * s, br[1] * s, xr_hi0, xr_lo0);
    split2<BF16>(br[2] * s, br[3] * s, xr_hi1, xr_lo1);
    split2<BF16>(bi[0] * s, bi[1] * s, xi_hi0, xi_lo0);
    split2<BF16>(bi[2] * s, bi[3] * s, xi_hi1, xi_lo1);
    // forward: Yr = C Xr + (-S) Xi, Yi = S Xr + C Xi
    // inverse (conj F = C - iS): Yr = C Xr + S Xi, Yi = (-S) Xr + C Xi
    const uint32_t(&pr_hi)[4] = INV ? F.s_hi : F.ns_hi;
    const uint32_t(&pr_lo)[4] = INV ? F.s_lo : F.ns_lo;
    const uint32_t(&pi_hi)[4] = INV ? F.ns_hi : F.s_hi;
    const uint32_t(&pi_lo)[4] = INV ? F.ns_lo : F.s_lo;
    // four independent accumulation chains: main (hi*hi) and correction
    // (hi*lo + lo*hi) terms of the real and imaginary parts, summed at the end
    float r[4] = {0.f, 0.f, 0.f, 0.f}, im[4] = {0.f, 0.f, 0.f, 0.f};
    float rc[4] = {0.f, 0.f, 0.f, 0.f}, imc[4] = {0.f, 0.f, 0.f, 0.f};
    mma16816<BF16>(rc, F.c_lo, xr_hi0, xr_hi1);
    mma16816<BF16>(imc, pi_lo, xr_hi0, xr_hi1);
    mma16816<BF16>(r, F.c_hi, xr_hi0, xr_hi1);
    mma16816<BF16>(im, pi_hi, xr_hi0, xr_hi1);
    mma16816<BF16>(rc, F.c_hi, xr_lo0, xr_lo1);
    mma16816<BF16>(imc, pi_hi, xr_lo0, xr_lo1);
    mma16816<BF16>(r, pr_hi, xi_hi0, xi_hi1);
    mma16816<BF16>(im, F.c_hi, xi_hi0, xi_hi1);
    mma16816<BF16>(rc, pr_lo, xi_hi0, xi_hi1);
    mma16816<BF16>(imc, F.c_lo, xi_hi0, xi_hi1);
    mma16816<BF16>(rc, pr_hi, xi_lo0, xi_lo1);
    mma16816<BF16>(imc, F.c_hi, xi_lo0, xi_lo1);
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        r[i] += rc[i];
        im[i] += imc[i];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        dr[i] = r[i] * inv_s;
        di[i] = im[i] * inv_s;
    }
}

}  // namespace pgb
