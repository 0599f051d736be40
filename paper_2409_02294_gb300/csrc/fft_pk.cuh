// Packed line transforms: two complex lines that undergo the same sequence
// of operations (the even and odd halves of one padded transform, which
// share every butterfly and every twiddle) are carried together, lane 0 of
// each FP32 pair holding line A and lane 1 line B, in planar form:
//
//     re = (A.re, B.re),  im = (A.im, B.im).
//
// Every add, multiply and fused multiply-add of a butterfly then acts on
// both lines with one packed FP32x2 instruction (sm_100 family), a rotation
// by +-i is a swap of the re and im pairs, and one 16-byte shared-memory
// access moves one element of both lines.  Each lane follows the scalar
// transform of fft_core.cuh (same radices, same twiddle values, same
// order of operations); where the scalar form leaves the pairing of a
// product with an add to the compiler, the packed form fixes it as a fused
// multiply-add, so the two agree to rounding.
#pragma once

#include <cuda_runtime.h>

#include "fft_core.cuh"

namespace pgb {

// --------------------------------------------------------------------------
// packed FP32 pairs and planar complex pairs
// --------------------------------------------------------------------------
__device__ __forceinline__ float2 p2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 pb(float a) { return make_float2(a, a); }  // broadcast
__device__ __forceinline__ float2 padd(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 pmul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 pneg(float2 a) { return make_float2(-a.x, -a.y); }

struct c2 {
    float2 re, im;
};
__device__ __forceinline__ c2 operator+(c2 a, c2 b) { return {padd(a.re, b.re), padd(a.im, b.im)}; }
__device__ __forceinline__ c2 operator-(c2 a, c2 b) { return {psub(a.re, b.re), psub(a.im, b.im)}; }
// -i a and +i a
__device__ __forceinline__ c2 c2_mi(c2 a) { return {a.im, pneg(a.re)}; }
__device__ __forceinline__ c2 c2_pi(c2 a) { return {pneg(a.im), a.re}; }
// a + (-i) b and a - (-i) b without forming -i b
__device__ __forceinline__ c2 add_mi(c2 a, c2 b) { return {padd(a.re, b.im), psub(a.im, b.re)}; }
__device__ __forceinline__ c2 sub_mi(c2 a, c2 b) { return {psub(a.re, b.im), padd(a.im, b.re)}; }

// a * w (forward) or a * conj(w) (inverse) for a twiddle w = (wx, wy),
// applied to both lines through the broadcast pairs (wx, wx), (wy, wy) and
// (-wy, -wy): re = a.re wx -/+ a.im wy, im = a.im wx +/- a.re wy
template <bool INV> __device__ __forceinline__ c2 c2_tw(c2 a, float wx, float wy) {
    const float2 X = pb(wx), Y = pb(wy), NY = pb(-wy);
    if constexpr (INV) return {pfma(a.im, Y, pmul(a.re, X)), pfma(a.re, NY, pmul(a.im, X))};
    else return {pfma(a.im, NY, pmul(a.re, X)), pfma(a.re, Y, pmul(a.im, X))};
}

// pack / unpack: line A from x, line B from y
__device__ __forceinline__ c2 c2_pack(cpx<float> x, cpx<float> y) { return {p2(x.x, y.x), p2(x.y, y.y)}; }
__device__ __forceinline__ cpx<float> c2_a(c2 v) { return {v.re.x, v.im.x}; }
__device__ __forceinline__ cpx<float> c2_b(c2 v) { return {v.re.y, v.im.y}; }

// --------------------------------------------------------------------------
// compile-time twiddles W_N^E (constants folded), packed
// --------------------------------------------------------------------------
template <int N, int E, bool INV>
__device__ __forceinline__ c2 twc_pk(c2 a) {
    static_assert(96 % N == 0, "twiddle base must divide 96");
    constexpr int e = ((E % N) + N) % N;
    constexpr int u = e * (96 / N);
    if constexpr (u == 0) {
        return a;
    } else if constexpr (u == 48) {
        return {pneg(a.re), pneg(a.im)};
    } else if constexpr (u == 24) {  // W = -i (fwd), +i (inv)
        if constexpr (INV) return c2_pi(a); else return c2_mi(a);
    } else if constexpr (u == 72) {  // W = +i (fwd), -i (inv)
        if constexpr (INV) return c2_mi(a); else return c2_pi(a);
    } else {
        constexpr float c = (float)cos96(u);
        constexpr float s = INV ? (float)sin96(u) : (float)(-sin96(u));  // W = c + i s
        // scalar form: {a.x c - a.y s, a.x s + a.y c}
        return {pfma(a.im, pb(-s), pmul(a.re, pb(c))), pfma(a.im, pb(c), pmul(a.re, pb(s)))};
    }
}

// --------------------------------------------------------------------------
// in-register DFTs on packed pairs (natural order in and out)
// --------------------------------------------------------------------------
template <int R_, bool INV> struct DftPk;

template <bool INV> struct DftPk<1, INV> {
    __device__ __forceinline__ static void run(c2*) {}
};
template <bool INV> struct DftPk<2, INV> {
    __device__ __forceinline__ static void run(c2* a) {
        const c2 t = a[0] - a[1];
        a[0] = a[0] + a[1];
        a[1] = t;
    }
};
template <bool INV> struct DftPk<3, INV> {
    __device__ __forceinline__ static void run(c2* a) {
        // X1,2 = a0 - (a1+a2)/2 -/+ i s (a1 - a2), s = sqrt(3)/2 (sign flips for inverse)
        constexpr float s = INV ? -0.866025403784438646764f : 0.866025403784438646764f;
        const c2 sum = a[1] + a[2];
        const c2 dif = a[1] - a[2];
        const c2 m = {pfma(pb(-0.5f), sum.re, a[0].re), pfma(pb(-0.5f), sum.im, a[0].im)};
        a[0] = a[0] + sum;
        a[1] = {pfma(pb(s), dif.im, m.re), pfma(pb(-s), dif.re, m.im)};
        a[2] = {pfma(pb(-s), dif.im, m.re), pfma(pb(s), dif.re, m.im)};
    }
};
template <bool INV> struct DftPk<4, INV> {
    __device__ __forceinline__ static void run(c2* a) {
        const c2 s02 = a[0] + a[2], d02 = a[0] - a[2];
        const c2 s13 = a[1] + a[3], d13 = a[1] - a[3];
        a[0] = s02 + s13;
        a[2] = s02 - s13;
        if constexpr (INV) {  // W_4^1 = +i
            a[1] = sub_mi(d02, d13);
            a[3] = add_mi(d02, d13);
        } else {              // W_4^1 = -i
            a[1] = add_mi(d02, d13);
            a[3] = sub_mi(d02, d13);
        }
    }
};

// Cooley-Tukey in registers: N = N1 * N2, n = N2*n1 + n2, k = k1 + N1*k2.
template <int N1, int N2, bool INV>
__device__ __forceinline__ void dft_split_pk(c2* a) {
    constexpr int N = N1 * N2;
    c2 t[N];
    sfor<N2>([&](auto n2c) {
        constexpr int n2 = decltype(n2c)::value;
        c2 u[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) u[n1] = a[N2 * n1 + n2];
        DftPk<N1, INV>::run(u);
        sfor<N1>([&](auto k1c) {
            constexpr int k1 = decltype(k1c)::value;
            t[n2 * N1 + k1] = twc_pk<N, n2 * k1, INV>(u[k1]);
        });
    });
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
        c2 u[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) u[n2] = t[n2 * N1 + k1];
        DftPk<N2, INV>::run(u);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) a[k1 + N1 * k2] = u[k2];
    }
}

template <bool INV> struct DftPk<6, INV> {
    __device__ __forceinline__ static void run(c2* a) { dft_split_pk<2, 3, INV>(a); }
};
template <bool INV> struct DftPk<8, INV> {
    __device__ __forceinline__ static void run(c2* a) { dft_split_pk<2, 4, INV>(a); }
};
template <bool INV> struct DftPk<12, INV> {
    __device__ __forceinline__ static void run(c2* a) { dft_split_pk<4, 3, INV>(a); }
};
template <bool INV> struct DftPk<16, INV> {
    __device__ __forceinline__ static void run(c2* a) { dft_split_pk<4, 4, INV>(a); }
};
template <bool INV> struct DftPk<24, INV> {
    __device__ __forceinline__ static void run(c2* a) { dft_split_pk<8, 3, INV>(a); }
};
template <bool INV> struct DftPk<32, INV> {
    __device__ __forceinline__ static void run(c2* a) { dft_split_pk<4, 8, INV>(a); }
};

// Exchange buffer of a packed line: element i (both lines) at base[idx(i)],
// idx(i) = i * stride + (i >> pad_shift) * pad, one 16-byte float4
// (A.re, B.re, A.im, B.im) per element.
struct LineSmemPk {
    float4* base;
    int stride;
    int pad_shift;
    int pad;
    __device__ __forceinline__ float4& operator[](int i) const { return base[i * stride + (i >> pad_shift) * pad]; }
};
__device__ __forceinline__ float4 c2_to4(c2 v) { return make_float4(v.re.x, v.re.y, v.im.x, v.im.y); }
__device__ __forceinline__ c2 c2_from4(float4 f) { return {p2(f.x, f.y), p2(f.z, f.w)}; }

// Stockham stages over a thread's E packed registers: v[m] = x[t + T m] of
// both lines.  tw2N: the axis' twiddle table of fft_core.cuh (W_2N^j, then
// the per-stage tables, read exactly as the scalar stages read them); each
// twiddle is applied to both lines as broadcast pairs.  TOFF: this stage's
// table offset.
template <int N, int E, bool INV, int NS, int TOFF, int RAD, int... REST>
__device__ __forceinline__ void stockham_pk(c2 (&v)[E], int t, const LineSmemPk& sm,
                                            const cpx<float>* __restrict__ tw2N) {
    constexpr int T = N / E;
    constexpr int B = E / RAD;
    static_assert(E % RAD == 0, "radix must divide the per-thread element count");
    static_assert(RAD % 2 == 0 || NS == 1, "twiddled stages need an even radix");
    constexpr bool LAST = sizeof...(REST) == 0;
    static_assert(!LAST || NS * RAD == N, "radices must multiply to N");
#pragma unroll
    for (int g = 0; g < B; ++g) {
        const int b = t + T * g;
        int k = 0;
        if constexpr (NS > 1) {
            k = b % NS;
            const cpx<float>* st = tw2N + TOFF;
            if constexpr (RAD == 2) {
                const cpx<float> w = ldg_c(st + k);
                v[g + B] = c2_tw<INV>(v[g + B], w.x, w.y);
            } else {
#pragma unroll
                for (int q = 0; q < RAD / 2; ++q) {
                    const int r0 = 2 * q + 1;
                    cpx<float> w0, w1;
                    if (r0 + 1 < RAD) ldg_c2(st + 2 * (q * NS + k), w0, w1);
                    else w0 = ldg_c(st + 2 * (q * NS + k));
                    v[g + B * r0] = c2_tw<INV>(v[g + B * r0], w0.x, w0.y);
                    if (r0 + 1 < RAD) v[g + B * (r0 + 1)] = c2_tw<INV>(v[g + B * (r0 + 1)], w1.x, w1.y);
                }
            }
        }
        c2 u[RAD];
#pragma unroll
        for (int r = 0; r < RAD; ++r) u[r] = v[g + B * r];
        DftPk<RAD, INV>::run(u);
        if constexpr (LAST) {
#pragma unroll
            for (int r = 0; r < RAD; ++r) v[g + B * r] = u[r];
        } else {
            const int base = (b / NS) * NS * RAD + k;
#pragma unroll
            for (int r = 0; r < RAD; ++r) sm[base + r * NS] = c2_to4(u[r]);
        }
    }
    if constexpr (!LAST) {
        __syncthreads();
#pragma unroll
        for (int m = 0; m < E; ++m) v[m] = c2_from4(sm[t + T * m]);
        __syncthreads();
        stockham_pk<N, E, INV, NS * RAD, TOFF + stage_tw_size<NS, RAD>(), REST...>(v, t, sm, tw2N);
    }
}

template <int N, int E, bool INV, int... Rs>
__device__ __forceinline__ void line_fft_pk(c2 (&v)[E], int t, const LineSmemPk& sm,
                                            const cpx<float>* __restrict__ tw2N, Radices<Rs...>) {
    static_assert(RadProd<Rs...>::v == N, "radices must multiply to N");
    stockham_pk<N, E, INV, 1, 2 * N, Rs...>(v, t, sm, tw2N);
}

}  // namespace pgb
