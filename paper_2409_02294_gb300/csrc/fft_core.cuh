// Register/shared-memory FFT building blocks for the Poisson passes (sm_103a).
//
// A line of length N is spread over T = N / E threads; thread t holds the E
// elements x[t + T*m], m = 0..E-1, in registers.  A transform is a sequence of
// Stockham (self-sorting) stages with compile-time radices; every radix
// divides E, so each thread performs E / radix butterflies per stage, and
// consecutive stages exchange data through one shared-memory buffer per
// line.  After the last stage thread t holds X[t + T*m] in natural order, so
// loads and stores of a line use the same index pattern on both sides.
//
// Butterflies use twiddle constants folded at compile time (cos(2*pi*u/96)
// table below, values from the exact trigonometric definition); the
// inter-stage twiddles come from a per-axis table of the 2N-th roots of
// unity computed in FP64 on the host and rounded once, re-laid out per stage
// (below) so that a warp's twiddle reads are contiguous.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <type_traits>
#include <utility>

namespace pgb {

// --------------------------------------------------------------------------
// complex numbers
// --------------------------------------------------------------------------
template <class R> struct alignas(2 * sizeof(R)) cpx {
    R x, y;
};

template <class R> __device__ __forceinline__ cpx<R> mk(R x, R y) { return cpx<R>{x, y}; }
template <class R> __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return {a.x + b.x, a.y + b.y}; }
template <class R> __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return {a.x - b.x, a.y - b.y}; }
template <class R> __device__ __forceinline__ cpx<R> operator-(cpx<R> a) { return {-a.x, -a.y}; }
template <class R> __device__ __forceinline__ cpx<R> scale(cpx<R> a, R s) { return {a.x * s, a.y * s}; }
// conj(a) * s
template <class R> __device__ __forceinline__ cpx<R> scale_conj(cpx<R> a, R s) { return {a.x * s, a.y * -s}; }
// a * b
template <class R> __device__ __forceinline__ cpx<R> cmul(cpx<R> a, cpx<R> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// a * conj(b)
template <class R> __device__ __forceinline__ cpx<R> cmulc(cpx<R> a, cpx<R> b) {
    return {a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y};
}
// a * w for w = b (forward) or conj(b) (inverse)
template <bool INV, class R> __device__ __forceinline__ cpx<R> cmul_dir(cpx<R> a, cpx<R> b) {
    if constexpr (INV) return cmulc(a, b);
    else return cmul(a, b);
}
// -i * a and +i * a
template <class R> __device__ __forceinline__ cpx<R> mul_mi(cpx<R> a) { return {a.y, -a.x}; }
template <class R> __device__ __forceinline__ cpx<R> mul_pi(cpx<R> a) { return {-a.y, a.x}; }

template <class R> __device__ __forceinline__ cpx<R> ldg_c(const cpx<R>* p) {
    if constexpr (std::is_same<R, float>::value) {
        float2 v = __ldg(reinterpret_cast<const float2*>(p));
        return {v.x, v.y};
    } else {
        double2 v = __ldg(reinterpret_cast<const double2*>(p));
        return {v.x, v.y};
    }
}

// two adjacent entries p[0], p[1] (p 16-byte aligned)
template <class R> __device__ __forceinline__ void ldg_c2(const cpx<R>* p, cpx<R>& a, cpx<R>& b) {
    if constexpr (std::is_same<R, float>::value) {
        const float4 v = __ldg(reinterpret_cast<const float4*>(p));
        a = {v.x, v.y};
        b = {v.z, v.w};
    } else {
        a = ldg_c(p);
        b = ldg_c(p + 1);
    }
}

// Twiddle-table reads: from global memory through the read-only path, or
// (SM) from a copy of the table in shared memory (the persistent column
// kernels keep one per CTA: their tiles fill most of the unified L1/shared
// storage, and table reads through the small L1 that remains mostly miss).
template <bool SM, class R> __device__ __forceinline__ cpx<R> tw_ld(const cpx<R>* p) {
    if constexpr (SM) return *p;
    else return ldg_c(p);
}
template <bool SM, class R> __device__ __forceinline__ void tw_ld2(const cpx<R>* p, cpx<R>& a, cpx<R>& b) {
    if constexpr (SM && std::is_same<R, float>::value) {
        const float4 v = *reinterpret_cast<const float4*>(p);
        a = {v.x, v.y};
        b = {v.z, v.w};
    } else if constexpr (SM) {
        a = p[0];
        b = p[1];
    } else {
        ldg_c2(p, a, b);
    }
}

// Load of data that this kernel launch may also have written elsewhere on
// the GPU: CG = true bypasses L1 (ld.global.cg), which is required when a
// persistent kernel reads data produced by other SMs in the same launch.
template <bool CG, class R> __device__ __forceinline__ cpx<R> ld_c(const cpx<R>* p) {
    if constexpr (CG) {
        if constexpr (std::is_same<R, float>::value) {
            float2 v = __ldcg(reinterpret_cast<const float2*>(p));
            return {v.x, v.y};
        } else {
            double2 v = __ldcg(reinterpret_cast<const double2*>(p));
            return {v.x, v.y};
        }
    } else {
        return *p;
    }
}

// --------------------------------------------------------------------------
// compile-time twiddles: W_n^e = exp(-2 pi i e / n) for n dividing 96
// --------------------------------------------------------------------------
__host__ __device__ constexpr double cos96_q(int u) {  // u in [0, 24]
    constexpr double t[25] = {
        1.0,
        0.997858923238603506738,
        0.991444861373810411145,
        0.980785280403230449126,
        0.965925826289068286750,
        0.946930129495105664256,
        0.923879532511286756128,
        0.896872741532688303894,
        0.866025403784438646764,
        0.831469612302545237079,
        0.793353340291235164580,
        0.751839807478977396408,
        0.707106781186547524401,
        0.659345815100068868425,
        0.608761429008720639416,
        0.555570233019602224743,
        0.5,
        0.442288690219001281995,
        0.382683432365089771728,
        0.321439465303161580701,
        0.258819045102520762349,
        0.195090322016128267848,
        0.130526192220051591548,
        0.0654031292301430668153,
        0.0,
    };
    return t[u];
}
__host__ __device__ constexpr double cos96(int u) {  // cos(2 pi u / 96), any integer u
    u = ((u % 96) + 96) % 96;
    if (u <= 24) return cos96_q(u);
    if (u <= 48) return -cos96_q(48 - u);
    if (u <= 72) return -cos96_q(u - 48);
    return cos96_q(96 - u);
}
__host__ __device__ constexpr double sin96(int u) { return cos96(u - 24); }

// multiply a by W_N^E (forward) or its conjugate (inverse), constants folded
template <int N, int E, bool INV, class R>
__device__ __forceinline__ cpx<R> twc(cpx<R> a) {
    static_assert(96 % N == 0, "twiddle base must divide 96");
    constexpr int e = ((E % N) + N) % N;
    constexpr int u = e * (96 / N);
    if constexpr (u == 0) {
        return a;
    } else if constexpr (u == 48) {
        return -a;
    } else if constexpr (u == 24) {  // W = -i (fwd), +i (inv)
        if constexpr (INV) return mul_pi(a); else return mul_mi(a);
    } else if constexpr (u == 72) {  // W = +i (fwd), -i (inv)
        if constexpr (INV) return mul_mi(a); else return mul_pi(a);
    } else {
        constexpr R c = (R)cos96(u);
        constexpr R s = INV ? (R)sin96(u) : (R)(-sin96(u));  // W = c + i s
        return {a.x * c - a.y * s, a.x * s + a.y * c};
    }
}

// --------------------------------------------------------------------------
// compile-time loops
// --------------------------------------------------------------------------
template <int I, int N, class F>
__device__ __forceinline__ void sfor_impl(F&& f) {
    if constexpr (I < N) {
        f(std::integral_constant<int, I>{});
        sfor_impl<I + 1, N>(f);
    }
}
template <int N, class F> __device__ __forceinline__ void sfor(F&& f) { sfor_impl<0, N>(f); }

// --------------------------------------------------------------------------
// compile-time cos and sin of pi p / q: the angle is reduced exactly (in
// integers) to a quarter turn plus phi in [0, pi/2), phi or pi/2 - phi
// (whichever is <= pi/4) goes through the Taylor series, summed to far below
// double rounding, and the quarter turns rotate the result
// --------------------------------------------------------------------------
__host__ __device__ constexpr double taylor_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int k = 1; k <= 12; ++k) {
        term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k));
        sum += term;
    }
    return sum;
}
__host__ __device__ constexpr double taylor_sin(double x) {
    double term = x, sum = x;
    for (int k = 1; k <= 12; ++k) {
        term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0));
        sum += term;
    }
    return sum;
}
struct CosSin {
    double c, s;
};
__host__ __device__ constexpr CosSin cos_sin_pi_frac(long long p, long long q) {
    const long long P = ((p % (2 * q)) + 2 * q) % (2 * q);  // angle pi P / q in [0, 2 pi)
    const long long k = (2 * P) / q;                          // quarter turns
    const long long r = 2 * P - k * q;                        // phi = pi r / (2 q) in [0, pi/2)
    const double half_pi_over_q = 1.57079632679489661923132169163975144 / (double)q;
    double c = 0.0, s = 0.0;
    if (2 * r <= q) {
        c = taylor_cos(half_pi_over_q * (double)r);
        s = taylor_sin(half_pi_over_q * (double)r);
    } else {
        c = taylor_sin(half_pi_over_q * (double)(q - r));
        s = taylor_cos(half_pi_over_q * (double)(q - r));
    }
    if (k == 0) return {c, s};
    if (k == 1) return {-s, c};
    if (k == 2) return {-c, -s};
    return {s, -c};
}

// The pre- and post-multiplies of a padded (length 2N) transform use
// W_2N^j at j = t + T m, m < E (T = N / E).  They factor as W_2N^t, one
// table load per thread, times W_2E^m = exp(-i pi m / E), a constant of the
// unrolled loop, instead of one table load per element.
template <int N, int E, class R, bool TWS = false> struct LineRamp {
    cpx<R> wt;
    __device__ __forceinline__ LineRamp(const cpx<R>* tw2N, int t) : wt(tw_ld<TWS>(tw2N + t)) {}
    template <int M> __device__ __forceinline__ cpx<R> at() const {
        if constexpr (M == 0) {
            return wt;
        } else if constexpr (2 * M == E) {  // W_2E^(E/2) = -i
            return mul_mi(wt);
        } else {
            constexpr CosSin w = cos_sin_pi_frac(M, E);
            constexpr R c = (R)w.c, s = (R)(-w.s);
            return {wt.x * c - wt.y * s, wt.x * s + wt.y * c};
        }
    }
};

// --------------------------------------------------------------------------
// in-register DFTs, natural order in and out: a[k] <- sum_n a[n] W_R^{nk}
// --------------------------------------------------------------------------
template <int R_, bool INV, class R> struct Dft;

template <bool INV, class R> struct Dft<1, INV, R> {
    __device__ __forceinline__ static void run(cpx<R>*) {}
};
template <bool INV, class R> struct Dft<2, INV, R> {
    __device__ __forceinline__ static void run(cpx<R>* a) {
        cpx<R> t = a[0] - a[1];
        a[0] = a[0] + a[1];
        a[1] = t;
    }
};
template <bool INV, class R> struct Dft<3, INV, R> {
    __device__ __forceinline__ static void run(cpx<R>* a) {
        // X1,2 = a0 - (a1+a2)/2 -/+ i s (a1 - a2), s = sqrt(3)/2 (sign flips for inverse)
        constexpr R s = INV ? (R)(-0.866025403784438646764) : (R)0.866025403784438646764;
        cpx<R> sum = a[1] + a[2];
        cpx<R> dif = a[1] - a[2];
        cpx<R> m = {a[0].x - (R)0.5 * sum.x, a[0].y - (R)0.5 * sum.y};
        a[0] = a[0] + sum;
        a[1] = {m.x + s * dif.y, m.y - s * dif.x};
        a[2] = {m.x - s * dif.y, m.y + s * dif.x};
    }
};
template <bool INV, class R> struct Dft<4, INV, R> {
    __device__ __forceinline__ static void run(cpx<R>* a) {
        cpx<R> s02 = a[0] + a[2], d02 = a[0] - a[2];
        cpx<R> s13 = a[1] + a[3], d13 = a[1] - a[3];
        cpx<R> r = INV ? mul_pi(d13) : mul_mi(d13);  // W_4^1 (b - d)
        a[0] = s02 + s13;
        a[2] = s02 - s13;
        a[1] = d02 + r;
        a[3] = d02 - r;
    }
};

// Cooley-Tukey in registers: N = N1 * N2, n = N2*n1 + n2, k = k1 + N1*k2.
template <int N1, int N2, bool INV, class R>
__device__ __forceinline__ void dft_split(cpx<R>* a) {
    constexpr int N = N1 * N2;
    cpx<R> t[N];
    sfor<N2>([&](auto n2c) {
        constexpr int n2 = decltype(n2c)::value;
        cpx<R> u[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) u[n1] = a[N2 * n1 + n2];
        Dft<N1, INV, R>::run(u);
        sfor<N1>([&](auto k1c) {
            constexpr int k1 = decltype(k1c)::value;
            t[n2 * N1 + k1] = twc<N, n2 * k1, INV>(u[k1]);
        });
    });
#pragma unroll
    for (int k1 = 0; k1 < N1; ++k1) {
        cpx<R> u[N2];
#pragma unroll
        for (int n2 = 0; n2 < N2; ++n2) u[n2] = t[n2 * N1 + k1];
        Dft<N2, INV, R>::run(u);
#pragma unroll
        for (int k2 = 0; k2 < N2; ++k2) a[k1 + N1 * k2] = u[k2];
    }
}

template <bool INV, class R> struct Dft<6, INV, R> {
    __device__ __forceinline__ static void run(cpx<R>* a) { dft_split<2, 3, INV, R>(a); }
};
template <bool INV, class R> struct Dft<8, INV, R> {
    __device__ __forceinline__ static void run(cpx<R>* a) { dft_split<2, 4, INV, R>(a); }
};
template <bool INV, class R> struct Dft<12, INV, R> {
    __device__ __forceinline__ static void run(cpx<R>* a) { dft_split<4, 3, INV, R>(a); }
};
template <bool INV, class R> struct Dft<16, INV, R> {
    __device__ __forceinline__ static void run(cpx<R>* a) { dft_split<4, 4, INV, R>(a); }
};
template <bool INV, class R> struct Dft<24, INV, R> {
    __device__ __forceinline__ static void run(cpx<R>* a) { dft_split<8, 3, INV, R>(a); }
};
template <bool INV, class R> struct Dft<32, INV, R> {
    __device__ __forceinline__ static void run(cpx<R>* a) { dft_split<4, 8, INV, R>(a); }
};

// --------------------------------------------------------------------------
// Stockham stages over a thread's E registers
// --------------------------------------------------------------------------
template <int... Rs> struct Radices {};

template <int A, int... Rs> struct RadProd { static constexpr int v = A * RadProd<Rs...>::v; };
template <int A> struct RadProd<A> { static constexpr int v = A; };

// --------------------------------------------------------------------------
// per-stage twiddle tables
// --------------------------------------------------------------------------
// A Stockham stage with NS > 1 multiplies input r of butterfly k (k < NS) by
// W_{NS RAD}^{r k}.  Read straight from the W_2N table, lanes with
// consecutive k are r*k entries apart and one warp request touches up to 16
// cache lines.  So every such stage gets its own table, stored after the 2N
// entries of W_2N^j, with k fastest:
//   RAD == 2: entry k                      = W_{2 NS}^k
//   RAD >  2: entry 2 (p NS + k) + i       = W_{NS RAD}^{(2p+1+i) k},  p < RAD/2, i < 2
// (pairs, so that an FP32 thread fetches two twiddles with one 16-byte load).
// Entries are copies of W_2N entries (W_{NS RAD}^{rk} = W_2N^{rk 2N/(NS RAD)}),
// so the transform's arithmetic is unchanged.  All radices are even, hence so
// is every table offset and the 16-byte loads stay aligned.
template <int NS, int RAD> constexpr int stage_tw_size() { return NS > 1 ? (RAD == 2 ? NS : NS * RAD) : 0; }
template <int NS, int RAD, int... REST> constexpr int stage_tw_total() {
    if constexpr (sizeof...(REST) == 0) return stage_tw_size<NS, RAD>();
    else return stage_tw_size<NS, RAD>() + stage_tw_total<NS * RAD, REST...>();
}
// complex entries of an axis' twiddle table for a radix sequence
template <int N, int... Rs> constexpr int tw_entries(Radices<Rs...>) { return 2 * N + stage_tw_total<1, Rs...>(); }

// Host-side description of the stage tables of one radix sequence.
struct StageTwList {
    int count = 0;      // stages with a table
    int ns[8] = {};     // their NS
    int rad[8] = {};    // their radix
    int off[8] = {};    // offset of their table (complex entries)
    int total = 0;      // entries of the whole axis table
};
template <int N, int... Rs> StageTwList stage_tw_list(Radices<Rs...>) {
    StageTwList L;
    int ns = 1, off = 2 * N;
    for (int r : {Rs...}) {
        if (ns > 1) {
            L.ns[L.count] = ns;
            L.rad[L.count] = r;
            L.off[L.count] = off;
            off += r == 2 ? ns : ns * r;
            ++L.count;
        }
        ns *= r;
    }
    L.total = off;
    return L;
}

// Shared-memory view of one line's exchange buffer: element i lives at
// base[idx(i)], idx(i) = i * stride + (i >> pad_shift) * pad.  Column tiles
// use stride = line slots, pad = 0; row tiles use stride = 1 and one
// padding element every 2^pad_shift elements to break stride conflicts.
template <class R> struct LineSmem {
    cpx<R>* base;
    int stride;
    int pad_shift;
    int pad;
    __device__ __forceinline__ cpx<R>& operator[](int i) const {
        return base[i * stride + (i >> pad_shift) * pad];
    }
};

// One line per "lane set": NL independent lines (e.g. the even and odd
// halves of a padded transform) are transformed together, stage by stage,
// to give the scheduler independent work.  v[l][m] = x_l[t + T*m].
// tw2N: an axis twiddle table (W_{2N}^j, j < 2N, then the stage tables);
// TOFF: offset of this stage's table.
template <class R, int N, int E, bool INV, int NL, bool TWS, int NS, int TOFF, int RAD, int... REST>
__device__ __forceinline__ void stockham(cpx<R> (&v)[NL][E], int t, const LineSmem<R> (&sm)[NL],
                                         const cpx<R>* __restrict__ tw2N) {
    constexpr int T = N / E;
    constexpr int B = E / RAD;
    static_assert(E % RAD == 0, "radix must divide the per-thread element count");
    static_assert(RAD % 2 == 0 || NS == 1, "twiddled stages need an even radix");
    constexpr bool LAST = sizeof...(REST) == 0;
    static_assert(!LAST || NS * RAD == N, "radices must multiply to N");
#pragma unroll
    for (int g = 0; g < B; ++g) {
        const int b = t + T * g;  // butterfly index in [0, N/RAD)
        int k = 0;
        if constexpr (NS > 1) {
            k = b % NS;
            const cpx<R>* st = tw2N + TOFF;
            if constexpr (RAD == 2) {
                const cpx<R> w = tw_ld<TWS>(st + k);
#pragma unroll
                for (int l = 0; l < NL; ++l) v[l][g + B] = cmul_dir<INV>(v[l][g + B], w);
            } else {
#pragma unroll
                for (int q = 0; q < RAD / 2; ++q) {
                    const int r0 = 2 * q + 1;
                    cpx<R> w0, w1;
                    if (r0 + 1 < RAD) tw_ld2<TWS>(st + 2 * (q * NS + k), w0, w1);
                    else w0 = tw_ld<TWS>(st + 2 * (q * NS + k));
#pragma unroll
                    for (int l = 0; l < NL; ++l) {
                        v[l][g + B * r0] = cmul_dir<INV>(v[l][g + B * r0], w0);
                        if (r0 + 1 < RAD) v[l][g + B * (r0 + 1)] = cmul_dir<INV>(v[l][g + B * (r0 + 1)], w1);
                    }
                }
            }
        }
#pragma unroll
        for (int l = 0; l < NL; ++l) {
            cpx<R> u[RAD];
#pragma unroll
            for (int r = 0; r < RAD; ++r) u[r] = v[l][g + B * r];
            Dft<RAD, INV, R>::run(u);
            if constexpr (LAST) {
#pragma unroll
                for (int r = 0; r < RAD; ++r) v[l][g + B * r] = u[r];
            } else {
                const int base = (b / NS) * NS * RAD + k;
#pragma unroll
                for (int r = 0; r < RAD; ++r) sm[l][base + r * NS] = u[r];
            }
        }
    }
    if constexpr (!LAST) {
        __syncthreads();
#pragma unroll
        for (int l = 0; l < NL; ++l)
#pragma unroll
            for (int m = 0; m < E; ++m) v[l][m] = sm[l][t + T * m];
        __syncthreads();
        stockham<R, N, E, INV, NL, TWS, NS * RAD, TOFF + stage_tw_size<NS, RAD>(), REST...>(v, t, sm, tw2N);
    }
}

// TWS: tw2N points to a copy of the table in shared memory
template <class R, int N, int E, bool INV, int NL, bool TWS = false, int... Rs>
__device__ __forceinline__ void line_fft(cpx<R> (&v)[NL][E], int t, const LineSmem<R> (&sm)[NL],
                                         const cpx<R>* __restrict__ tw2N, Radices<Rs...>) {
    static_assert(RadProd<Rs...>::v == N, "radices must multiply to N");
    stockham<R, N, E, INV, NL, TWS, 1, 2 * N, Rs...>(v, t, sm, tw2N);
}

}  // namespace pgb
