// Column passes with packed line transforms (FP32): each thread carries the
// even and odd halves of its padded column transform as one packed line
// (fft_pk.cuh), so every butterfly, twiddle product and exchange acts on
// both halves at once.  Same tiles, layouts and arithmetic as the two-line
// column kernels of passes.cuh (y forward, z convolve, y inverse); only the
// instruction form differs.
#pragma once

#include "fft_pk.cuh"
#include "passes.cuh"

namespace pgb {

template <int N, int SLOTS> constexpr size_t pk_col_smem() { return (size_t)N * SLOTS * sizeof(float4); }
template <int N, int SLOTS> constexpr size_t pk_col_smem_z() {
    return pk_col_smem<N, SLOTS>() + (size_t)gsl_elems<float, N, SLOTS>() * sizeof(float);
}

template <class Cfg, int SLOTS> struct PkIds {
    int slot, t;
    __device__ __forceinline__ PkIds() {
        static_assert(SLOTS >= 8, "packed column tiles need rows of at least 128 bytes");
        slot = threadIdx.x % SLOTS;
        t = threadIdx.x / SLOTS;
    }
};

// the padded transform's odd half starts as x_j W_2N^j: pack (x, x W)
__device__ __forceinline__ c2 pack_even_odd(cpx<float> x, cpx<float> w) { return c2_pack(x, cmul(x, w)); }

// pass 1: pad + forward FFT along y, W1 -> W2 (both halves of a column).
template <class Cfg, int SLOTS>
__device__ __forceinline__ void tile_y_fwd_pk(const PassParams<float>& p, int tile, unsigned char* smem_raw) {
    constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T;
    const PkIds<Cfg, SLOTS> id;
    const int ny = p.ny;
    const ColTile<float, SLOTS> c = col_tile<float, SLOTS>(p.nx + 1, p.nz, id.slot, tile);
    const cpx<float>* __restrict__ in = static_cast<const cpx<float>*>(p.in);
    cpx<float>* __restrict__ out = static_cast<cpx<float>*>(p.out);
    const long long sx = p.sx;

    c2 v[E];
    const cpx<float>* src = in + (long long)c.other * ny * sx + c.kx + (long long)id.t * sx;
    const LineRamp<N, E, float> rw(p.tw, id.t);
    sfor<E>([&](auto m_) {
        constexpr int m = decltype(m_)::value;
        const cpx<float> x = c.valid ? src[(long long)(T * m) * sx] : cpx<float>{0, 0};
        v[m] = pack_even_odd(x, rw.template at<m>());
    });
    const LineSmemPk ls{reinterpret_cast<float4*>(smem_raw) + id.slot, SLOTS, 30, 0};
    line_fft_pk<N, E, false>(v, id.t, ls, p.tw, typename Cfg::Rads{});
    if (c.valid) {
        cpx<float>* dst = out + (long long)c.other * 2 * ny * sx + c.kx + (long long)id.t * sx;
        const long long odd = (long long)ny * sx;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            dst[(long long)(T * m) * sx] = c2_a(v[m]);
            dst[odd + (long long)(T * m) * sx] = c2_b(v[m]);
        }
    }
}

// pass 2: pad + FFT along z, multiply by Ghat, inverse FFT along z, crop;
// in place on W2.  The column's Green's row is staged exactly as in
// tile_z_conv (two lines per thread).
template <class Cfg, int SLOTS>
__device__ __forceinline__ void tile_z_conv_pk(const PassParams<float>& p, int tile, unsigned char* smem_raw) {
    using R = float;
    constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T;
    const PkIds<Cfg, SLOTS> id;
    const int nx = p.nx, ny = p.ny;
    const ColTile<R, SLOTS> c = col_tile<R, SLOTS>(nx + 1, 2 * ny, id.slot, tile);
    cpx<R>* __restrict__ w = static_cast<cpx<R>*>(p.out);
    const long long plane = 2LL * ny * p.sx;
    float4* smp = reinterpret_cast<float4*>(smem_raw);

    R* gsl = reinterpret_cast<R*>(smp + N * SLOTS);
    if (c.valid) {
        const int kys = c.other;
        const int ky = kys < ny ? 2 * kys : 2 * (kys - ny) + 1;
        const int kyf = ky <= ny ? ky : 2 * ny - ky;
        constexpr int gz = greens_xw<R>();  // kz stride within the block
        const R* g = p.greens + greens_base<R>(c.kx, kyf, nx, p.nz);
        const int u = id.t;
        if constexpr (T % gsl_group<R, SLOTS>() == 0) {
            R* sp = gsl + gsl_idx<R, SLOTS>(u, id.slot);
            const R* gp = g + u * gz;
#pragma unroll
            for (int i = 0; i < N / T; ++i) cp_async_real(sp + i * T * SLOTS, gp + i * T * gz);
            if (u == 0) cp_async_real(sp + N * SLOTS, gp + N * gz);
        } else {
            for (int kz = u; kz <= N; kz += T) cp_async_real(gsl + gsl_idx<R, SLOTS>(kz, id.slot), g + kz * gz);
        }
    }
    cp_async_commit();

    c2 v[E];
    cpx<R>* col = w + (long long)c.other * p.sx + c.kx;
    const LineRamp<N, E, R> rw(p.tw, id.t);
    sfor<E>([&](auto m_) {
        constexpr int m = decltype(m_)::value;
        const cpx<R> x = c.valid ? col[(long long)(id.t + T * m) * plane] : cpx<R>{0, 0};
        v[m] = pack_even_odd(x, rw.template at<m>());
    });
    const LineSmemPk ls{smp + id.slot, SLOTS, 30, 0};
    line_fft_pk<N, E, false>(v, id.t, ls, p.tw, typename Cfg::Rads{});

    // Green's multiply: lane A (even half) at kz = 2 (t + T m), lane B (odd
    // half) at kz + 1, folded into the octant (kz <= N exactly for m < E/2)
    cp_async_commit_wait_all();
    __syncthreads();
    if (c.valid) {
        const int kz0 = 2 * id.t;
        if constexpr (T % gsl_group<R, SLOTS>() == 0) {
            const int lo0 = gsl_idx<R, SLOTS>(kz0, id.slot), hi0 = gsl_idx<R, SLOTS>(2 * N - kz0, id.slot);
            const int lo1 = gsl_idx<R, SLOTS>(kz0 + 1, id.slot), hi1 = gsl_idx<R, SLOTS>(2 * N - kz0 - 1, id.slot);
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int d = 2 * T * m * SLOTS;
                const float2 G = m < E / 2 ? p2(gsl[lo0 + d], gsl[lo1 + d]) : p2(gsl[hi0 - d], gsl[hi1 - d]);
                v[m] = {pmul(v[m].re, G), pmul(v[m].im, G)};
            }
        } else {
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int kz = kz0 + 2 * T * m;
                const int ke = m < E / 2 ? kz : 2 * N - kz;
                const int ko = m < E / 2 ? kz + 1 : 2 * N - kz - 1;
                const float2 G = p2(gsl[gsl_idx<R, SLOTS>(ke, id.slot)], gsl[gsl_idx<R, SLOTS>(ko, id.slot)]);
                v[m] = {pmul(v[m].re, G), pmul(v[m].im, G)};
            }
        }
    }

    line_fft_pk<N, E, true>(v, id.t, ls, p.tw, typename Cfg::Rads{});

    // x[j] = a[j] + W_2N^-j b[j], j < N
    if (c.valid) {
        sfor<E>([&](auto m_) {
            constexpr int m = decltype(m_)::value;
            col[(long long)(id.t + T * m) * plane] = c2_a(v[m]) + cmulc(c2_b(v[m]), rw.template at<m>());
        });
    }
}

// pass 3: inverse FFT along y + crop, W2 -> W1.
template <class Cfg, int SLOTS>
__device__ __forceinline__ void tile_y_inv_pk(const PassParams<float>& p, int tile, unsigned char* smem_raw) {
    constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T;
    const PkIds<Cfg, SLOTS> id;
    const int ny = p.ny;
    const ColTile<float, SLOTS> c = col_tile<float, SLOTS>(p.nx + 1, p.nz, id.slot, tile);
    const cpx<float>* __restrict__ in = static_cast<const cpx<float>*>(p.in);
    cpx<float>* __restrict__ out = static_cast<cpx<float>*>(p.out);
    const long long sx = p.sx;

    c2 v[E];
    const cpx<float>* src = in + (long long)c.other * 2 * ny * sx + c.kx + (long long)id.t * sx;
    const long long odd = (long long)ny * sx;
#pragma unroll
    for (int m = 0; m < E; ++m) {
        cpx<float> a{0, 0}, b{0, 0};
        if (c.valid) {
            a = src[(long long)(T * m) * sx];
            b = src[odd + (long long)(T * m) * sx];
        }
        v[m] = c2_pack(a, b);
    }
    const LineSmemPk ls{reinterpret_cast<float4*>(smem_raw) + id.slot, SLOTS, 30, 0};
    line_fft_pk<N, E, true>(v, id.t, ls, p.tw, typename Cfg::Rads{});
    if (c.valid) {
        cpx<float>* dst = out + (long long)c.other * ny * sx + c.kx + (long long)id.t * sx;
        const LineRamp<N, E, float> rw(p.tw, id.t);
        sfor<E>([&](auto m_) {
            constexpr int m = decltype(m_)::value;
            dst[(long long)(T * m) * sx] = c2_a(v[m]) + cmulc(c2_b(v[m]), rw.template at<m>());
        });
    }
}

template <class Cfg, int SLOTS, int MINB>
__global__ void __launch_bounds__(SLOTS * Cfg::T, MINB) k_y_fwd_pk(PassParams<float> p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_y_fwd_pk<Cfg, SLOTS>(p, blockIdx.x + p.tile0, smem_raw);
}
template <class Cfg, int SLOTS, int MINB>
__global__ void __launch_bounds__(SLOTS * Cfg::T, MINB) k_z_conv_pk(PassParams<float> p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_z_conv_pk<Cfg, SLOTS>(p, blockIdx.x + p.tile0, smem_raw);
}
template <class Cfg, int SLOTS, int MINB>
__global__ void __launch_bounds__(SLOTS * Cfg::T, MINB) k_y_inv_pk(PassParams<float> p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_y_inv_pk<Cfg, SLOTS>(p, blockIdx.x + p.tile0, smem_raw);
}

// Launch one packed column pass (pass 1, 2 or 3) of tile width S.
template <class Cfg, int S, int MINB>
cudaError_t launch_col_pk(int pass, const PassParams<float>& p, cudaStream_t st) {
    constexpr int NT = S * Cfg::T;
    static_assert(NT <= 1024, "column CTA too large");
    const int lines = pass == 2 ? 2 * p.ny : p.nz;
    const int grid = p.ntile > 0 ? p.ntile : col_grid<float, S>(p.nx + 1, lines);
    if (grid == 0) return cudaSuccess;
    cudaError_t e;
    constexpr size_t sm = pk_col_smem<Cfg::N, S>();
    if (pass == 1) {
        if ((e = set_smem<SmemTag<51, Cfg, S, MINB>>(k_y_fwd_pk<Cfg, S, MINB>, sm)) != cudaSuccess) return e;
        k_y_fwd_pk<Cfg, S, MINB><<<grid, NT, sm, st>>>(p);
    } else if (pass == 3) {
        if ((e = set_smem<SmemTag<53, Cfg, S, MINB>>(k_y_inv_pk<Cfg, S, MINB>, sm)) != cudaSuccess) return e;
        k_y_inv_pk<Cfg, S, MINB><<<grid, NT, sm, st>>>(p);
    } else {
        constexpr size_t smz = pk_col_smem_z<Cfg::N, S>();
        if ((e = set_smem<SmemTag<52, Cfg, S, MINB>>(k_z_conv_pk<Cfg, S, MINB>, smz)) != cudaSuccess) return e;
        k_z_conv_pk<Cfg, S, MINB><<<grid, NT, smz, st>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace pgb
