// poisson_solve_unfused: the plain FP32 pipeline, kept as the yardstick for
// what the pruned and fused passes buy.
//
// It is the convolution method of Section 3 written the straightforward way,
// with this library's own line transforms: the padded M^3 grid (M = 2n per
// axis) is materialised as complex values, transformed along x, y and z in
// three separate passes of full length-M FFTs, multiplied by the transformed
// Green's function in a pass of its own, transformed back along z, y and x,
// and cropped.  Nothing is pruned (the padding zeros are transformed, and all
// M^3 outputs of the inverse are computed) and nothing is fused.
//
// Layout: P[z][y][x], complex FP32, Mx My Mz elements, owned by the plan and
// allocated on the first call, with one W_2M twiddle table per axis.
#include <algorithm>

#include "configs.cuh"
#include "internal.h"
#include "plan.h"
#include "poisson.h"

namespace pgb {
namespace {

// line configuration of a full padded length M = 2n
template <int M> struct PlainCfg { using C = typename SizeCfg<float, M>::C; };
template <> struct PlainCfg<768> { using C = LineCfg<float, 768, 24, Radices<8, 12, 8>>; };
template <> struct PlainCfg<1024> { using C = LineCfg<float, 1024, 32, Radices<32, 32>>; };

template <int M> StageTwList plain_tw_list() { return stage_tw_list<M>(typename PlainCfg<M>::C::Rads{}); }
StageTwList plain_tw_list(int M) {
    switch (M) {
        case 32: return plain_tw_list<32>();
        case 64: return plain_tw_list<64>();
        case 96: return plain_tw_list<96>();
        case 128: return plain_tw_list<128>();
        case 192: return plain_tw_list<192>();
        case 256: return plain_tw_list<256>();
        case 384: return plain_tw_list<384>();
        case 512: return plain_tw_list<512>();
        case 768: return plain_tw_list<768>();
        case 1024: return plain_tw_list<1024>();
        default: return StageTwList{};
    }
}

// W_2M^j = exp(-i pi j / M), j < 2M, from the FP64 sincospi, rounded once.
__global__ void k_unf_twiddles(cpx<float>* __restrict__ tw, int M) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < 2 * M; j += gridDim.x * blockDim.x) {
        double s, c;
        sincospi((double)j / (double)M, &s, &c);
        tw[j] = cpx<float>{(float)c, (float)-s};
    }
}

// P = rho zero-padded to M^3, as complex values
__global__ void k_unf_pad(cpx<float>* __restrict__ P, const float* __restrict__ rho, int nx, int ny, int nz,
                          int Mx, int My, long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % Mx);
        const long long r = i / Mx;
        const int y = (int)(r % My), z = (int)(r / My);
        const float v = (x < nx && y < ny && z < nz) ? rho[((long long)z * ny + y) * nx + x] : 0.0f;
        P[i] = cpx<float>{v, 0.0f};
    }
}

// P *= Ghat(fold(kx), fold(ky), fold(kz)), fold(k) = min(k, M - k)
__global__ void k_unf_mul(cpx<float>* __restrict__ P, const float* __restrict__ g, int nx, int ny, int Mx, int My,
                          int Mz, long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int kx = (int)(i % Mx);
        const long long r = i / Mx;
        const int ky = (int)(r % My), kz = (int)(r / My);
        const int fx = min(kx, Mx - kx), fy = min(ky, My - ky), fz = min(kz, Mz - kz);
        P[i] = scale(P[i], g[greens_index<float>(fx, fy, fz, nx, Mz / 2)]);
    }
}

// phi = Re P on the user grid (the inverse's 1/(Mx My Mz) is in Ghat)
__global__ void k_unf_crop(float* __restrict__ phi, const cpx<float>* __restrict__ P, int nx, int ny, int Mx, int My,
                           long long total) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int x = (int)(i % nx);
        const long long r = i / nx;
        const int y = (int)(r % ny), z = (int)(r / ny);
        phi[i] = P[((long long)z * My + y) * Mx + x].x;
    }
}

// FFT of the rows of P (length M = Mx, contiguous): ROWS rows per CTA,
// thread = (t, row) with t fastest so that a warp reads whole row segments.
template <class Cfg, int ROWS, bool INV>
__global__ void __launch_bounds__(ROWS * Cfg::T) k_unf_rows(cpx<float>* __restrict__ P, const cpx<float>* tw,
                                                            long long nrows) {
    constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T;
    constexpr int LS = N + N / 16;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<float>* sm = reinterpret_cast<cpx<float>*>(smem_raw);
    const int t = threadIdx.x % T, r = threadIdx.x / T;
    const long long row = (long long)blockIdx.x * ROWS + r;
    const bool valid = row < nrows;
    cpx<float>* line = P + row * N;
    cpx<float> v[1][E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[0][m] = valid ? line[t + T * m] : cpx<float>{0, 0};
    const LineSmem<float> ls[1] = {{sm + r * LS, 1, 4, 1}};
    line_fft<float, N, E, INV, 1>(v, t, ls, tw, typename Cfg::Rads{});
    if (valid) {
#pragma unroll
        for (int m = 0; m < E; ++m) line[t + T * m] = v[0][m];
    }
}

// FFT of strided columns of P: element i of line (x, o) at
// P[o * outer + x + i * stride]; SLOTS adjacent x per CTA, slot fastest.
template <class Cfg, int SLOTS, bool INV>
__global__ void __launch_bounds__(SLOTS * Cfg::T) k_unf_cols(cpx<float>* __restrict__ P, const cpx<float>* tw,
                                                             int Mx, long long stride, long long outer) {
    constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<float>* sm = reinterpret_cast<cpx<float>*>(smem_raw);
    const int slot = threadIdx.x % SLOTS, t = threadIdx.x / SLOTS;
    const int xt = Mx / SLOTS;
    const int x = (int)(blockIdx.x % xt) * SLOTS + slot;
    const long long o = blockIdx.x / xt;
    cpx<float>* line = P + o * outer + x + (long long)t * stride;
    cpx<float> v[1][E];
#pragma unroll
    for (int m = 0; m < E; ++m) v[0][m] = line[(long long)(T * m) * stride];
    const LineSmem<float> ls[1] = {col_line<float, N, SLOTS>(sm, 0, slot)};
    line_fft<float, N, E, INV, 1>(v, t, ls, tw, typename Cfg::Rads{});
#pragma unroll
    for (int m = 0; m < E; ++m) line[(long long)(T * m) * stride] = v[0][m];
}

template <class Cfg> constexpr int unf_rows_per_cta() { return Cfg::T >= 128 ? 1 : 128 / Cfg::T; }
template <class Cfg> constexpr int unf_slots() { return Cfg::T >= 32 ? 8 : 16; }

template <class Cfg, bool INV> cudaError_t unf_rows(cpx<float>* P, const cpx<float>* tw, long long nrows, cudaStream_t st) {
    constexpr int ROWS = unf_rows_per_cta<Cfg>();
    constexpr size_t sm = (size_t)ROWS * (Cfg::N + Cfg::N / 16) * sizeof(cpx<float>);
    auto k = k_unf_rows<Cfg, ROWS, INV>;
    cudaError_t e = set_smem<SmemTag<60 + INV, Cfg, ROWS, 0>>(k, sm);
    if (e != cudaSuccess) return e;
    const long long grid = (nrows + ROWS - 1) / ROWS;
    k<<<(unsigned)grid, ROWS * Cfg::T, sm, st>>>(P, tw, nrows);
    return cudaGetLastError();
}

template <class Cfg, bool INV>
cudaError_t unf_cols(cpx<float>* P, const cpx<float>* tw, int Mx, long long stride, long long outer, long long nouter,
                     cudaStream_t st) {
    constexpr int S = unf_slots<Cfg>();
    constexpr size_t sm = (size_t)col_rows<float, Cfg::N, S>() * S * sizeof(cpx<float>);
    auto k = k_unf_cols<Cfg, S, INV>;
    cudaError_t e = set_smem<SmemTag<62 + INV, Cfg, S, 0>>(k, sm);
    if (e != cudaSuccess) return e;
    const long long grid = (long long)(Mx / S) * nouter;
    k<<<(unsigned)grid, S * Cfg::T, sm, st>>>(P, tw, Mx, stride, outer);
    return cudaGetLastError();
}

// axis 0: rows (x); axis 1, 2: columns (y, z)
template <int M>
cudaError_t unf_axis_m(int axis, bool inv, cpx<float>* P, const cpx<float>* tw, int Mx, int My, int Mz,
                       cudaStream_t st) {
    using C = typename PlainCfg<M>::C;
    const long long plane = (long long)Mx * My;
    if (axis == 0) {
        const long long rows = (long long)My * Mz;
        return inv ? unf_rows<C, true>(P, tw, rows, st) : unf_rows<C, false>(P, tw, rows, st);
    }
    if (axis == 1)  // lines (x, z): stride Mx, outer z
        return inv ? unf_cols<C, true>(P, tw, Mx, Mx, plane, Mz, st) : unf_cols<C, false>(P, tw, Mx, Mx, plane, Mz, st);
    // lines (x, y): stride Mx My, outer y
    return inv ? unf_cols<C, true>(P, tw, Mx, plane, Mx, My, st) : unf_cols<C, false>(P, tw, Mx, plane, Mx, My, st);
}

cudaError_t unf_axis(int M, int axis, bool inv, cpx<float>* P, const cpx<float>* tw, int Mx, int My, int Mz,
                     cudaStream_t st) {
    switch (M) {
        case 32: return unf_axis_m<32>(axis, inv, P, tw, Mx, My, Mz, st);
        case 64: return unf_axis_m<64>(axis, inv, P, tw, Mx, My, Mz, st);
        case 96: return unf_axis_m<96>(axis, inv, P, tw, Mx, My, Mz, st);
        case 128: return unf_axis_m<128>(axis, inv, P, tw, Mx, My, Mz, st);
        case 192: return unf_axis_m<192>(axis, inv, P, tw, Mx, My, Mz, st);
        case 256: return unf_axis_m<256>(axis, inv, P, tw, Mx, My, Mz, st);
        case 384: return unf_axis_m<384>(axis, inv, P, tw, Mx, My, Mz, st);
        case 512: return unf_axis_m<512>(axis, inv, P, tw, Mx, My, Mz, st);
        case 768: return unf_axis_m<768>(axis, inv, P, tw, Mx, My, Mz, st);
        case 1024: return unf_axis_m<1024>(axis, inv, P, tw, Mx, My, Mz, st);
        default: return cudaErrorInvalidValue;
    }
}

poisson_status to_status(cudaError_t e) {
    if (e == cudaSuccess) return POISSON_OK;
    if (e == cudaErrorMemoryAllocation) return POISSON_ERR_ALLOC;
    return POISSON_ERR_CUDA;
}

// the plan's padded buffer and per-axis tables, made on the first call
cudaError_t unf_prepare(poisson_plan_s* pl, cudaStream_t st) {
    if (pl->unf_buf) return cudaSuccess;
    const int M[3] = {2 * pl->nx, 2 * pl->ny, 2 * pl->nz};
    cudaError_t e;
    for (int a = 0; a < 3; ++a) {
        const StageTwList L = plain_tw_list(M[a]);
        if (L.total == 0) return cudaErrorInvalidValue;
        if ((e = cudaMalloc(&pl->unf_tw[a], (size_t)L.total * sizeof(cpx<float>))) != cudaSuccess) return e;
        cpx<float>* tw = static_cast<cpx<float>*>(pl->unf_tw[a]);
        k_unf_twiddles<<<(2 * M[a] + 255) / 256, 256, 0, st>>>(tw, M[a]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = fill_stage_twiddles_list(tw, M[a], L, st)) != cudaSuccess) return e;
    }
    return cudaMalloc(&pl->unf_buf, (size_t)M[0] * M[1] * M[2] * sizeof(cpx<float>));
}

}  // namespace
}  // namespace pgb

extern "C" poisson_status poisson_solve_unfused(poisson_plan_t plan, const void* rho_dev, void* phi_dev,
                                                void* cuda_stream) {
    using namespace pgb;
    if (!plan || !rho_dev || !phi_dev) return POISSON_ERR_ARG;
    if (((reinterpret_cast<uintptr_t>(rho_dev) | reinterpret_cast<uintptr_t>(phi_dev)) & 15u) != 0)
        return POISSON_ERR_ARG;
    if (plan->prec != POISSON_FP32) return POISSON_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    cudaError_t e = unf_prepare(plan, st);
    if (e != cudaSuccess) return to_status(e);
    const int nx = plan->nx, ny = plan->ny, nz = plan->nz;
    const int Mx = 2 * nx, My = 2 * ny, Mz = 2 * nz;
    const int M[3] = {Mx, My, Mz};
    const long long total = (long long)Mx * My * Mz;
    cpx<float>* P = static_cast<cpx<float>*>(plan->unf_buf);
    const unsigned grid = 152u * 16u;  // grid-stride element passes
    k_unf_pad<<<grid, 256, 0, st>>>(P, static_cast<const float*>(rho_dev), nx, ny, nz, Mx, My, total);
    if ((e = cudaGetLastError()) != cudaSuccess) return to_status(e);
    for (int a = 0; a < 3; ++a)
        if ((e = unf_axis(M[a], a, false, P, static_cast<const cpx<float>*>(plan->unf_tw[a]), Mx, My, Mz, st)) !=
            cudaSuccess)
            return to_status(e);
    k_unf_mul<<<grid, 256, 0, st>>>(P, static_cast<const float*>(plan->greens), nx, ny, Mx, My, Mz, total);
    if ((e = cudaGetLastError()) != cudaSuccess) return to_status(e);
    for (int a = 2; a >= 0; --a)
        if ((e = unf_axis(M[a], a, true, P, static_cast<const cpx<float>*>(plan->unf_tw[a]), Mx, My, Mz, st)) !=
            cudaSuccess)
            return to_status(e);
    k_unf_crop<<<grid, 256, 0, st>>>(static_cast<float*>(phi_dev), P, nx, ny, Mx, My, (long long)nx * ny * nz);
    return to_status(cudaGetLastError());
}
