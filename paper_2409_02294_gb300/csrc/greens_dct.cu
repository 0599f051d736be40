// Plan-time DCT-I of the Green's kernel octant by FP64 FFTs, O(n^3 log n).
//
// Along an axis of edge n the octant holds k(d), d = 0..n, and the padded
// M = 2n transform of the even, real sequence it stands for is
//   K(q) = sum_{j=0}^{2n-1} x_j W_2n^{jq},  x_j = k(j) (j <= n), k(2n - j) (j > n),
// which is real and equals sum_d c_d k(d) cos(pi q d / n) (c_0 = c_n = 1,
// else 2): the DCT-I.  Splitting the 2n outputs by parity gives two
// length-n transforms of the folded sequences
//   a_j = k(j) + k(n - j),  b_j = (k(j) - k(n - j)) W_2n^j,   j = 0..n-1:
//   K(2q) = DFT_n(a)(q),    K(2q + 1) = DFT_n(b)(q),
// which the FP64 line transforms of fft_core.cuh run as two lines per
// thread (the column configuration's radices).  Only real parts are kept:
// K is real, so the imaginary parts are rounding noise.
#include <algorithm>

#include "configs.cuh"
#include "greens_dct.h"
#include "internal.h"

namespace pgb {
namespace {

// W_2n^j = exp(-i pi j / n), j < 2n, from the FP64 sincospi.
__global__ void k_dct_twiddles(cpx<double>* __restrict__ tw, int n) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < 2 * n; j += gridDim.x * blockDim.x) {
        double s, c;
        sincospi((double)j / (double)n, &s, &c);
        tw[j] = cpx<double>{c, -s};
    }
}

// One DCT-I per line: element d of line (o1, o2) at in[o1 s1 + o2 s2 + d se],
// d = 0..n; SLOTS lines of consecutive o1 per CTA (slot fastest across
// lanes), T = n / E threads per line.
template <class Cfg, int SLOTS>
__global__ void __launch_bounds__(SLOTS * Cfg::T) k_dct1_axis(const double* __restrict__ in, double* __restrict__ out,
                                                             const cpx<double>* __restrict__ tw, long long se,
                                                             long long s1, long long s2, int n1, long long nlines) {
    using R = double;
    constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
    const int slot = threadIdx.x % SLOTS, t = threadIdx.x / SLOTS;
    const long long line = (long long)blockIdx.x * SLOTS + slot;
    const bool valid = line < nlines;
    const long long base = valid ? (line % n1) * s1 + (line / n1) * s2 : 0;

    cpx<R> v[2][E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int j = t + T * m;  // < N
        R kj = 0.0, knj = 0.0;
        if (valid) {
            kj = in[base + j * se];
            knj = in[base + (N - j) * se];
        }
        const cpx<R> w = ldg_c(tw + j);
        const R b = kj - knj;
        v[0][m] = cpx<R>{kj + knj, 0.0};
        v[1][m] = cpx<R>{b * w.x, b * w.y};
    }
    const LineSmem<R> ls[2] = {col_line<R, N, SLOTS>(sm, 0, slot), col_line<R, N, SLOTS>(sm, 1, slot)};
    line_fft<R, N, E, false, 2>(v, t, ls, tw, typename Cfg::Rads{});
    if (valid) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int q = t + T * m;
            if (2 * q <= N) out[base + (long long)(2 * q) * se] = v[0][m].x;
            if (2 * q + 1 < N) out[base + (long long)(2 * q + 1) * se] = v[1][m].x;
        }
    }
}

template <int N>
cudaError_t dct1_axis_n(const double* in, double* out, const cpx<double>* tw, long long se, long long s1,
                        long long s2, int n1, long long nlines, cudaStream_t st) {
    using C = typename SizeCfg<double, N>::C;
    constexpr int S = 128 / C::T < 4 ? 4 : 128 / C::T;
    constexpr size_t sm = 2ull * col_rows<double, N, S>() * S * sizeof(cpx<double>);
    auto k = k_dct1_axis<C, S>;
    cudaError_t e = set_smem<SmemTag<70, C, S, 0>>(k, sm);
    if (e != cudaSuccess) return e;
    const long long grid = (nlines + S - 1) / S;
    k<<<(unsigned)grid, S * C::T, sm, st>>>(in, out, tw, se, s1, s2, n1, nlines);
    return cudaGetLastError();
}

cudaError_t dct1_axis(int n, const double* in, double* out, const cpx<double>* tw, long long se, long long s1,
                      long long s2, int n1, long long nlines, cudaStream_t st) {
    switch (n) {
        case 16: return dct1_axis_n<16>(in, out, tw, se, s1, s2, n1, nlines, st);
        case 32: return dct1_axis_n<32>(in, out, tw, se, s1, s2, n1, nlines, st);
        case 48: return dct1_axis_n<48>(in, out, tw, se, s1, s2, n1, nlines, st);
        case 64: return dct1_axis_n<64>(in, out, tw, se, s1, s2, n1, nlines, st);
        case 96: return dct1_axis_n<96>(in, out, tw, se, s1, s2, n1, nlines, st);
        case 128: return dct1_axis_n<128>(in, out, tw, se, s1, s2, n1, nlines, st);
        case 192: return dct1_axis_n<192>(in, out, tw, se, s1, s2, n1, nlines, st);
        case 256: return dct1_axis_n<256>(in, out, tw, se, s1, s2, n1, nlines, st);
        case 384: return dct1_axis_n<384>(in, out, tw, se, s1, s2, n1, nlines, st);
        case 512: return dct1_axis_n<512>(in, out, tw, se, s1, s2, n1, nlines, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

size_t dct1_twiddle_entries(int n) { return (size_t)axis_tw_list<double>(n, false).total; }

cudaError_t dct1_octant(double* k, double* tmp, cpx<double>* const tw[3], int nx, int ny, int nz, cudaStream_t st) {
    const int n[3] = {nx, ny, nz};
    cudaError_t e;
    for (int a = 0; a < 3; ++a) {
        k_dct_twiddles<<<(2 * n[a] + 255) / 256, 256, 0, st>>>(tw[a], n[a]);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = fill_stage_twiddles<double>(tw[a], n[a], false, st)) != cudaSuccess) return e;
    }
    const long long ex = nx + 1, ey = ny + 1, ez = nz + 1;
    // x: lines (y, z), elements contiguous; k -> tmp
    if ((e = dct1_axis(nx, k, tmp, tw[0], 1, ex, ex * ey, (int)ey, ey * ez, st)) != cudaSuccess) return e;
    // y: lines (x, z); tmp -> k
    if ((e = dct1_axis(ny, tmp, k, tw[1], ex, 1, ex * ey, (int)ex, ex * ez, st)) != cudaSuccess) return e;
    // z: lines (x, y); k -> tmp
    return dct1_axis(nz, k, tmp, tw[2], ex * ey, 1, ex, (int)ex, ex * ey, st);
}

}  // namespace pgb
