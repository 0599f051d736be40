// The five passes of the free-space Poisson solve Phi = G * rho by zero-padded
// FFT convolution (the convolution method of the paper's case study,
// Section 3): pad + R2C along x, pad + C2C along y, [pad + FFT along z,
// multiply by the transformed Green's function, inverse FFT along z, crop],
// inverse C2C along y + crop, C2R along x + crop.
//
// Padding is M = 2n per axis and is never materialised.  A length-2n
// transform of a sequence that is zero beyond n splits into two length-n
// transforms: X[2k] = FFT_n(x)[k] and X[2k+1] = FFT_n(x_j W_2n^j)[k]; the
// cropped inverse is x[j] = IFFT_n(X_even)[j] + W_2n^-j IFFT_n(X_odd)[j]
// for j < n.  The even and odd halves are stored as separate blocks of rows
// ("parity-major"), so no pass ever interleaves them.  The x axis packs two
// real rows into one complex line (a + i b) and separates their spectra with
// the Hermitian pairing of k and 2n - k.
//
// Layout (complex elements, x fastest):
//   W1[z][y][kx]        z < nz, y < ny,  kx <= nx   row stride sx
//   W2[z][q*ny + k][kx] z < nz, q in {0,1} parity of ky = 2k + q, row stride sx
//   Ghat[kz][ky][kx]    octant (nz+1)(ny+1)(nx+1) of the real, even transformed
//                       Green's function, scaled by -G V / (Mx My Mz)
#pragma once

#include "fft_core.cuh"

namespace pgb {

template <class R_, int N_, int E_, class Rads_> struct LineCfg {
    using R = R_;
    static constexpr int N = N_;
    static constexpr int E = E_;
    static constexpr int T = N_ / E_;
    using Rads = Rads_;
    static_assert(N_ % E_ == 0, "E must divide N");
};

template <class R> struct PassParams {
    const void* in;
    void* out;
    const R* greens;          // octant, z-pass only
    const cpx<R>* tw;         // W_{2N}^j, j < 2N, for this pass's axis
    int nx, ny, nz;
    long long sx;             // complex row stride of W1/W2
    unsigned* status;         // device status word (unused by these passes)
};

// bytes of one 128-byte segment in complex elements
template <class R> struct Seg { static constexpr int XW = 128 / (int)sizeof(cpx<R>); };

// ==========================================================================
// Column passes (y and z axes; lines are strided, tiles span x)
// ==========================================================================
//
// Thread layout: slot = tid % SLOTS (fastest), t = tid / SLOTS.  "Wide"
// tiles map slot -> (kx = x0 + slot % XW, other = o0 + slot / XW), so 16
// (FP32) or 8 (FP64) consecutive lanes read one 128-byte segment of a row.
// Columns beyond the last full segment (the Nyquist column kx = nx when nx
// is a multiple of XW) go to "narrow" tiles: slot -> other index.

template <class R, int SLOTS> struct ColTile {
    int kx;
    int other;
    bool valid;
};

template <class R, int SLOTS>
__device__ __forceinline__ ColTile<R, SLOTS> col_tile(int ncols, int L, int slot) {
    constexpr int XW = Seg<R>::XW;
    constexpr int NLW = SLOTS / XW;
    const int nxw = ncols / XW;
    const int wide_l = (L + NLW - 1) / NLW;
    const int n_wide = nxw * wide_l;
    ColTile<R, SLOTS> c;
    int b = blockIdx.x;
    if (b < n_wide) {
        const int xt = b % nxw, lt = b / nxw;
        c.kx = xt * XW + slot % XW;
        c.other = lt * NLW + slot / XW;
    } else {
        b -= n_wide;
        const int nleft = ncols - nxw * XW;
        const int cc = b % nleft, lt = b / nleft;
        c.kx = nxw * XW + cc;
        c.other = lt * SLOTS + slot;
    }
    c.valid = c.other < L;
    return c;
}

template <class R, int SLOTS>
inline int col_grid(int ncols, int L) {
    constexpr int XW = Seg<R>::XW;
    constexpr int NLW = SLOTS / XW;
    const int nxw = ncols / XW;
    const int nleft = ncols - nxw * XW;
    return nxw * ((L + NLW - 1) / NLW) + nleft * ((L + SLOTS - 1) / SLOTS);
}

// pass 1: pad + forward FFT along y.  W1 -> W2.
template <class Cfg, int SLOTS>
__global__ void __launch_bounds__(SLOTS * Cfg::T)
k_y_fwd(PassParams<typename Cfg::R> p) {
    using R = typename Cfg::R;
    constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
    const int slot = threadIdx.x % SLOTS, t = threadIdx.x / SLOTS;
    const int ny = p.ny, nz = p.nz;
    const ColTile<R, SLOTS> c = col_tile<R, SLOTS>(p.nx + 1, nz, slot);
    const cpx<R>* __restrict__ in = static_cast<const cpx<R>*>(p.in);
    cpx<R>* __restrict__ out = static_cast<cpx<R>*>(p.out);
    const long long sx = p.sx;

    cpx<R> v[2][E];
    const long long ibase = (long long)c.other * ny * sx + c.kx;
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int j = t + T * m;
        v[0][m] = c.valid ? in[ibase + (long long)j * sx] : cpx<R>{0, 0};
    }
#pragma unroll
    for (int m = 0; m < E; ++m) v[1][m] = cmul(v[0][m], ldg_c(p.tw + t + T * m));

    const LineSmem<R> ls[2] = {{sm + slot, SLOTS, 30, 0}, {sm + N * SLOTS + slot, SLOTS, 30, 0}};
    line_fft<R, N, E, false, 2>(v, t, ls, p.tw, typename Cfg::Rads{});

    if (c.valid) {
        const long long obase = (long long)c.other * 2 * ny * sx + c.kx;
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int m = 0; m < E; ++m)
                out[obase + (long long)(q * ny + t + T * m) * sx] = v[q][m];
    }
}

// pass 2: pad + FFT along z, multiply by Ghat, inverse FFT along z, crop.
// In place on W2.  Ghat is real (the kernel is real and even), so the
// adjoint's conj(Ghat) is the same multiply.
template <class Cfg, int SLOTS>
__global__ void __launch_bounds__(SLOTS * Cfg::T)
k_z_conv(PassParams<typename Cfg::R> p) {
    using R = typename Cfg::R;
    constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
    const int slot = threadIdx.x % SLOTS, t = threadIdx.x / SLOTS;
    const int nx = p.nx, ny = p.ny;
    const ColTile<R, SLOTS> c = col_tile<R, SLOTS>(nx + 1, 2 * ny, slot);
    cpx<R>* __restrict__ w = static_cast<cpx<R>*>(p.out);
    const long long sx = p.sx;
    const long long plane = 2LL * ny * sx;

    cpx<R> v[2][E];
    const long long base = (long long)c.other * sx + c.kx;
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int j = t + T * m;
        v[0][m] = c.valid ? w[base + (long long)j * plane] : cpx<R>{0, 0};
    }
#pragma unroll
    for (int m = 0; m < E; ++m) v[1][m] = cmul(v[0][m], ldg_c(p.tw + t + T * m));

    const LineSmem<R> ls[2] = {{sm + slot, SLOTS, 30, 0}, {sm + N * SLOTS + slot, SLOTS, 30, 0}};
    line_fft<R, N, E, false, 2>(v, t, ls, p.tw, typename Cfg::Rads{});

    // Green's multiply: frequency (kx, ky, kz), folded into the octant.
    {
        const int kys = c.other;
        const int ky = kys < ny ? 2 * kys : 2 * (kys - ny) + 1;
        const int kyf = ky <= ny ? ky : 2 * ny - ky;
        const R* __restrict__ g = p.greens + (long long)kyf * (nx + 1) + c.kx;
        const long long gz = (long long)(ny + 1) * (nx + 1);
#pragma unroll
        for (int q = 0; q < 2; ++q)
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const int kz = 2 * (t + T * m) + q;
                const int kzf = kz <= N ? kz : 2 * N - kz;
                const R gv = c.valid ? __ldg(g + kzf * gz) : (R)0;
                v[q][m] = scale(v[q][m], gv);
            }
    }

    line_fft<R, N, E, true, 2>(v, t, ls, p.tw, typename Cfg::Rads{});

    if (c.valid) {
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int j = t + T * m;
            w[base + (long long)j * plane] = v[0][m] + cmulc(v[1][m], ldg_c(p.tw + j));
        }
    }
}

// pass 3: inverse FFT along y + crop.  W2 -> W1.
template <class Cfg, int SLOTS>
__global__ void __launch_bounds__(SLOTS * Cfg::T)
k_y_inv(PassParams<typename Cfg::R> p) {
    using R = typename Cfg::R;
    constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
    const int slot = threadIdx.x % SLOTS, t = threadIdx.x / SLOTS;
    const int ny = p.ny, nz = p.nz;
    const ColTile<R, SLOTS> c = col_tile<R, SLOTS>(p.nx + 1, nz, slot);
    const cpx<R>* __restrict__ in = static_cast<const cpx<R>*>(p.in);
    cpx<R>* __restrict__ out = static_cast<cpx<R>*>(p.out);
    const long long sx = p.sx;

    cpx<R> v[2][E];
    const long long ibase = (long long)c.other * 2 * ny * sx + c.kx;
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int m = 0; m < E; ++m)
            v[q][m] = c.valid ? in[ibase + (long long)(q * ny + t + T * m) * sx] : cpx<R>{0, 0};

    const LineSmem<R> ls[2] = {{sm + slot, SLOTS, 30, 0}, {sm + N * SLOTS + slot, SLOTS, 30, 0}};
    line_fft<R, N, E, true, 2>(v, t, ls, p.tw, typename Cfg::Rads{});

    if (c.valid) {
        const long long obase = (long long)c.other * ny * sx + c.kx;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int j = t + T * m;
            out[obase + (long long)j * sx] = v[0][m] + cmulc(v[1][m], ldg_c(p.tw + j));
        }
    }
}

// ==========================================================================
// Row passes (x axis; lines are contiguous rows, two real rows per line)
// ==========================================================================
//
// Thread layout: t = tid % T (fastest), pair = tid / T.  A tile holds PAIRS
// row pairs, i.e. 2*PAIRS consecutive rows, which are contiguous in rho/phi.

template <class R> struct RowPad { static constexpr int SHIFT = sizeof(R) == 4 ? 4 : 3; };

template <class Cfg> constexpr int row_line_stride() {
    return Cfg::N + (Cfg::N >> RowPad<typename Cfg::R>::SHIFT);
}

// pass 0: pad + R2C along x.  rho (real rows of nx) -> W1 (nx+1 bins).
template <class Cfg, int PAIRS>
__global__ void __launch_bounds__(PAIRS * Cfg::T)
k_x_fwd(PassParams<typename Cfg::R> p, int rows) {
    using R = typename Cfg::R;
    constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T;
    constexpr int LS = row_line_stride<Cfg>();
    constexpr int SH = RowPad<R>::SHIFT;
    constexpr int NT = PAIRS * T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    R* stage = reinterpret_cast<R*>(smem_raw);
    cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
    const int t = threadIdx.x % T, pr = threadIdx.x / T;
    const int r0 = blockIdx.x * 2 * PAIRS;
    const int nrows = min(2 * PAIRS, rows - r0);
    const R* __restrict__ in = static_cast<const R*>(p.in) + (long long)r0 * N;
    cpx<R>* __restrict__ out = static_cast<cpx<R>*>(p.out);

    // stage the tile's rows (contiguous in rho) with 16-byte loads
    {
        using V = typename std::conditional<sizeof(R) == 4, float4, double2>::type;
        constexpr int VW = 16 / sizeof(R);
        const int nvec = nrows * N / VW;
        const V* __restrict__ src = reinterpret_cast<const V*>(in);
        V* dst = reinterpret_cast<V*>(stage);
        for (int i = threadIdx.x; i < nvec; i += NT) dst[i] = __ldg(src + i);
    }
    __syncthreads();
    cpx<R> v[2][E];
    const bool has_a = 2 * pr < nrows, has_b = 2 * pr + 1 < nrows;
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int j = t + T * m;
        const R a = has_a ? stage[(2 * pr) * N + j] : (R)0;
        const R b = has_b ? stage[(2 * pr + 1) * N + j] : (R)0;
        v[0][m] = {a, b};
    }
    __syncthreads();  // the staging area becomes the line buffers
#pragma unroll
    for (int m = 0; m < E; ++m) v[1][m] = cmul(v[0][m], ldg_c(p.tw + t + T * m));

    const LineSmem<R> ls[2] = {{sm + (0 * PAIRS + pr) * LS, 1, SH, 1},
                               {sm + (1 * PAIRS + pr) * LS, 1, SH, 1}};
    line_fft<R, N, E, false, 2>(v, t, ls, p.tw, typename Cfg::Rads{});
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int m = 0; m < E; ++m) ls[q][t + T * m] = v[q][m];
    __syncthreads();

    // separate the two rows' spectra: A[k] = (Z[k] + conj Z[2N-k]) / 2,
    // B[k] = -i (Z[k] - conj Z[2N-k]) / 2, k = 0..N; Z[2k'] = E[k'],
    // Z[2k'+1] = O[k'].
    const long long sx = p.sx;
    const int nout = nrows * (N + 1);
    for (int i = threadIdx.x; i < nout; i += NT) {
        const int s = i / (N + 1), k = i - s * (N + 1);
        const int pp = s >> 1;
        cpx<R> P, Q;
        if ((k & 1) == 0) {
            const int kh = k >> 1;
            const LineSmem<R> e = {sm + pp * LS, 1, SH, 1};
            P = e[kh];
            Q = e[kh == 0 ? 0 : N - kh];
        } else {
            const int kh = k >> 1;
            const LineSmem<R> o = {sm + (PAIRS + pp) * LS, 1, SH, 1};
            P = o[kh];
            Q = o[N - 1 - kh];
        }
        Q.y = -Q.y;
        cpx<R> r;
        if ((s & 1) == 0) r = {(R)0.5 * (P.x + Q.x), (R)0.5 * (P.y + Q.y)};
        else r = {(R)0.5 * (P.y - Q.y), (R)(-0.5) * (P.x - Q.x)};
        out[(long long)(r0 + s) * sx + k] = r;
    }
}

// pass 4: C2R along x + crop.  W1 (nx+1 bins) -> phi (real rows of nx).
template <class Cfg, int PAIRS>
__global__ void __launch_bounds__(PAIRS * Cfg::T)
k_x_inv(PassParams<typename Cfg::R> p, int rows) {
    using R = typename Cfg::R;
    constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T;
    constexpr int LS = row_line_stride<Cfg>();
    constexpr int SH = RowPad<R>::SHIFT;
    constexpr int NT = PAIRS * T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
    R* stage = reinterpret_cast<R*>(smem_raw);
    const int t = threadIdx.x % T, pr = threadIdx.x / T;
    const int r0 = blockIdx.x * 2 * PAIRS;
    const int nrows = min(2 * PAIRS, rows - r0);
    const cpx<R>* __restrict__ in = static_cast<const cpx<R>*>(p.in);
    const long long sx = p.sx;

    // stage the spectra rows: row s occupies [s*(N+1), (s+1)*(N+1))
    const int nin = nrows * (N + 1);
    for (int i = threadIdx.x; i < nin; i += NT) {
        const int s = i / (N + 1), k = i - s * (N + 1);
        sm[i] = in[(long long)(r0 + s) * sx + k];
    }
    __syncthreads();
    // Z[k] = A[k] + i B[k] with A[2N-k] = conj A[k] (same for B)
    cpx<R> v[2][E];
    const bool has_a = 2 * pr < nrows, has_b = 2 * pr + 1 < nrows;
    const cpx<R>* ra = sm + (2 * pr) * (N + 1);
    const cpx<R>* rb = sm + (2 * pr + 1) * (N + 1);
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int k = 2 * (t + T * m) + q;
            const bool lo = k <= N;
            const int kk = lo ? k : 2 * N - k;
            const cpx<R> a = has_a ? ra[kk] : cpx<R>{0, 0};
            const cpx<R> b = has_b ? rb[kk] : cpx<R>{0, 0};
            v[q][m] = lo ? cpx<R>{a.x - b.y, a.y + b.x} : cpx<R>{a.x + b.y, b.x - a.y};
        }
    __syncthreads();  // the staging area becomes the line buffers

    const LineSmem<R> ls[2] = {{sm + (0 * PAIRS + pr) * LS, 1, SH, 1},
                               {sm + (1 * PAIRS + pr) * LS, 1, SH, 1}};
    line_fft<R, N, E, true, 2>(v, t, ls, p.tw, typename Cfg::Rads{});
    __syncthreads();  // line buffers become the output staging area

    // z[j] = a[j] + W_2N^-j b[j]; real part -> row 2 pr, imaginary -> 2 pr + 1
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int j = t + T * m;
        const cpx<R> z = v[0][m] + cmulc(v[1][m], ldg_c(p.tw + j));
        stage[(2 * pr) * N + j] = z.x;
        stage[(2 * pr + 1) * N + j] = z.y;
    }
    __syncthreads();
    {
        using V = typename std::conditional<sizeof(R) == 4, float4, double2>::type;
        constexpr int VW = 16 / sizeof(R);
        const int nvec = nrows * N / VW;
        V* dst = reinterpret_cast<V*>(static_cast<R*>(p.out) + (long long)r0 * N);
        const V* src = reinterpret_cast<const V*>(stage);
        for (int i = threadIdx.x; i < nvec; i += NT) dst[i] = src[i];
    }
}

// ==========================================================================
// launch helpers
// ==========================================================================
template <class Cfg> constexpr int col_slots() {
    constexpr int XW = Seg<typename Cfg::R>::XW;
    constexpr int s = 256 / Cfg::T;
    return s < XW ? XW : s;
}
template <class Cfg> constexpr int row_pairs() {
    constexpr int s = 256 / Cfg::T;
    return s < 1 ? 1 : s;
}
template <class Cfg> constexpr size_t col_smem() {
    return 2ull * Cfg::N * col_slots<Cfg>() * sizeof(cpx<typename Cfg::R>);
}
template <class Cfg> constexpr size_t row_smem() {
    using R = typename Cfg::R;
    constexpr int P = row_pairs<Cfg>();
    constexpr size_t lines = 2ull * P * row_line_stride<Cfg>() * sizeof(cpx<R>);
    constexpr size_t stage_c = 2ull * P * (Cfg::N + 1) * sizeof(cpx<R>);
    constexpr size_t stage_r = 2ull * P * Cfg::N * sizeof(R);
    constexpr size_t m1 = lines > stage_c ? lines : stage_c;
    return m1 > stage_r ? m1 : stage_r;
}

template <class K> inline cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// pass ids: 0 x_fwd, 1 y_fwd, 2 z_conv, 3 y_inv, 4 x_inv
template <class Cfg>
cudaError_t launch_row(int pass, const PassParams<typename Cfg::R>& p, int rows, cudaStream_t st) {
    constexpr int P = row_pairs<Cfg>();
    constexpr size_t sm = row_smem<Cfg>();
    const int grid = (rows + 2 * P - 1) / (2 * P);
    if (grid == 0) return cudaSuccess;
    cudaError_t e;
    if (pass == 0) {
        e = set_smem(k_x_fwd<Cfg, P>, sm);
        if (e != cudaSuccess) return e;
        k_x_fwd<Cfg, P><<<grid, P * Cfg::T, sm, st>>>(p, rows);
    } else {
        e = set_smem(k_x_inv<Cfg, P>, sm);
        if (e != cudaSuccess) return e;
        k_x_inv<Cfg, P><<<grid, P * Cfg::T, sm, st>>>(p, rows);
    }
    return cudaGetLastError();
}

template <class Cfg>
cudaError_t launch_col(int pass, const PassParams<typename Cfg::R>& p, cudaStream_t st) {
    using R = typename Cfg::R;
    constexpr int S = col_slots<Cfg>();
    constexpr size_t sm = col_smem<Cfg>();
    const int L = pass == 2 ? 2 * p.ny : p.nz;
    const int grid = col_grid<R, S>(p.nx + 1, L);
    if (grid == 0) return cudaSuccess;
    cudaError_t e;
    if (pass == 1) {
        e = set_smem(k_y_fwd<Cfg, S>, sm);
        if (e != cudaSuccess) return e;
        k_y_fwd<Cfg, S><<<grid, S * Cfg::T, sm, st>>>(p);
    } else if (pass == 3) {
        e = set_smem(k_y_inv<Cfg, S>, sm);
        if (e != cudaSuccess) return e;
        k_y_inv<Cfg, S><<<grid, S * Cfg::T, sm, st>>>(p);
    } else {
        e = set_smem(k_z_conv<Cfg, S>, sm);
        if (e != cudaSuccess) return e;
        k_z_conv<Cfg, S><<<grid, S * Cfg::T, sm, st>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace pgb
