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
//   Ghat(kx, ky, kz)    octant (nz+1)(ny+1)(nx+1) of the real, even transformed
//                       Green's function, scaled by -G V / (Mx My Mz), in
//                       blocks of 64 bytes of kx by all kz (greens_layout.h)
#pragma once

#include <cstdlib>

#include "fft_core.cuh"
#include "greens_layout.h"
#include "tma.cuh"

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
    int tile0;                // first tile of this launch (column passes)
    int ntile;                // tiles in this launch, 0 = all
    int check_finite;         // x inverse: set bit 0 of *status if an output is not finite
};

// Record a non-finite output in the status word (POISSON_FLAG_CHECK_FINITE).
template <class R> __device__ __forceinline__ bool not_finite(R v) { return !isfinite(v); }
__device__ __forceinline__ void flag_non_finite(unsigned* status, bool bad) {
    if (bad && status) atomicOr(status, 1u);
}

// bytes of one 128-byte segment in complex elements
template <class R> struct Seg { static constexpr int XW = 128 / (int)sizeof(cpx<R>); };

// ==========================================================================
// Column passes (y and z axes; lines are strided, tiles span x)
// ==========================================================================
//
// Tiles: "wide" tiles map slot -> (kx = x0 + slot % XW, other = o0 + slot /
// XW), so XW consecutive lanes read one row segment of up to 128 bytes.
// Tiles are numbered chunk-major (all line groups of one band of XW columns,
// then the next band), so a range of columns is a contiguous range of tiles.
// Columns beyond the last full segment (the Nyquist column kx = nx when nx
// is a multiple of XW) go to "narrow" tiles: slot -> other index.

template <class R, int SLOTS> struct ColTile {
    int kx;
    int other;
    bool valid;
};

template <class R, int SLOTS>
__device__ __forceinline__ ColTile<R, SLOTS> col_tile(int ncols, int L, int slot, int tile) {
    constexpr int XW = SLOTS < Seg<R>::XW ? SLOTS : Seg<R>::XW;
    constexpr int NLW = SLOTS / XW;
    const int nxw = ncols / XW;
    const int wide_l = (L + NLW - 1) / NLW;
    const int n_wide = nxw * wide_l;
    ColTile<R, SLOTS> c;
    int b = tile;
    if (b < n_wide) {  // chunk-major: all line groups of band xt, then band xt + 1
        const int xt = b / wide_l, lt = b - xt * wide_l;
        c.kx = xt * XW + slot % XW;
        c.other = lt * NLW + slot / XW;
    } else {
        b -= n_wide;
        const int narrow_l = (L + SLOTS - 1) / SLOTS;
        const int cc = b / narrow_l, lt = b - cc * narrow_l;
        c.kx = nxw * XW + cc;
        c.other = lt * SLOTS + slot;
    }
    c.valid = c.other < L;
    return c;
}

template <class R, int SLOTS>
inline int col_grid(int ncols, int L) {
    constexpr int XW = SLOTS < Seg<R>::XW ? SLOTS : Seg<R>::XW;
    constexpr int NLW = SLOTS / XW;
    const int nxw = ncols / XW;
    const int nleft = ncols - nxw * XW;
    return nxw * ((L + NLW - 1) / NLW) + nleft * ((L + SLOTS - 1) / SLOTS);
}

// Column kernels: thread = (slot, t[, q]) with slot fastest, then t (the
// position within the line).  LPT = 2: a thread carries both halves of its
// column (X[2k] and X[2k+1] of the padded transform); LPT = 1: the halves go
// to two thread groups (q = tid / (SLOTS T)) that meet through shared memory
// for the final combine.

// Exchange-buffer layout of a column tile: element i of a line lives in row
// i (+ one padding row every 16 rows when a row is narrower than 128 bytes,
// which spreads the stride-16 row patterns of the first Stockham stage over
// all banks instead of one part of them).
template <class R, int SLOTS> struct ColPad {
    static constexpr bool on = SLOTS * (int)sizeof(cpx<R>) < 128;
    static constexpr int shift = on ? 4 : 30;
    static constexpr int pad = on ? SLOTS : 0;
};
template <class R, int N, int SLOTS> constexpr int col_rows() {
    return N + (ColPad<R, SLOTS>::on ? N / 16 : 0);
}
template <class R, int N, int SLOTS>
__device__ __forceinline__ LineSmem<R> col_line(cpx<R>* sm, int half, int slot) {
    return {sm + half * col_rows<R, N, SLOTS>() * SLOTS + slot, SLOTS, ColPad<R, SLOTS>::shift,
            ColPad<R, SLOTS>::pad};
}

// Asynchronous global -> shared copy of one real value (4 or 8 bytes); it
// has landed once cp.async.wait_group 0 returns in the issuing thread.
template <class R> __device__ __forceinline__ void cp_async_real(R* smem, const R* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (sizeof(R) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

template <class Cfg, int SLOTS, int LPT> struct ColIds {
    int slot, t, q;
    __device__ __forceinline__ ColIds() {
        slot = threadIdx.x % SLOTS;
        const int rest = threadIdx.x / SLOTS;
        t = rest % Cfg::T;
        q = LPT == 1 ? rest / Cfg::T : 0;
    }
    // half carried in register line l
    __device__ __forceinline__ int half(int l) const { return LPT == 2 ? l : q; }
};

template <class Cfg, int SLOTS, int LPT> constexpr int col_threads() {
    return (LPT == 1 ? 2 : 1) * SLOTS * Cfg::T;
}

// Where a column tile's input comes from: straight from global memory
// (ColFromGlobal) or from a copy of the tile in shared memory that a TMA load
// placed there (ColFromSmem: element of tile row r at base[r * stride]).
// The hook runs right after the inputs are in registers; the TMA kernel
// uses it to start loading its next tile into the same buffer.
// TW_SMEM: the tile's p.tw points to a copy of the axis twiddle table in
// shared memory (the persistent TMA kernels), read with shared loads.
struct ColFromGlobal {
    static constexpr bool TW_SMEM = false;
};
template <class R> struct ColFromSmem {
    static constexpr bool TW_SMEM = true;
    const cpx<R>* base;
    int stride;
};
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};
template <bool CG, class R>
__device__ __forceinline__ cpx<R> col_in(const ColFromGlobal&, const cpx<R>* g, int) {
    return ld_c<CG>(g);
}
template <bool CG, class R>
__device__ __forceinline__ cpx<R> col_in(const ColFromSmem<R>& s, const cpx<R>*, int row) {
    return s.base[row * s.stride];
}

// Transform the LPT register lines of a column thread (forward or inverse).
// SEQ (two lines per thread): the even and odd halves go one after the other
// through the first exchange buffer, so the tile needs one buffer instead of
// two (each transform's last shared-memory read ends with a barrier, so the
// next may write the buffer at once); otherwise both halves run in lockstep,
// each through its own buffer.
template <class Cfg, int SLOTS, int LPT, bool SEQ, bool INV, bool TWS = false>
__device__ __forceinline__ void col_line_ffts(cpx<typename Cfg::R> (&v)[LPT][Cfg::E], const ColIds<Cfg, SLOTS, LPT>& id,
                                              cpx<typename Cfg::R>* sm, const cpx<typename Cfg::R>* tw) {
    using R = typename Cfg::R;
    constexpr int N = Cfg::N, E = Cfg::E;
    if constexpr (SEQ && LPT == 2) {
        const LineSmem<R> l0[1] = {col_line<R, N, SLOTS>(sm, 0, id.slot)};
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            cpx<R> u[1][E];
#pragma unroll
            for (int m = 0; m < E; ++m) u[0][m] = v[l][m];
            line_fft<R, N, E, INV, 1, TWS>(u, id.t, l0, tw, typename Cfg::Rads{});
#pragma unroll
            for (int m = 0; m < E; ++m) v[l][m] = u[0][m];
        }
    } else {
        LineSmem<R> ls[LPT];
#pragma unroll
        for (int l = 0; l < LPT; ++l) ls[l] = col_line<R, N, SLOTS>(sm, id.half(l), id.slot);
        line_fft<R, N, E, INV, LPT, TWS>(v, id.t, ls, tw, typename Cfg::Rads{});
    }
}
// exchange buffers a column tile needs
template <int LPT, bool SEQ> constexpr int col_buffers() { return SEQ && LPT == 2 ? 1 : 2; }

// pass 1: pad + forward FFT along y.  W1 -> W2.  SEQ (two lines per
// thread): the halves are transformed one after the other through one
// exchange buffer, and each half is stored as soon as it is done, so the
// even half's stores drain while the odd half is transformed.
template <class Cfg, int SLOTS, int LPT, bool CG, bool SEQ = false, class In = ColFromGlobal, class Hook = NoHook>
__device__ __forceinline__ void tile_y_fwd(const PassParams<typename Cfg::R>& p, int tile,
                                            unsigned char* smem_raw, const In& in_src = In{},
                                            const Hook& after_load = Hook{}) {
    using R = typename Cfg::R;
    constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T;
    cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
    const ColIds<Cfg, SLOTS, LPT> id;
    const int ny = p.ny;
    const ColTile<R, SLOTS> c = col_tile<R, SLOTS>(p.nx + 1, p.nz, id.slot, tile);
    const cpx<R>* __restrict__ in = static_cast<const cpx<R>*>(p.in);
    cpx<R>* __restrict__ out = static_cast<cpx<R>*>(p.out);
    const long long sx = p.sx;

    cpx<R> v[LPT][E];
    const cpx<R>* src = in + (long long)c.other * ny * sx + c.kx + (long long)id.t * sx;
#pragma unroll
    for (int m = 0; m < E; ++m)
        v[0][m] = c.valid ? col_in<CG>(in_src, src + (long long)(T * m) * sx, id.t + T * m) : cpx<R>{0, 0};
    after_load();
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
        if (id.half(l)) {
            const LineRamp<N, E, R, In::TW_SMEM> rw(p.tw, id.t);
            sfor<E>([&](auto m_) {
                constexpr int m = decltype(m_)::value;
                v[l][m] = cmul(v[0][m], rw.template at<m>());
            });
        }
    }
    if constexpr (SEQ && LPT == 2) {
        const LineSmem<R> l0[1] = {col_line<R, N, SLOTS>(sm, 0, id.slot)};
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            cpx<R> u[1][E];
#pragma unroll
            for (int m = 0; m < E; ++m) u[0][m] = v[l][m];
            line_fft<R, N, E, false, 1, In::TW_SMEM>(u, id.t, l0, p.tw, typename Cfg::Rads{});
            if (c.valid) {
                cpx<R>* dst = out + (long long)c.other * 2 * ny * sx + c.kx + (long long)(l * ny + id.t) * sx;
#pragma unroll
                for (int m = 0; m < E; ++m) dst[(long long)(T * m) * sx] = u[0][m];
            }
        }
    } else {
        LineSmem<R> ls[LPT];
#pragma unroll
        for (int l = 0; l < LPT; ++l) ls[l] = col_line<R, N, SLOTS>(sm, id.half(l), id.slot);
        line_fft<R, N, E, false, LPT, In::TW_SMEM>(v, id.t, ls, p.tw, typename Cfg::Rads{});

        if (c.valid) {
#pragma unroll
            for (int l = 0; l < LPT; ++l) {
                cpx<R>* dst = out + (long long)c.other * 2 * ny * sx + c.kx +
                              (long long)(id.half(l) * ny + id.t) * sx;
#pragma unroll
                for (int m = 0; m < E; ++m) dst[(long long)(T * m) * sx] = v[l][m];
            }
        }
    }
}

// Final combine of the cropped inverse, x[j] = a[j] + W_2N^-j b[j] with a,b
// the inverse transforms of the even and odd halves.  CONJ: the halves hold
// conj(a) and conj(b) (an inverse run as a conjugated forward transform),
// and x = conj(conj(a) + W_2N^j conj(b)).  Returns true in the threads that
// hold x[t + T m] in v[0][m] afterwards.
template <class Cfg, int SLOTS, int LPT, bool CONJ = false, bool TWS = false>
__device__ __forceinline__ bool combine_halves(cpx<typename Cfg::R> (&v)[LPT][Cfg::E],
                                               const ColIds<Cfg, SLOTS, LPT>& id,
                                               cpx<typename Cfg::R>* sm,
                                               const cpx<typename Cfg::R>* tw) {
    using R = typename Cfg::R;
    constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T;
    const LineRamp<N, E, R, TWS> rw(tw, id.t);
    if constexpr (LPT == 2) {
        sfor<E>([&](auto m_) {
            constexpr int m = decltype(m_)::value;
            if constexpr (CONJ) {
                const cpx<R> s = v[0][m] + cmul(v[1][m], rw.template at<m>());
                v[0][m] = {s.x, -s.y};
            } else {
                v[0][m] = v[0][m] + cmulc(v[1][m], rw.template at<m>());
            }
        });
        return true;
    } else {
        const LineSmem<R> lodd = col_line<R, N, SLOTS>(sm, 1, id.slot);
        if (id.q) {
            sfor<E>([&](auto m_) {
                constexpr int m = decltype(m_)::value;
                lodd[id.t + T * m] = CONJ ? cmul(v[0][m], rw.template at<m>()) : cmulc(v[0][m], rw.template at<m>());
            });
        }
        __syncthreads();
        if (!id.q) {
#pragma unroll
            for (int m = 0; m < E; ++m) {
                const cpx<R> s = v[0][m] + lodd[id.t + T * m];
                v[0][m] = CONJ ? cpx<R>{s.x, -s.y} : s;
            }
        }
        return id.q == 0;
    }
}

// pass 2: pad + FFT along z, multiply by Ghat, inverse FFT along z, crop.
// In place on W2.  Ghat is real (the kernel is real and even), so the
// adjoint's conj(Ghat) is the same multiply.
// Staging of a tile's Green's function rows in shared memory: row kz
// (kz <= N) holds the SLOTS columns' values.  With SLOTS < BW (elements per
// row of banks) a row covers one of G = BW/SLOTS bank windows; rows are
// permuted within aligned blocks of G so that row kz = 2a + b sits in window
// (a + b G/2) mod G.  The copy-in (lanes on G consecutive rows of a block)
// and the multiply (lanes on G rows two apart, either direction) then never
// put two lanes of a warp on one bank.
template <class R, int SLOTS> constexpr int gsl_group() {
    constexpr int BW = 128 / (int)sizeof(R);
    return SLOTS >= BW ? 1 : BW / SLOTS;
}
template <class R, int SLOTS> __device__ __forceinline__ int gsl_idx(int kz, int slot) {
    constexpr int G = gsl_group<R, SLOTS>();
    if constexpr (G == 1) {
        return kz * SLOTS + slot;
    } else {
        const int w = ((kz >> 1) + (kz & 1) * (G / 2)) & (G - 1);
        return ((kz & ~(G - 1)) + w) * SLOTS + slot;
    }
}
template <class R, int N, int SLOTS> constexpr int gsl_elems() {
    constexpr int G = gsl_group<R, SLOTS>();
    return (N + 1 + G - 1) / G * G * SLOTS;
}

template <class Cfg, int SLOTS, int LPT, bool CG, bool SEQ = false, class In = ColFromGlobal, class Hook = NoHook>
__device__ __forceinline__ void tile_z_conv(const PassParams<typename Cfg::R>& p, int tile,
                                            unsigned char* smem_raw, const In& in_src = In{},
                                            const Hook& after_load = Hook{}) {
    using R = typename Cfg::R;
    constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T;
    cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
    const ColIds<Cfg, SLOTS, LPT> id;
    const int nx = p.nx, ny = p.ny;
    const ColTile<R, SLOTS> c = col_tile<R, SLOTS>(nx + 1, 2 * ny, id.slot, tile);
    cpx<R>* __restrict__ w = static_cast<cpx<R>*>(p.out);
    const long long plane = 2LL * ny * p.sx;

    // start copying this column's octant row Ghat[kz][kyf][kx], kz <= N, to
    // shared memory (after the exchange buffers); it is needed only after
    // the forward transform
    R* gsl = reinterpret_cast<R*>(sm + col_buffers<LPT, SEQ>() * col_rows<R, N, SLOTS>() * SLOTS);
    if (c.valid) {
        const int kys = c.other;
        const int ky = kys < ny ? 2 * kys : 2 * (kys - ny) + 1;
        const int kyf = ky <= ny ? ky : 2 * ny - ky;
        constexpr int gz = greens_xw<R>();  // kz stride within the block
        const R* g = p.greens + greens_base<R>(c.kx, kyf, nx, p.nz);
        constexpr int TPS = (LPT == 1 ? 2 : 1) * T;  // threads per slot
        const int u = id.t + (LPT == 1 ? id.q * T : 0);
        if constexpr (TPS % gsl_group<R, SLOTS>() == 0) {
            // rows u + TPS i keep u's place within their block of G rows, so
            // the staged index and the source advance by constant steps
            R* sp = gsl + gsl_idx<R, SLOTS>(u, id.slot);
            const R* gp = g + u * gz;
#pragma unroll
            for (int i = 0; i < N / TPS; ++i) cp_async_real(sp + i * TPS * SLOTS, gp + i * TPS * gz);
            if (u == 0) cp_async_real(sp + N * SLOTS, gp + N * gz);
        } else {
            for (int kz = u; kz <= N; kz += TPS) cp_async_real(gsl + gsl_idx<R, SLOTS>(kz, id.slot), g + kz * gz);
        }
    }
    cp_async_commit();

    cpx<R> v[LPT][E];
    cpx<R>* col = w + (long long)c.other * p.sx + c.kx;
#pragma unroll
    for (int m = 0; m < E; ++m)
        v[0][m] = c.valid ? col_in<CG>(in_src, col + (long long)(id.t + T * m) * plane, id.t + T * m) : cpx<R>{0, 0};
    after_load();
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
        if (id.half(l)) {
            const LineRamp<N, E, R, In::TW_SMEM> rw(p.tw, id.t);
            sfor<E>([&](auto m_) {
                constexpr int m = decltype(m_)::value;
                v[l][m] = cmul(v[0][m], rw.template at<m>());
            });
        }
    }
    // The inverse transform runs as conj(FFT(conj(.))) through the forward
    // transform's code: a two-trip loop that is not unrolled, so the tile
    // holds one copy of the line transforms (half the instruction footprint
    // of a forward and an inverse copy).  The Green's multiply conjugates its
    // products and the combine conjugates back.
#pragma unroll 1
    for (int ph = 0; ph < 2; ++ph) {
        col_line_ffts<Cfg, SLOTS, LPT, SEQ, false, In::TW_SMEM>(v, id, sm, p.tw);
        if (ph == 1) break;

        // Green's multiply at frequency (kx, ky, kz), folded into the octant;
        // the column's octant row was copied to shared memory while the forward
        // transform ran.  kz = 2 (t + T m) + q is <= N exactly for m < E/2.
        cp_async_commit_wait_all();
        __syncthreads();
        if (c.valid) {
#pragma unroll
            for (int l = 0; l < LPT; ++l) {
                const int kz0 = 2 * id.t + id.half(l);
                if constexpr (T % gsl_group<R, SLOTS>() == 0) {
                    // kz0 + 2 T m and 2N - kz0 - 2 T m keep the place of kz0 and
                    // 2N - kz0 within their blocks of G rows: constant offsets
                    // from two bases (the second base, beyond row N for small
                    // kz0, is only read back at rows <= N)
                    const int i_lo = gsl_idx<R, SLOTS>(kz0, id.slot);
                    const int i_hi = gsl_idx<R, SLOTS>(2 * N - kz0, id.slot);
#pragma unroll
                    for (int m = 0; m < E; ++m)
                        v[l][m] = scale_conj(v[l][m], gsl[m < E / 2 ? i_lo + 2 * T * m * SLOTS : i_hi - 2 * T * m * SLOTS]);
                } else {
#pragma unroll
                    for (int m = 0; m < E; ++m) {
                        const int kz = kz0 + 2 * T * m;
                        const int kzf = (m < E / 2) ? kz : 2 * N - kz;
                        v[l][m] = scale_conj(v[l][m], gsl[gsl_idx<R, SLOTS>(kzf, id.slot)]);
                    }
                }
            }
        }
    }

    if (combine_halves<Cfg, SLOTS, LPT, true, In::TW_SMEM>(v, id, sm, p.tw) && c.valid) {
#pragma unroll
        for (int m = 0; m < E; ++m) col[(long long)(id.t + T * m) * plane] = v[0][m];
    }
}

// pass 3: inverse FFT along y + crop.  W2 -> W1.  SEQ (two lines per
// thread): the even and odd halves are transformed one after the other
// through one exchange buffer, which halves the tile's work area (the
// single-buffered persistent TMA tile of 512-long columns then fits).
template <class Cfg, int SLOTS, int LPT, bool CG, bool SEQ = false, class In = ColFromGlobal, class Hook = NoHook>
__device__ __forceinline__ void tile_y_inv(const PassParams<typename Cfg::R>& p, int tile,
                                            unsigned char* smem_raw, const In& in_src = In{},
                                            const Hook& after_load = Hook{}) {
    using R = typename Cfg::R;
    constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T;
    cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
    const ColIds<Cfg, SLOTS, LPT> id;
    const int ny = p.ny;
    const ColTile<R, SLOTS> c = col_tile<R, SLOTS>(p.nx + 1, p.nz, id.slot, tile);
    const cpx<R>* __restrict__ in = static_cast<const cpx<R>*>(p.in);
    cpx<R>* __restrict__ out = static_cast<cpx<R>*>(p.out);
    const long long sx = p.sx;

    cpx<R> v[LPT][E];
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
        const cpx<R>* src = in + (long long)c.other * 2 * ny * sx + c.kx +
                            (long long)(id.half(l) * ny + id.t) * sx;
#pragma unroll
        for (int m = 0; m < E; ++m)
            v[l][m] = c.valid ? col_in<CG>(in_src, src + (long long)(T * m) * sx, id.half(l) * ny + id.t + T * m)
                              : cpx<R>{0, 0};
    }
    after_load();
    col_line_ffts<Cfg, SLOTS, LPT, SEQ, true, In::TW_SMEM>(v, id, sm, p.tw);

    if (combine_halves<Cfg, SLOTS, LPT, false, In::TW_SMEM>(v, id, sm, p.tw) && c.valid) {
        cpx<R>* dst = out + (long long)c.other * ny * sx + c.kx + (long long)id.t * sx;
#pragma unroll
        for (int m = 0; m < E; ++m) dst[(long long)(T * m) * sx] = v[0][m];
    }
}

// ==========================================================================
// Row passes (x axis; lines are contiguous rows, two real rows per line)
// ==========================================================================
//
// Thread = (t, pair[, q]): t fastest, then the row pair within the tile,
// then (LPT = 1) the half q.  A tile holds PAIRS row pairs (2*PAIRS
// consecutive rows, which are contiguous in rho and phi).

template <class R> struct RowPad { static constexpr int SHIFT = sizeof(R) == 4 ? 4 : 3; };

template <class Cfg> constexpr int row_line_stride() {
    return Cfg::N + (Cfg::N >> RowPad<typename Cfg::R>::SHIFT);
}
// Offset (complex elements) of row pair pr's line for half h in a row
// tile's exchange area.  The odd halves start 64 bytes further on: the
// x-forward spectrum separation has neighbouring lanes read the even and the
// odd line of a pair at the same index, which without the skew fall on the
// same banks.
template <class Cfg> constexpr int row_odd_skew() { return 64 / (int)sizeof(cpx<typename Cfg::R>); }
template <class Cfg, int PAIRS> __device__ __forceinline__ int row_line_off(int half, int pr) {
    return (half * PAIRS + pr) * row_line_stride<Cfg>() + half * row_odd_skew<Cfg>();
}
// real staging row stride: skews consecutive pairs' rows across banks
template <class Cfg> constexpr int row_stage_stride() {
    return Cfg::N + (Cfg::T >= 8 ? Cfg::T / 2 : 4);
}
template <class Cfg, int PAIRS, int LPT> constexpr int row_threads() {
    return (LPT == 1 ? 2 : 1) * PAIRS * Cfg::T;
}

template <class Cfg, int PAIRS, int LPT> struct RowIds {
    int t, pr, q;
    __device__ __forceinline__ RowIds() {
        t = threadIdx.x % Cfg::T;
        pr = (threadIdx.x / Cfg::T) % PAIRS;
        q = LPT == 1 ? threadIdx.x / (Cfg::T * PAIRS) : 0;
    }
    __device__ __forceinline__ int half(int l) const { return LPT == 2 ? l : q; }
};

// pass 0: pad + R2C along x.  rho (real rows of nx) -> W1 (nx+1 bins).
template <class Cfg, int PAIRS, int LPT, bool CG>
__device__ __forceinline__ void tile_x_fwd(const PassParams<typename Cfg::R>& p, int rows, int tile,
                                            unsigned char* smem_raw) {
    using R = typename Cfg::R;
    constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T;
    constexpr int RS = row_stage_stride<Cfg>();
    constexpr int SH = RowPad<R>::SHIFT;
    constexpr int NT = row_threads<Cfg, PAIRS, LPT>();
    using V = typename std::conditional<sizeof(R) == 4, float4, double2>::type;
    constexpr int VW = 16 / sizeof(R);
    constexpr int VPR = N / VW;  // vectors per row
    R* stage = reinterpret_cast<R*>(smem_raw);
    cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
    const RowIds<Cfg, PAIRS, LPT> id;
    const int t = id.t, pr = id.pr;
    const int r0 = tile * 2 * PAIRS;
    const int nrows = min(2 * PAIRS, rows - r0);

    cpx<R> v[LPT][E];
    const bool has_a = 2 * pr < nrows, has_b = 2 * pr + 1 < nrows;
    if constexpr (LPT == 2) {
        // both halves in one thread: read x[j], j = t + T m, of the pair's two
        // rows straight from rho (lanes of consecutive j read consecutive words)
        const R* __restrict__ xa = static_cast<const R*>(p.in) + (long long)(r0 + 2 * pr) * N;
        const R* __restrict__ xb = xa + N;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int j = t + T * m;
            v[0][m] = {has_a ? xa[j] : (R)0, has_b ? xb[j] : (R)0};
        }
    } else {
    // stage the tile's rows with 16-byte loads, all issued before any store
    {
        const V* __restrict__ src = reinterpret_cast<const V*>(static_cast<const R*>(p.in) + (long long)r0 * N);
        constexpr int PER = (2 * PAIRS * VPR + NT - 1) / NT;
        V buf[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int i = threadIdx.x + u * NT;
            if (i < nrows * VPR) buf[u] = __ldg(src + i);
        }
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int i = threadIdx.x + u * NT;
            if (i < nrows * VPR) {
                const int s = i / VPR, c = i - s * VPR;
                *reinterpret_cast<V*>(stage + s * RS + c * VW) = buf[u];
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int j = t + T * m;
        const R a = has_a ? stage[(2 * pr) * RS + j] : (R)0;
        const R b = has_b ? stage[(2 * pr + 1) * RS + j] : (R)0;
        v[0][m] = {a, b};
    }
    __syncthreads();  // the staging area becomes the line buffers
    }
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
        if (id.half(l)) {
            const LineRamp<N, E, R> rw(p.tw, t);
            sfor<E>([&](auto m_) {
                constexpr int m = decltype(m_)::value;
                v[l][m] = cmul(v[0][m], rw.template at<m>());
            });
        }
    }
    LineSmem<R> ls[LPT];
#pragma unroll
    for (int l = 0; l < LPT; ++l) ls[l] = {sm + row_line_off<Cfg, PAIRS>(id.half(l), pr), 1, SH, 1};
    line_fft<R, N, E, false, LPT>(v, t, ls, p.tw, typename Cfg::Rads{});
#pragma unroll
    for (int l = 0; l < LPT; ++l)
#pragma unroll
        for (int m = 0; m < E; ++m) ls[l][t + T * m] = v[l][m];
    __syncthreads();

    // separate the two rows' spectra: A[k] = (Z[k] + conj Z[2N-k]) / 2,
    // B[k] = -i (Z[k] - conj Z[2N-k]) / 2, k = 0..N; Z[2k'] = E[k'],
    // Z[2k'+1] = O[k'].
    cpx<R>* __restrict__ out = static_cast<cpx<R>*>(p.out);
    const long long sx = p.sx;
    // each row pair is handled by the NT / PAIRS threads that share its pair
    // index; one (P, Q) read gives both rows' bin k
    constexpr int U = NT / PAIRS;
    const int u = t + (LPT == 1 ? id.q * T : 0);
    if (has_a) {
        const LineSmem<R> e = {sm + row_line_off<Cfg, PAIRS>(0, pr), 1, SH, 1};
        const LineSmem<R> o = {sm + row_line_off<Cfg, PAIRS>(1, pr), 1, SH, 1};
        cpx<R>* ra = out + (long long)(r0 + 2 * pr) * sx;
        cpx<R>* rb = ra + sx;
        for (int k = u; k <= N; k += U) {
            const int kh = k >> 1;
            cpx<R> P, Q;
            if ((k & 1) == 0) {
                P = e[kh];
                Q = e[kh == 0 ? 0 : N - kh];
            } else {
                P = o[kh];
                Q = o[N - 1 - kh];
            }
            Q.y = -Q.y;
            ra[k] = cpx<R>{(R)0.5 * (P.x + Q.x), (R)0.5 * (P.y + Q.y)};
            if (has_b) rb[k] = cpx<R>{(R)0.5 * (P.y - Q.y), (R)(-0.5) * (P.x - Q.x)};
        }
    }
}

// pass 4: C2R along x + crop.  W1 (nx+1 bins) -> phi (real rows of nx).
// Two adjacent complex values p[0], p[1] (p 16-byte aligned), L1-bypassing
// when CG.
template <bool CG, class R> __device__ __forceinline__ void ld_c2(const cpx<R>* p, cpx<R>& a, cpx<R>& b) {
    if constexpr (std::is_same<R, float>::value) {
        const float4 v = CG ? __ldcg(reinterpret_cast<const float4*>(p)) : *reinterpret_cast<const float4*>(p);
        a = {v.x, v.y};
        b = {v.z, v.w};
    } else {
        a = ld_c<CG>(p);
        b = ld_c<CG>(p + 1);
    }
}

// pass 4 with both halves in one thread (LPT = 2): every thread reads the
// spectrum bins it needs straight from W1 (bins 2j and 2j+1 of both rows as
// 16-byte pairs below the Nyquist bin, mirrored pairs above it; lanes of
// consecutive j read consecutive pairs), combines the halves in registers
// and writes its outputs x[j] straight to phi (lanes of consecutive j write
// consecutive words).  Only the line transform's exchange uses shared memory.
template <class Cfg, int PAIRS, bool CG>
__device__ __forceinline__ void tile_x_inv_direct(const PassParams<typename Cfg::R>& p, int rows, int tile,
                                                   unsigned char* smem_raw) {
    using R = typename Cfg::R;
    constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T;
    constexpr int SH = RowPad<R>::SHIFT;
    cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
    const RowIds<Cfg, PAIRS, 2> id;
    const int t = id.t, pr = id.pr;
    const int r0 = tile * 2 * PAIRS;
    const int nrows = min(2 * PAIRS, rows - r0);
    const bool has_a = 2 * pr < nrows, has_b = 2 * pr + 1 < nrows;
    const cpx<R>* __restrict__ in = static_cast<const cpx<R>*>(p.in);
    const cpx<R>* ra = in + (long long)(r0 + 2 * pr) * p.sx;
    const cpx<R>* rb = ra + p.sx;

    // Z[k] = A[k] + i B[k]; A[2N-k] = conj A[k] (same for B).  Register line
    // l holds Z[2j + l], j = t + T m.
    cpx<R> v[2][E];
#pragma unroll
    for (int m = 0; m < E; ++m) {
        const int k0 = 2 * (t + T * m);
        cpx<R> a0{0, 0}, a1{0, 0}, b0{0, 0}, b1{0, 0};
        if (m < E / 2) {  // k0 + 1 < N: the pair (k0, k0 + 1)
            if (has_a) ld_c2<CG>(ra + k0, a0, a1);
            if (has_b) ld_c2<CG>(rb + k0, b0, b1);
            v[0][m] = {a0.x - b0.y, a0.y + b0.x};
            v[1][m] = {a1.x - b1.y, a1.y + b1.x};
        } else {          // k0 >= N: bins 2N - k0 and 2N - k0 - 1
            const int kk = 2 * N - k0;
            if (has_a) { a0 = ld_c<CG>(ra + kk); a1 = ld_c<CG>(ra + kk - 1); }
            if (has_b) { b0 = ld_c<CG>(rb + kk); b1 = ld_c<CG>(rb + kk - 1); }
            v[0][m] = k0 <= N ? cpx<R>{a0.x - b0.y, a0.y + b0.x} : cpx<R>{a0.x + b0.y, b0.x - a0.y};
            v[1][m] = cpx<R>{a1.x + b1.y, b1.x - a1.y};
        }
    }
    LineSmem<R> ls[2];
#pragma unroll
    for (int l = 0; l < 2; ++l) ls[l] = {sm + row_line_off<Cfg, PAIRS>(l, pr), 1, SH, 1};
    line_fft<R, N, E, true, 2>(v, t, ls, p.tw, typename Cfg::Rads{});

    // x[j] = a[j] + W_2N^-j b[j]: real part -> row 2 pr, imaginary -> row 2 pr + 1
    R* oa = static_cast<R*>(p.out) + (long long)(r0 + 2 * pr) * N;
    R* ob = oa + N;
    bool bad = false;
    const LineRamp<N, E, R> rw(p.tw, t);
    sfor<E>([&](auto m_) {
        constexpr int m = decltype(m_)::value;
        const int j = t + T * m;
        const cpx<R> x = v[0][m] + cmulc(v[1][m], rw.template at<m>());
        if (has_a) oa[j] = x.x;
        if (has_b) ob[j] = x.y;
        bad |= (has_a && not_finite(x.x)) || (has_b && not_finite(x.y));
    });
    if (p.check_finite) flag_non_finite(p.status, bad);
}

template <class Cfg, int PAIRS, int LPT, bool CG>
__device__ __forceinline__ void tile_x_inv(const PassParams<typename Cfg::R>& p, int rows, int tile,
                                            unsigned char* smem_raw) {
    if constexpr (LPT == 2) {
        tile_x_inv_direct<Cfg, PAIRS, CG>(p, rows, tile, smem_raw);
        return;
    }
    using R = typename Cfg::R;
    constexpr int N = Cfg::N, E = Cfg::E, T = Cfg::T;
    constexpr int RS = row_stage_stride<Cfg>();
    constexpr int SH = RowPad<R>::SHIFT;
    constexpr int NT = row_threads<Cfg, PAIRS, LPT>();
    using V = typename std::conditional<sizeof(R) == 4, float4, double2>::type;
    constexpr int VW = 16 / sizeof(R);
    constexpr int VPR = N / VW;
    cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
    R* stage = reinterpret_cast<R*>(smem_raw);
    const RowIds<Cfg, PAIRS, LPT> id;
    const int t = id.t, pr = id.pr;
    const int r0 = tile * 2 * PAIRS;
    const int nrows = min(2 * PAIRS, rows - r0);
    const long long sx = p.sx;

    // stage the spectra rows (row s at [s*(N+1), (s+1)*(N+1))), loads first
    {
        const cpx<R>* __restrict__ in = static_cast<const cpx<R>*>(p.in);
        constexpr int PER = (2 * PAIRS * (N + 1) + NT - 1) / NT;
        cpx<R> buf[PER];
        const int nin = nrows * (N + 1);
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int i = threadIdx.x + u * NT;
            if (i < nin) {
                const int s = i / (N + 1), k = i - s * (N + 1);
                buf[u] = ld_c<CG>(in + (long long)(r0 + s) * sx + k);
            }
        }
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int i = threadIdx.x + u * NT;
            if (i < nin) sm[i] = buf[u];
        }
    }
    __syncthreads();
    // Z[k] = A[k] + i B[k] with A[2N-k] = conj A[k] (same for B); register
    // line l holds Z[2k' + half(l)], k' = t + T m.
    cpx<R> v[LPT][E];
    const bool has_a = 2 * pr < nrows, has_b = 2 * pr + 1 < nrows;
    const cpx<R>* ra = sm + (2 * pr) * (N + 1);
    const cpx<R>* rb = sm + (2 * pr + 1) * (N + 1);
#pragma unroll
    for (int l = 0; l < LPT; ++l)
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int k = 2 * (t + T * m) + id.half(l);
            const bool lo = k <= N;
            const int kk = lo ? k : 2 * N - k;
            const cpx<R> a = has_a ? ra[kk] : cpx<R>{0, 0};
            const cpx<R> b = has_b ? rb[kk] : cpx<R>{0, 0};
            v[l][m] = lo ? cpx<R>{a.x - b.y, a.y + b.x} : cpx<R>{a.x + b.y, b.x - a.y};
        }
    __syncthreads();  // the staging area becomes the line buffers

    LineSmem<R> ls[LPT];
#pragma unroll
    for (int l = 0; l < LPT; ++l) ls[l] = {sm + row_line_off<Cfg, PAIRS>(id.half(l), pr), 1, SH, 1};
    line_fft<R, N, E, true, LPT>(v, t, ls, p.tw, typename Cfg::Rads{});

    // z[j] = a[j] + W_2N^-j b[j]
    bool holder = true;
    const LineRamp<N, E, R> rw(p.tw, t);
    if constexpr (LPT == 2) {
        sfor<E>([&](auto m_) {
            constexpr int m = decltype(m_)::value;
            v[0][m] = v[0][m] + cmulc(v[1][m], rw.template at<m>());
        });
    } else {
        const LineSmem<R> lodd = {sm + row_line_off<Cfg, PAIRS>(1, pr), 1, SH, 1};
        if (id.q) {
            sfor<E>([&](auto m_) {
                constexpr int m = decltype(m_)::value;
                lodd[t + T * m] = cmulc(v[0][m], rw.template at<m>());
            });
        }
        __syncthreads();
        if (!id.q) {
#pragma unroll
            for (int m = 0; m < E; ++m) v[0][m] = v[0][m] + lodd[t + T * m];
        }
        holder = id.q == 0;
    }
    __syncthreads();  // line buffers become the output staging area
    if (holder) {
        bool bad = false;
#pragma unroll
        for (int m = 0; m < E; ++m) {
            const int j = t + T * m;
            stage[(2 * pr) * RS + j] = v[0][m].x;
            stage[(2 * pr + 1) * RS + j] = v[0][m].y;
            bad |= (has_a && not_finite(v[0][m].x)) || (has_b && not_finite(v[0][m].y));
        }
        if (p.check_finite) flag_non_finite(p.status, bad);
    }
    __syncthreads();
    {
        V* dst = reinterpret_cast<V*>(static_cast<R*>(p.out) + (long long)r0 * N);
        constexpr int PER = (2 * PAIRS * VPR + NT - 1) / NT;
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int i = threadIdx.x + u * NT;
            if (i < nrows * VPR) {
                const int s = i / VPR, c = i - s * VPR;
                dst[i] = *reinterpret_cast<const V*>(stage + s * RS + c * VW);
            }
        }
    }
}

// ==========================================================================
// kernels: one tile per CTA
// ==========================================================================
template <class Cfg, int SLOTS, int LPT, int MINB>
__global__ void __launch_bounds__(col_threads<Cfg, SLOTS, LPT>(), MINB) k_y_fwd(PassParams<typename Cfg::R> p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_y_fwd<Cfg, SLOTS, LPT, false>(p, blockIdx.x + p.tile0, smem_raw);
}
template <class Cfg, int SLOTS, int LPT, int MINB>
__global__ void __launch_bounds__(col_threads<Cfg, SLOTS, LPT>(), MINB) k_z_conv(PassParams<typename Cfg::R> p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_z_conv<Cfg, SLOTS, LPT, false>(p, blockIdx.x + p.tile0, smem_raw);
}
template <class Cfg, int SLOTS, int LPT, int MINB>
__global__ void __launch_bounds__(col_threads<Cfg, SLOTS, LPT>(), MINB) k_y_inv(PassParams<typename Cfg::R> p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_y_inv<Cfg, SLOTS, LPT, false>(p, blockIdx.x + p.tile0, smem_raw);
}
template <class Cfg, int PAIRS, int LPT, int MINB>
__global__ void __launch_bounds__(row_threads<Cfg, PAIRS, LPT>(), MINB) k_x_fwd(PassParams<typename Cfg::R> p, int rows) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_x_fwd<Cfg, PAIRS, LPT, false>(p, rows, blockIdx.x, smem_raw);
}
template <class Cfg, int PAIRS, int LPT, int MINB>
__global__ void __launch_bounds__(row_threads<Cfg, PAIRS, LPT>(), MINB) k_x_inv(PassParams<typename Cfg::R> p, int rows) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_x_inv<Cfg, PAIRS, LPT, false>(p, rows, blockIdx.x, smem_raw);
}

// --------------------------------------------------------------------------
// Persistent column kernels with TMA prefetch (FP32, wide tiles)
// --------------------------------------------------------------------------
//
// Each CTA walks tiles t0 + blockIdx.x, + gridDim.x, ... of [t0, t1).  A
// tile's input (ROWS rows x SLOTS columns) is one 3-D box of the W1/W2 array
// (up to 256 rows per TMA copy), copied into one of NBUF shared-memory
// buffers; once every thread holds tile i in registers, thread 0 starts the
// copy of tile i+NBUF into the buffer tile i came from, so NBUF tiles' loads
// are in flight under the transforms.  NBUF = 1 is for the long columns
// (384, 512), where one CTA per SM holds a 16-column tile: its next tile's
// load then overlaps the current tile's transforms and stores instead of
// following them.  Box layouts in shared memory:
//   y passes (PASS 1, 3): [other][row][kx]   (other = z, outermost dim)
//   z pass (PASS 2):      [row][other][kx]   (other = ky line, middle dim)
template <int PASS, class Cfg, int SLOTS, int NBUF> struct TmaBox {
    static constexpr int ROWS = PASS == 3 ? 2 * Cfg::N : Cfg::N;
    static constexpr int XW = SLOTS < Seg<float>::XW ? SLOTS : Seg<float>::XW;
    static constexpr int NLW = SLOTS / XW;
    // rows per copy: the largest of ROWS, 256, 192, 128 that divides ROWS and is <= 256 (box limit)
    static constexpr int CH = ROWS <= 256 ? ROWS : ROWS % 256 == 0 ? 256 : ROWS % 192 == 0 ? 192 : 128;
    static constexpr int NCH = ROWS / CH;
    static constexpr unsigned BYTES = (unsigned)ROWS * SLOTS * 8u;  // one buffer
    static constexpr size_t WORK_OFF = (size_t)NBUF * BYTES + 128;  // NBUF mbarriers, then the work area
    static_assert(NBUF == 1 || NBUF == 2, "one or two tile buffers");
    static_assert(ROWS % CH == 0, "rows must split into whole copies");
    // more than 256 rows needs one line per box column
    static constexpr bool LAYOUT_OK = NCH == 1 || NLW == 1;
};
constexpr int kTmaWaitPolls = 1 << 20;  // bounded wait for one tile's copy

template <int PASS, class Cfg, int SLOTS, int LPT, int MINB, int NBUF>
__global__ void __launch_bounds__(col_threads<Cfg, SLOTS, LPT>(), MINB)
    k_col_tma(PassParams<float> p, const __grid_constant__ CUtensorMap map, int t0, int t1, int hold, int tw_off,
              int tw_n) {
    using B = TmaBox<PASS, Cfg, SLOTS, NBUF>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    cpx<float>* buf = reinterpret_cast<cpx<float>*>(smem_raw);  // buffer k at buf + k * ROWS * SLOTS
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem_raw + NBUF * B::BYTES);  // bar[0 .. NBUF)
    unsigned char* work = smem_raw + B::WORK_OFF;
    // the axis twiddle table (tw_n entries), copied once per CTA behind the
    // work area; the tiles read their twiddles from here
    cpx<float>* tws = reinterpret_cast<cpx<float>*>(smem_raw + tw_off);
    for (int i = threadIdx.x; i < tw_n; i += blockDim.x) tws[i] = ldg_c(p.tw + i);
    PassParams<float> q = p;
    q.tw = tws;
    const int lines = PASS == 2 ? 2 * p.ny : p.nz;
    const int wide_l = (lines + B::NLW - 1) / B::NLW;
    auto issue = [&](int tile, int k) {
        const int xt = tile / wide_l, lt = tile - xt * wide_l;
        const int c0 = 2 * xt * B::XW, o0 = lt * B::NLW;
        cpx<float>* dst = buf + k * B::ROWS * SLOTS;
        mbar_arrive_expect_tx(bar + k, B::BYTES);
#pragma unroll
        for (int ch = 0; ch < B::NCH; ++ch) {
            if constexpr (PASS == 2) tma_load_3d(dst + ch * B::CH * SLOTS, &map, bar + k, c0, o0, ch * B::CH);
            else tma_load_3d(dst + ch * B::CH * B::XW, &map, bar + k, c0, ch * B::CH, o0);
        }
    };
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NBUF; ++k) mbar_init(bar + k, 1);
        mbar_fence_init();
    }
    __syncthreads();
    int tile = t0 + (int)blockIdx.x;
    if (tile >= t1) return;
    const int G = (int)gridDim.x;
    if (threadIdx.x == 0) {
        if (!hold) issue(tile, 0);  // test hook: the first copy is never issued, its wait runs out
        if (NBUF == 2 && tile + G < t1) issue(tile + G, 1);
    }
    const int slot = threadIdx.x % SLOTS;
    const int off = PASS == 2 ? slot : (slot / B::XW) * B::ROWS * B::XW + slot % B::XW;
    const int stride = PASS == 2 ? SLOTS : B::XW;
    unsigned parity = 0;  // bit k: phase parity of bar[k]
    for (int k = 0; tile < t1; tile += G, k = NBUF == 2 ? k ^ 1 : 0) {
        const bool ok = __syncthreads_and(mbar_wait(bar + k, (parity >> k) & 1u, kTmaWaitPolls));
        if (!ok) {
            // record the timeout, give the copies in flight a last bounded
            // chance to land, and leave (uniformly for the whole CTA)
            if (threadIdx.x == 0 && p.status) atomicOr(p.status, 2u);
            (void)mbar_wait(bar + k, (parity >> k) & 1u, kTmaWaitPolls);
            if (NBUF == 2 && tile + G < t1) (void)mbar_wait(bar + (k ^ 1), (parity >> (k ^ 1)) & 1u, kTmaWaitPolls);
            return;
        }
        parity ^= 1u << k;
        const ColFromSmem<float> in{buf + k * B::ROWS * SLOTS + off, stride};
        const int next = tile + NBUF * G;
        auto hook = [&]() {
            __syncthreads();  // every thread has its inputs: buffer k is free
            if (threadIdx.x == 0 && next < t1) {
                fence_proxy_async_smem();
                issue(next, k);
            }
        };
        if constexpr (PASS == 1) tile_y_fwd<Cfg, SLOTS, LPT, false, NBUF == 1 && LPT == 2>(q, tile, work, in, hook);
        else if constexpr (PASS == 2) tile_z_conv<Cfg, SLOTS, LPT, false, NBUF == 1 && LPT == 2>(q, tile, work, in, hook);
        else tile_y_inv<Cfg, SLOTS, LPT, false, NBUF == 1 && LPT == 2>(q, tile, work, in, hook);
    }
}

// ==========================================================================
// launch helpers and variants
// ==========================================================================

// Opt a kernel in to more than 48 KB of dynamic shared memory, once per
// kernel and device (Tag makes one flag set per kernel instantiation).
template <class Tag, class K> inline cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    static unsigned long long done = 0;  // bit d: attribute set on device d
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? (1ull << dev) : 0ull;
    if (bit && (done & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) done |= bit;
    return e;
}
template <int PASS, class Cfg, int A, int B> struct SmemTag {};

// A variant fixes lines per thread and the CTA's target thread count; the
// tile width (column passes: SLOTS lines, row passes: PAIRS row pairs)
// follows from the line's thread count T.
template <int LPT_, int THREADS_, int MINB_ = 1, int TMA_ = 0, bool PK_ = false> struct Var {
    static constexpr int LPT = LPT_;
    static constexpr int THREADS = THREADS_;
    static constexpr int MINB = MINB_;  // minimum resident CTAs per SM (register cap)
    static constexpr int TMA = TMA_;    // column passes: persistent kernel with TMA prefetch into TMA_ (1, 2) buffers (FP32)
    static constexpr bool PK = PK_;     // column passes: packed FP32x2 line transforms (FP32, LPT 2)
    static_assert(!PK_ || (LPT_ == 2 && !TMA_), "packed tiles carry both halves and load from global");
};

template <class Cfg, class V> constexpr int var_slots() {
    constexpr int XW = Seg<typename Cfg::R>::XW;
    constexpr int lo = XW / 4;  // >= 32-byte row segments
    constexpr int s = V::THREADS / ((V::LPT == 1 ? 2 : 1) * Cfg::T);
    return s < lo ? lo : s;
}
template <class Cfg, class V> constexpr int var_pairs() {
    constexpr int s = V::THREADS / ((V::LPT == 1 ? 2 : 1) * Cfg::T);
    return s < 1 ? 1 : s;
}
template <class Cfg, int SLOTS> constexpr size_t col_smem() {
    return 2ull * col_rows<typename Cfg::R, Cfg::N, SLOTS>() * SLOTS * sizeof(cpx<typename Cfg::R>);
}
// the z pass also stages each column's Green's function row
template <class Cfg, int SLOTS> constexpr size_t col_smem_z() {
    return col_smem<Cfg, SLOTS>() + (size_t)gsl_elems<typename Cfg::R, Cfg::N, SLOTS>() * sizeof(typename Cfg::R);
}
template <class Cfg, int PAIRS> constexpr size_t row_smem() {
    using R = typename Cfg::R;
    constexpr size_t lines = (2ull * PAIRS * row_line_stride<Cfg>() + row_odd_skew<Cfg>()) * sizeof(cpx<R>);
    constexpr size_t stage_c = 2ull * PAIRS * (Cfg::N + 1) * sizeof(cpx<R>);
    constexpr size_t stage_r = 2ull * PAIRS * row_stage_stride<Cfg>() * sizeof(R);
    constexpr size_t m1 = lines > stage_c ? lines : stage_c;
    return m1 > stage_r ? m1 : stage_r;
}

// pass ids: 0 x_fwd, 1 y_fwd, 2 z_conv, 3 y_inv, 4 x_inv
template <class Cfg, class V>
cudaError_t launch_row(int pass, const PassParams<typename Cfg::R>& p, int rows, cudaStream_t st) {
    constexpr int P = var_pairs<Cfg, V>();
    constexpr int L = V::LPT;
    constexpr size_t sm = row_smem<Cfg, P>();
    constexpr int NT = row_threads<Cfg, P, L>();
    static_assert(NT <= 1024, "row CTA too large");
    const int grid = (rows + 2 * P - 1) / (2 * P);
    if (grid == 0) return cudaSuccess;
    cudaError_t e;
    if (pass == 0) {
        if ((e = set_smem<SmemTag<0, Cfg, P, L * 16 + V::MINB>>(k_x_fwd<Cfg, P, L, V::MINB>, sm)) != cudaSuccess) return e;
        k_x_fwd<Cfg, P, L, V::MINB><<<grid, NT, sm, st>>>(p, rows);
    } else {
        if ((e = set_smem<SmemTag<4, Cfg, P, L * 16 + V::MINB>>(k_x_inv<Cfg, P, L, V::MINB>, sm)) != cudaSuccess) return e;
        k_x_inv<Cfg, P, L, V::MINB><<<grid, NT, sm, st>>>(p, rows);
    }
    return cudaGetLastError();
}

// Host side of k_col_tma: tensor map of the pass's input array, grid of at
// most the resident CTAs, then the narrow tiles (Nyquist column, not a TMA
// box) through the plain kernel.
template <int PASS, class Cfg, int S, int L, int MINB, int NBUF>
cudaError_t launch_col_tma(const PassParams<float>& p, int t_begin, int t_end, int n_wide, cudaStream_t st) {
    using B = TmaBox<PASS, Cfg, S, NBUF>;
    constexpr int NT = col_threads<Cfg, S, L>();
    // (the single-buffered tiles transform their halves one after the other
    // through one exchange buffer)
    constexpr bool SEQ = NBUF == 1 && L == 2;
    constexpr size_t work = (SEQ ? col_smem<Cfg, S>() / 2 : col_smem<Cfg, S>()) +
                            (PASS == 2 ? col_smem_z<Cfg, S>() - col_smem<Cfg, S>() : 0);
    // behind the work area: the CTA's copy of the axis twiddle table
    constexpr size_t tw_off = (B::WORK_OFF + work + 15) / 16 * 16;
    constexpr int tw_n = tw_entries<Cfg::N>(typename Cfg::Rads{});
    constexpr size_t sm = tw_off + (size_t)tw_n * sizeof(cpx<float>);
    // a tile whose buffers do not fit one CTA's shared memory, or whose box
    // would need more than 256 rows and several lines per box column, runs
    // every tile through the plain kernel instead
    constexpr bool fits = B::LAYOUT_OK && sm <= 227u * 1024u;
    cudaError_t e;
    const int w1 = fits ? (t_end < n_wide ? t_end : n_wide) : t_begin;
    if constexpr (fits) if (t_begin < w1) {
        auto kern = k_col_tma<PASS, Cfg, S, L, MINB, NBUF>;
        if ((e = set_smem<SmemTag<40 + 10 * NBUF + PASS, Cfg, S, L * 16 + MINB>>(kern, sm)) != cudaSuccess) return e;
        static int per_sm[64] = {};  // resident CTAs on the device, per device
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        const int d = dev < 64 ? dev : 63;
        if (per_sm[d] == 0) {
            int occ = 0, nsm = 0;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, sm)) != cudaSuccess) return e;
            if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
            per_sm[d] = (occ > 0 ? occ : 1) * nsm;
        }
        // input array: W1 [nz][ny][sx] (y forward) or W2 [nz][2ny][sx]
        const int rows_mid = PASS == 1 ? p.ny : 2 * p.ny;
        const void* base = PASS == 2 ? p.out : p.in;
        const unsigned long long dims[3] = {2ull * (unsigned long long)(p.nx + 1), (unsigned long long)rows_mid,
                                            (unsigned long long)p.nz};
        const unsigned long long strides[2] = {(unsigned long long)p.sx * 8ull,
                                               (unsigned long long)p.sx * 8ull * rows_mid};
        const unsigned box[3] = {2u * B::XW, PASS == 2 ? (unsigned)B::NLW : (unsigned)B::CH,
                                 PASS == 2 ? (unsigned)B::CH : (unsigned)B::NLW};
        CUtensorMap map;
        if ((e = tma_encode_3d_f32(&map, base, dims, strides, box)) != cudaSuccess) return e;
        const int count = w1 - t_begin;
        const int grid = count < per_sm[d] ? count : per_sm[d];
        // test hook (failure detection without a GPU fault): the first copy of
        // every CTA is skipped, so its bounded wait runs out and reports
        const char* hold = std::getenv("POISSON_TEST_TMA_HOLD");
        kern<<<grid, NT, sm, st>>>(p, map, t_begin, w1, hold && hold[0] == '1' ? 1 : 0, (int)tw_off, tw_n);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int n0 = !fits ? t_begin : (t_begin > n_wide ? t_begin : n_wide);
    if (n0 < t_end) {
        PassParams<float> q = p;
        q.tile0 = n0;
        const int grid = t_end - n0;
        if constexpr (PASS == 1) {
            if ((e = set_smem<SmemTag<1, Cfg, S, L * 16 + MINB>>(k_y_fwd<Cfg, S, L, MINB>, col_smem<Cfg, S>())))
                return e;
            k_y_fwd<Cfg, S, L, MINB><<<grid, NT, col_smem<Cfg, S>(), st>>>(q);
        } else if constexpr (PASS == 3) {
            if ((e = set_smem<SmemTag<3, Cfg, S, L * 16 + MINB>>(k_y_inv<Cfg, S, L, MINB>, col_smem<Cfg, S>())))
                return e;
            k_y_inv<Cfg, S, L, MINB><<<grid, NT, col_smem<Cfg, S>(), st>>>(q);
        } else {
            if ((e = set_smem<SmemTag<2, Cfg, S, L * 16 + MINB>>(k_z_conv<Cfg, S, L, MINB>, col_smem_z<Cfg, S>())))
                return e;
            k_z_conv<Cfg, S, L, MINB><<<grid, NT, col_smem_z<Cfg, S>(), st>>>(q);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// wide tiles of a column pass (the ones k_col_tma takes)
template <class R, int SLOTS> inline int col_wide_tiles(int ncols, int L) {
    constexpr int XW = SLOTS < Seg<R>::XW ? SLOTS : Seg<R>::XW;
    constexpr int NLW = SLOTS / XW;
    return (ncols / XW) * ((L + NLW - 1) / NLW);
}

template <class Cfg, class V>
cudaError_t launch_col(int pass, const PassParams<typename Cfg::R>& p, cudaStream_t st) {
    using R = typename Cfg::R;
    if constexpr (V::TMA && std::is_same<R, float>::value) {
        constexpr int S = var_slots<Cfg, V>();
        const int lines = pass == 2 ? 2 * p.ny : p.nz;
        const int total = col_grid<R, S>(p.nx + 1, lines);
        const int n_wide = col_wide_tiles<R, S>(p.nx + 1, lines);
        const int tb = p.tile0, te = p.ntile > 0 ? p.tile0 + p.ntile : total;
        if (pass == 1) return launch_col_tma<1, Cfg, S, V::LPT, V::MINB, V::TMA>(p, tb, te, n_wide, st);
        if (pass == 3) return launch_col_tma<3, Cfg, S, V::LPT, V::MINB, V::TMA>(p, tb, te, n_wide, st);
        return launch_col_tma<2, Cfg, S, V::LPT, V::MINB, V::TMA>(p, tb, te, n_wide, st);
    }
    constexpr int S = var_slots<Cfg, V>();
    constexpr int L = V::LPT;
    constexpr size_t sm = col_smem<Cfg, S>();
    constexpr int NT = col_threads<Cfg, S, L>();
    static_assert(NT <= 1024, "column CTA too large");
    const int lines = pass == 2 ? 2 * p.ny : p.nz;
    const int grid = p.ntile > 0 ? p.ntile : col_grid<R, S>(p.nx + 1, lines);
    if (grid == 0) return cudaSuccess;
    cudaError_t e;
    if (pass == 1) {
        if ((e = set_smem<SmemTag<1, Cfg, S, L * 16 + V::MINB>>(k_y_fwd<Cfg, S, L, V::MINB>, sm)) != cudaSuccess) return e;
        k_y_fwd<Cfg, S, L, V::MINB><<<grid, NT, sm, st>>>(p);
    } else if (pass == 3) {
        if ((e = set_smem<SmemTag<3, Cfg, S, L * 16 + V::MINB>>(k_y_inv<Cfg, S, L, V::MINB>, sm)) != cudaSuccess) return e;
        k_y_inv<Cfg, S, L, V::MINB><<<grid, NT, sm, st>>>(p);
    } else {
        constexpr size_t smz = col_smem_z<Cfg, S>();
        if ((e = set_smem<SmemTag<2, Cfg, S, L * 16 + V::MINB>>(k_z_conv<Cfg, S, L, V::MINB>, smz)) != cudaSuccess)
            return e;
        k_z_conv<Cfg, S, L, V::MINB><<<grid, NT, smz, st>>>(p);
    }
    return cudaGetLastError();
}

}  // namespace pgb
