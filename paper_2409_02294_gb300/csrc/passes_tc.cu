// z pass with tensor-core radix-16 stages (POISSON_TC_FP16X2 / _BF16X2).
//
// For N = 16 M the length-N transform of each padded half line is written as
// stage 1 (radix M, FP32 in registers: thread t of 16 holds x[t + 16 r],
// r < M) followed by stage 2 (radix 16 with twiddles W_N^{r b}, b < M).  Stage
// 2 runs on tensor cores (tc_dft.cuh) for 8 lines at a time; the Green's
// multiply is applied to its FP32 results in registers; the inverse runs
// stage 2's conjugate transpose on tensor cores and stage 1's in registers.
// Twiddles are applied in FP32 before each split.
#include "configs.cuh"
#include "internal.h"
#include "tc_dft.cuh"

namespace pgb {

template <int N, bool BF16, bool CG>
__device__ __forceinline__ void tile_z_conv_tc(const PassParams<float>& p, int tile, unsigned char* smem_raw) {
    using R = float;
    constexpr int M = N / 16;
    constexpr int SLOTS = 8, LN = 16;  // 8 columns x 2 halves = 16 lines per tile
    static_assert(N % 16 == 0 && (M == 8 || M == 16 || M == 24 || M == 32), "N = 16 M");
    cpx<R>* buf = reinterpret_cast<cpx<R>*>(smem_raw);
    // element (row, line): 16 lines per 128-byte row; lines are swapped
    // between the two 64-byte halves of a row every 2M rows (bank spread)
    auto sidx = [](int row, int line) { return row * LN + (line ^ (((row / (2 * M)) & 1) << 3)); };
    const int tid = threadIdx.x;
    const int slot = tid & 7, t = (tid >> 3) & 15, q = tid >> 7;
    const int line = q * SLOTS + slot;
    const int nx = p.nx, ny = p.ny;
    const ColTile<R, SLOTS> c = col_tile<R, SLOTS>(nx + 1, 2 * ny, slot, tile);
    cpx<R>* __restrict__ w = static_cast<cpx<R>*>(p.out);
    const long long plane = 2LL * ny * p.sx;
    cpx<R>* col = w + (long long)c.other * p.sx + c.kx;

    // the tile's Green's function rows (8 columns x kz in [0, N]) go to shared
    // memory behind the line buffers, read once per tile
    R* gsl = reinterpret_cast<R*>(buf + N * LN);
    __shared__ long long s_goff[SLOTS];  // Ghat offset of each column's (ky, kx) row, -1 if invalid
    if (tid < SLOTS) {
        const ColTile<R, SLOTS> ce = col_tile<R, SLOTS>(nx + 1, 2 * ny, tid, tile);
        const int kys = ce.other;
        const int ky = kys < ny ? 2 * kys : 2 * (kys - ny) + 1;
        const int kyf = ky <= ny ? ky : 2 * ny - ky;
        s_goff[tid] = ce.valid ? greens_base<R>(ce.kx, kyf, nx, p.nz) : -1LL;
    }
    __syncthreads();
    {
        // columns fastest across threads: a warp reads four kz rows of the
        // tile's 8 columns (32 contiguous bytes each in the block layout)
        constexpr int gz = greens_xw<R>();
        for (int i = tid; i < SLOTS * (N + 1); i += 256) {
            const int kz = i / SLOTS, s = i - kz * SLOTS;
            const long long off = s_goff[s];
            gsl[s * (N + 1) + kz] = off >= 0 ? __ldg(p.greens + kz * gz + off) : (R)0;
        }
    }
    // 1. load x[t + 16 r]; the odd half is pre-twiddled by W_2N^j
    cpx<R> v[M];
#pragma unroll
    for (int r = 0; r < M; ++r)
        v[r] = c.valid ? ld_c<CG>(col + (long long)(t + 16 * r) * plane) : cpx<R>{0, 0};
    if (q) {
#pragma unroll
        for (int r = 0; r < M; ++r) v[r] = cmul(v[r], ldg_c(p.tw + t + 16 * r));
    }
    // 2. stage 1: y[M t + k] = sum_r W_M^{rk} x[t + 16 r]
    Dft<M, false, R>::run(v);
#pragma unroll
    for (int k = 0; k < M; ++k) buf[sidx(M * t + k, line)] = v[k];
    __syncthreads();

    // 3. per group (b, half h): tensor-core stage 2, Green's multiply,
    //    tensor-core inverse of stage 2
    const int warp = tid >> 5, lane = tid & 31, g = lane >> 2, cq = lane & 3;
    Dft16Frags<BF16> F;
    F.init(lane);
    const int rr[4] = {2 * cq, 2 * cq + 1, 2 * cq + 8, 2 * cq + 9};
    for (int grp = warp; grp < 2 * M; grp += 8) {
        const int b = grp >> 1, h = grp & 1;
        const int ln = h * 8 + g;
        float br[4], bi[4], dr[4], di[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const cpx<R> y = cmul(buf[sidx(b + M * rr[i], ln)], ldg_c(p.tw + 2 * rr[i] * b));
            br[i] = y.x;
            bi[i] = y.y;
        }
        __syncwarp();
        dft16_tc<BF16, false>(F, br, bi, dr, di);
        // dr/di[i] = X[b + M k] of line h*8 + n, (k, n) = (g + 8 (i>>1), 2cq + (i&1))
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int k = g + 8 * (i >> 1), e = i & 1;
            const int kz = 2 * (b + M * k) + h;
            const int kzf = kz <= N ? kz : 2 * N - kz;
            const R gv = gsl[(2 * cq + e) * (N + 1) + kzf];
            buf[sidx(b + M * k, h * 8 + 2 * cq + e)] = cpx<R>{dr[i] * gv, di[i] * gv};
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const cpx<R> y = buf[sidx(b + M * rr[i], ln)];
            br[i] = y.x;
            bi[i] = y.y;
        }
        __syncwarp();
        dft16_tc<BF16, true>(F, br, bi, dr, di);
        // rows r = g + 8 (i>>1) of stage 2's input, conj twiddle W_N^{-r b}
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = g + 8 * (i >> 1), e = i & 1;
            buf[sidx(b + M * r, h * 8 + 2 * cq + e)] = cmulc(cpx<R>{dr[i], di[i]}, ldg_c(p.tw + 2 * r * b));
        }
    }
    __syncthreads();
    // 4. inverse stage 1: x'[t + 16 r] = sum_k W_M^{-rk} y'[M t + k]
#pragma unroll
    for (int k = 0; k < M; ++k) v[k] = buf[sidx(M * t + k, line)];
    Dft<M, true, R>::run(v);
    __syncthreads();
    // 5. x[j] = a[j] + W_2N^-j b[j], j = t + 16 r
    if (q) {
#pragma unroll
        for (int r = 0; r < M; ++r) {
            const int j = t + 16 * r;
            buf[sidx(j, line)] = cmulc(v[r], ldg_c(p.tw + j));
        }
    }
    __syncthreads();
    if (!q && c.valid) {
#pragma unroll
        for (int r = 0; r < M; ++r) {
            const int j = t + 16 * r;
            col[(long long)j * plane] = v[r] + buf[sidx(j, line + 8)];
        }
    }
}

template <int N, bool BF16>
__global__ void __launch_bounds__(256) k_z_conv_tc(PassParams<float> p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    tile_z_conv_tc<N, BF16, false>(p, blockIdx.x + p.tile0, smem_raw);
}

template <int N, bool BF16>
cudaError_t launch_z_tc_n(const PassParams<float>& p, cudaStream_t st) {
    constexpr size_t sm = 128ull * N + 4ull * 8 * (N + 1);
    const int grid = p.ntile > 0 ? p.ntile : col_grid<float, 8>(p.nx + 1, 2 * p.ny);
    if (grid == 0) return cudaSuccess;
    cudaError_t e;
    if ((e = set_smem<SmemTag<20 + BF16, LineCfg<float, N, 16, Radices<N>>, 8, 1>>(k_z_conv_tc<N, BF16>, sm)))
        return e;
    k_z_conv_tc<N, BF16><<<grid, 256, sm, st>>>(p);
    return cudaGetLastError();
}

bool z_tc_supported(int N) { return N == 128 || N == 256 || N == 384 || N == 512; }

cudaError_t launch_z_tc(int N, bool bf16, const PassParams<float>& p, cudaStream_t st) {
    switch (N) {
        case 128: return bf16 ? launch_z_tc_n<128, true>(p, st) : launch_z_tc_n<128, false>(p, st);
        case 256: return bf16 ? launch_z_tc_n<256, true>(p, st) : launch_z_tc_n<256, false>(p, st);
        case 384: return bf16 ? launch_z_tc_n<384, true>(p, st) : launch_z_tc_n<384, false>(p, st);
        case 512: return bf16 ? launch_z_tc_n<512, true>(p, st) : launch_z_tc_n<512, false>(p, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pgb
