// Single-field solve in ONE persistent kernel with tile-level dataflow
// between the five passes (cubic FP32 grids).  Execution modes 1 and 2 are
// the same kernel compiled for 3 and 2 resident CTAs per SM (register caps
// of 170 and 255 per thread).
//
// The passes are run back to back by poisson_solve; here they overlap
// instead.  The z pass is arithmetic-bound and the x/y passes are
// memory-bound, so running the z tiles of one band of kx columns while the y
// tiles of other bands stream through HBM uses both resources at once.
//
// Dependencies are tracked per z-plane and per kx band ("chunk": one tile
// width of columns):
//   y forward (chunk c, planes P)  needs  x forward of every plane in P
//   z         (chunk c)            needs  y forward of chunk c, all planes
//   y inverse (chunk c, planes P)  needs  z of chunk c, all lines
//   x inverse (rows of planes P)   needs  y inverse of every chunk, planes P
// The work queue lists all x-forward tiles, then the column tiles as a
// software pipeline over chunks (y forward of chunk s, z of chunk s-3,
// y inverse of chunk s-6, ...), then all x-inverse tiles.  Every wait targets
// tiles earlier in the queue, which running CTAs have already claimed, so the
// kernel cannot deadlock.  Waits are bounded: on expiry the status word gets
// the timeout bit, an abort flag stops the other CTAs and the kernel
// returns.  Data written inside the launch is read with L1-bypassing loads.
#include <algorithm>
#include <vector>

#include "configs.cuh"
#include "internal.h"
#include "plan.h"

namespace pgb {

constexpr int FUSED_THREADS = 128;

template <int N> struct FusedShape {
    using C = typename SizeCfg<float, N>::C;      // column tiles
    using RC = typename RowSizeCfg<float, N>::C;  // row tiles
    static constexpr int L = C::E <= 16 ? 2 : 1;  // lines per thread
    using V = Var<L, FUSED_THREADS>;
    static constexpr int S = var_slots<C, V>();
    static constexpr int P = var_pairs<RC, V>();
    static constexpr int XW = S < Seg<float>::XW ? S : Seg<float>::XW;
    static constexpr int NLW = S / XW;
    static_assert(col_threads<C, S, L>() == FUSED_THREADS, "column tile must use 128 threads");
    static_assert(row_threads<RC, P, L>() == FUSED_THREADS, "row tile must use 128 threads");
    static constexpr size_t smem = col_smem_z<C, S>() > row_smem<RC, P>() ? col_smem_z<C, S>() : row_smem<RC, P>();
};

struct FusedArgs {
    PassParams<float> p[5];
    int n;              // edge length (cubic grid)
    int rows;           // n * n
    const int2* order;  // (pass, tile) per queue position
    int total;
    unsigned* ctl;      // [0] work, [1] abort, [2..] counters (see FusedCounters)
    unsigned* status;   // plan status word (bit 1: timeout)
    long long spin_limit;
};

// counter layout inside ctl
struct FusedCounters {
    int cx, cy, cz, cyi, count;  // offsets of the four arrays and the total
    __host__ __device__ FusedCounters(int n, int nch)
        : cx(2), cy(2 + n), cz(2 + n + nch), cyi(2 + n + 2 * nch), count(2 + 2 * n + 2 * nch) {}
};

__device__ __forceinline__ unsigned fused_ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ bool fused_wait(const unsigned* ctr, unsigned target, const FusedArgs& a) {
    for (long long it = 0; it < a.spin_limit; ++it) {
        if (fused_ld_acquire(ctr) >= target) return true;
        if (fused_ld_acquire(a.ctl + 1) != 0u) return false;
        __nanosleep(64);
    }
    atomicOr(a.status, 2u);
    atomicExch(a.ctl + 1, 1u);
    return false;
}

// Geometry of a column tile of the (cubic) grid: chunk and first/last line.
template <int N>
__device__ __forceinline__ void col_tile_span(int tile, int L, int& chunk, int& l0, int& l1) {
    using F = FusedShape<N>;
    const int ncols = N + 1;
    const int nxw = ncols / F::XW;
    const int n_wide = nxw * ((L + F::NLW - 1) / F::NLW);
    if (tile < n_wide) {
        const int nlt = (L + F::NLW - 1) / F::NLW;
        chunk = tile / nlt;
        l0 = (tile - chunk * nlt) * F::NLW;
        l1 = min(L, l0 + F::NLW);
    } else {
        const int b = tile - n_wide, nln = (L + F::S - 1) / F::S;
        chunk = nxw + b / nln;
        l0 = (b - (b / nln) * nln) * F::S;
        l1 = min(L, l0 + F::S);
    }
}
template <int N> __device__ __forceinline__ int col_chunk_tiles(int chunk, int L) {
    using F = FusedShape<N>;
    const int nxw = (N + 1) / F::XW;
    return chunk < nxw ? (L + F::NLW - 1) / F::NLW : (L + F::S - 1) / F::S;
}

template <int N, int MINB>
__global__ void __launch_bounds__(FUSED_THREADS, MINB) k_fused(FusedArgs a) {
    using F = FusedShape<N>;
    using C = typename F::C;
    using RC = typename F::RC;
    constexpr int S = F::S, P = F::P, L = F::L;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item, s_ok;
    const int nch = (N + 1) / F::XW + ((N + 1) - ((N + 1) / F::XW) * F::XW);
    const FusedCounters k(N, nch);
    for (;;) {
        __syncthreads();
        if (threadIdx.x == 0) s_item = (int)atomicAdd(a.ctl, 1u);
        __syncthreads();
        const int w = s_item;
        if (w >= a.total) return;
        const int2 e = a.order[w];
        const int pass = e.x, tile = e.y;
        int chunk = 0, l0 = 0, l1 = 0;  // planes (row and y passes) or lines (z)
        if (pass == 0 || pass == 4) {
            const int r0 = tile * 2 * P, r1 = min(a.rows, r0 + 2 * P);
            l0 = r0 / N;
            l1 = (r1 - 1) / N + 1;
        } else {
            col_tile_span<N>(tile, pass == 2 ? 2 * N : N, chunk, l0, l1);
        }
        if (threadIdx.x == 0) {
            bool ok = true;
            if (pass == 1) {
                for (int z = l0; z < l1 && ok; ++z) {
                    const int need = (z * N + N - 1) / (2 * P) - (z * N) / (2 * P) + 1;
                    ok = fused_wait(a.ctl + k.cx + z, (unsigned)need, a);
                }
            } else if (pass == 2) {
                ok = fused_wait(a.ctl + k.cy + chunk, (unsigned)col_chunk_tiles<N>(chunk, N), a);
            } else if (pass == 3) {
                ok = fused_wait(a.ctl + k.cz + chunk, (unsigned)col_chunk_tiles<N>(chunk, 2 * N), a);
            } else if (pass == 4) {
                for (int z = l0; z < l1 && ok; ++z) ok = fused_wait(a.ctl + k.cyi + z, (unsigned)nch, a);
            }
            s_ok = ok ? 1 : 0;
        }
        __syncthreads();
        if (!s_ok) return;
        switch (pass) {
            case 0: tile_x_fwd<RC, P, L, true>(a.p[0], a.rows, tile, smem_raw); break;
            case 1: tile_y_fwd<C, S, L, true>(a.p[1], tile, smem_raw); break;
            case 2: tile_z_conv<C, S, L, true>(a.p[2], tile, smem_raw); break;
            case 3: tile_y_inv<C, S, L, true>(a.p[3], tile, smem_raw); break;
            default: tile_x_inv<RC, P, L, true>(a.p[4], a.rows, tile, smem_raw); break;
        }
        // release: the barrier orders every thread's stores before thread 0's
        // device-scope fence, which orders them before the count update
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (pass == 0) {
                for (int z = l0; z < l1; ++z) atomicAdd(a.ctl + k.cx + z, 1u);
            } else if (pass == 1) {
                atomicAdd(a.ctl + k.cy + chunk, 1u);
            } else if (pass == 2) {
                atomicAdd(a.ctl + k.cz + chunk, 1u);
            } else if (pass == 3) {
                for (int z = l0; z < l1; ++z) atomicAdd(a.ctl + k.cyi + z, 1u);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

template <int N> struct FusedHost {
    using F = FusedShape<N>;
    static int nch() {
        const int nxw = (N + 1) / F::XW;
        return nxw + (N + 1) - nxw * F::XW;
    }
    static int row_tiles() { return (N * N + 2 * F::P - 1) / (2 * F::P); }
    // column tiles of one chunk for lines L, in line-group order
    static void chunk_tiles(int chunk, int L, std::vector<int>& out) {
        const int ncols = N + 1, nxw = ncols / F::XW;
        const int n_wide = nxw * ((L + F::NLW - 1) / F::NLW);
        out.clear();
        if (chunk < nxw) {
            const int nlt = (L + F::NLW - 1) / F::NLW;
            for (int lt = 0; lt < nlt; ++lt) out.push_back(chunk * nlt + lt);
        } else {
            const int cc = chunk - nxw, nln = (L + F::S - 1) / F::S;
            for (int lt = 0; lt < nln; ++lt) out.push_back(n_wide + cc * nln + lt);
        }
    }
    static std::vector<int2> order() {
        std::vector<int2> q;
        const int ntx = row_tiles(), nc = nch();
        for (int t = 0; t < ntx; ++t) q.push_back(make_int2(0, t));
        std::vector<int> tl;
        // lag of LAG chunks between the stages, so that a stage's tiles are
        // usually claimed after their inputs have finished
        constexpr int LAG = 3;
        for (int s = 0; s < nc + 2 * LAG; ++s) {
            if (s < nc) {
                chunk_tiles(s, N, tl);
                for (int t : tl) q.push_back(make_int2(1, t));
            }
            if (s - LAG >= 0 && s - LAG < nc) {
                chunk_tiles(s - LAG, 2 * N, tl);
                for (int t : tl) q.push_back(make_int2(2, t));
            }
            if (s - 2 * LAG >= 0 && s - 2 * LAG < nc) {
                chunk_tiles(s - 2 * LAG, N, tl);
                for (int t : tl) q.push_back(make_int2(3, t));
            }
        }
        for (int t = 0; t < ntx; ++t) q.push_back(make_int2(4, t));
        return q;
    }
    template <int MINB> static cudaError_t launch(const FusedArgs& a, cudaStream_t st) {
        const size_t sm = F::smem;
        cudaError_t e;
        if ((e = set_smem<SmemTag<30 + MINB, typename F::C, F::S, F::P>>(k_fused<N, MINB>, sm)) != cudaSuccess)
            return e;
        static int grid[64] = {0};
        int dev = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        const int d = dev < 64 ? dev : 0;
        if (grid[d] == 0) {
            int b = 0, sms = 0;
            if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_fused<N, MINB>, FUSED_THREADS, sm))) return e;
            if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
            grid[d] = std::max(1, b) * sms;
        }
        k_fused<N, MINB><<<std::min(grid[d], a.total), FUSED_THREADS, sm, st>>>(a);
        return cudaGetLastError();
    }
    static cudaError_t launch_mode(int mode, const FusedArgs& a, cudaStream_t st) {
        return mode == 2 ? launch<2>(a, st) : launch<3>(a, st);
    }
};

template <int N> cudaError_t fused_prepare_n(poisson_plan_s* pl, cudaStream_t st) {
    const std::vector<int2> q = FusedHost<N>::order();
    const FusedCounters k(N, FusedHost<N>::nch());
    cudaError_t e;
    if ((e = cudaMalloc(&pl->fused_order, q.size() * sizeof(int2)))) return e;
    if ((e = cudaMalloc(&pl->fused_ctl, (size_t)k.count * sizeof(unsigned)))) return e;
    if ((e = cudaMemcpyAsync(pl->fused_order, q.data(), q.size() * sizeof(int2), cudaMemcpyHostToDevice, st)))
        return e;
    pl->fused_total = (int)q.size();
    pl->fused_ctl_words = k.count;
    return cudaStreamSynchronize(st);  // q goes out of scope
}

}  // namespace

bool fused_supported(const poisson_plan_s* pl) {
    if (pl->prec != POISSON_FP32 || pl->nx != pl->ny || pl->nx != pl->nz) return false;
    switch (pl->nx) {
        case 64: case 128: case 192: case 256: case 384: case 512: return true;
        default: return false;
    }
}

cudaError_t fused_prepare(poisson_plan_s* pl, cudaStream_t st) {
    if (pl->fused_order) return cudaSuccess;
    switch (pl->nx) {
        case 64: return fused_prepare_n<64>(pl, st);
        case 128: return fused_prepare_n<128>(pl, st);
        case 192: return fused_prepare_n<192>(pl, st);
        case 256: return fused_prepare_n<256>(pl, st);
        case 384: return fused_prepare_n<384>(pl, st);
        case 512: return fused_prepare_n<512>(pl, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t fused_solve(const poisson_plan_s* pl, const PassParams<float> (&p)[5], cudaStream_t st) {
    FusedArgs a{};
    for (int i = 0; i < 5; ++i) a.p[i] = p[i];
    a.n = pl->nx;
    a.rows = pl->ny * pl->nz;
    a.order = static_cast<const int2*>(pl->fused_order);
    a.total = pl->fused_total;
    a.ctl = static_cast<unsigned*>(pl->fused_ctl);
    a.status = pl->status;
    a.spin_limit = 1LL << 24;
    cudaError_t e = cudaMemsetAsync(a.ctl, 0, (size_t)pl->fused_ctl_words * sizeof(unsigned), st);
    if (e != cudaSuccess) return e;
    const int m = pl->use_fused;
    switch (pl->nx) {
        case 64: return FusedHost<64>::launch_mode(m, a, st);
        case 128: return FusedHost<128>::launch_mode(m, a, st);
        case 192: return FusedHost<192>::launch_mode(m, a, st);
        case 256: return FusedHost<256>::launch_mode(m, a, st);
        case 384: return FusedHost<384>::launch_mode(m, a, st);
        case 512: return FusedHost<512>::launch_mode(m, a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pgb
