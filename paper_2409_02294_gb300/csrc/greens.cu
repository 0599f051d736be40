// Plan-time Green's function in FP64 on the GPU.
//
// 1. k(d) on the octant d in [0,nx] x [0,ny] x [0,nz] of the padded periodic
//    grid (M = 2n, so the wrapped offset of index m is min(m, M - m)):
//    - |d|_inf <= r_near: mean of 1/|r| over the source cell, the box of
//      size h centred at d h, from the closed-form antiderivative of 1/r
//      (the potential of a homogeneous rectangular prism);
//    - otherwise the point value 1/|d h|.
// 2. Its M-point DFT per axis.  k is real and even in every axis, so the
//    transform is real and even too and reduces to a DCT-I on the octant:
//      K^(q) = sum_{d=0}^{n} c_d k(d) cos(pi q d / n),  c_0 = c_n = 1, else 2,
//    applied along x, y, z by FP64 line FFTs (greens_dct.cu) for plans, and
//    as dense FP64 matrix products (a tiled DGEMM) for the no-allocation
//    solve's small grids.
// 3. Scale by -G V / (Mx My Mz) (sign, cell volume and the inverse-FFT
//    normalisation folded in) and store in the data-path precision.
#include <algorithm>
#include <cmath>

#include "greens_dct.h"
#include "greens_layout.h"
#include "internal.h"

namespace pgb {

// ---------------------------------------------------------------------------
// k(d)
// ---------------------------------------------------------------------------

// ln(a + r) for r = |(a, b, c)|, rewritten as ln((b^2 + c^2) / (r - a)) when
// a < 0 so that no digits cancel.
__device__ __forceinline__ double ln_a_plus_r(double a, double b, double c, double r) {
    return a >= 0.0 ? log(a + r) : log((b * b + c * c) / (r - a));
}

// Antiderivative P(x,y,z) of 1/r in all three variables:
//   yz ln(x+r) + zx ln(y+r) + xy ln(z+r)
//   - x^2/2 atan(yz/(xr)) - y^2/2 atan(zx/(yr)) - z^2/2 atan(xy/(zr)).
__device__ double prism_p(double x, double y, double z) {
    const double r = sqrt(x * x + y * y + z * z);
    double acc = 0.0;
    if (y != 0.0 && z != 0.0) acc += y * z * ln_a_plus_r(x, y, z, r);
    if (z != 0.0 && x != 0.0) acc += z * x * ln_a_plus_r(y, z, x, r);
    if (x != 0.0 && y != 0.0) acc += x * y * ln_a_plus_r(z, x, y, r);
    if (x != 0.0) acc -= 0.5 * x * x * atan(y * z / (x * r));
    if (y != 0.0) acc -= 0.5 * y * y * atan(z * x / (y * r));
    if (z != 0.0) acc -= 0.5 * z * z * atan(x * y / (z * r));
    return acc;
}

__device__ double cell_mean_inv_r(double cx, double cy, double cz, double hx, double hy, double hz) {
    // sum over the 8 corners; corner bit set = upper limit, sign (-1)^(#lower)
    double s = 0.0;
#pragma unroll
    for (int corner = 0; corner < 8; ++corner) {
        const int ux = corner & 1, uy = (corner >> 1) & 1, uz = (corner >> 2) & 1;
        const double x = cx + (ux ? 0.5 : -0.5) * hx;
        const double y = cy + (uy ? 0.5 : -0.5) * hy;
        const double z = cz + (uz ? 0.5 : -0.5) * hz;
        const int lowers = 3 - ux - uy - uz;
        s += ((lowers & 1) ? -1.0 : 1.0) * prism_p(x, y, z);
    }
    return s / (hx * hy * hz);
}

__global__ void k_kernel_octant(double* __restrict__ out, int ex, int ey, int ez, double hx,
                                double hy, double hz, int r_near) {
    const long long total = (long long)ex * ey * ez;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int dx = (int)(i % ex);
        const int dy = (int)((i / ex) % ey);
        const int dz = (int)(i / ((long long)ex * ey));
        const int cheb = max(dx, max(dy, dz));
        double v;
        if (cheb <= r_near) {
            v = cell_mean_inv_r(dx * hx, dy * hy, dz * hz, hx, hy, hz);
        } else {
            const double x = dx * hx, y = dy * hy, z = dz * hz;
            v = 1.0 / sqrt(x * x + y * y + z * z);
        }
        out[i] = v;
    }
}

// ---------------------------------------------------------------------------
// strided batched FP64 matrix product: D[b][i][j] = sum_l A[b][i][l] B[b][l][j]
// ---------------------------------------------------------------------------
struct GemmDesc {
    const double* A;
    const double* B;
    double* D;
    long long sAb, sAi, sAl;
    long long sBb, sBl, sBj;
    long long sDb, sDi, sDj;
    int I, J, L;
};

constexpr int GT = 64;   // tile edge
constexpr int GK = 16;   // contraction step

__global__ void __launch_bounds__(256) k_dgemm(GemmDesc g) {
    __shared__ double As[GK][GT + 1];
    __shared__ double Bs[GK][GT + 1];
    const int b = blockIdx.z;
    const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
    const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
    const double* A = g.A + b * g.sAb;
    const double* B = g.B + b * g.sBb;
    double acc[4][4] = {};
    for (int l0 = 0; l0 < g.L; l0 += GK) {
        for (int e = threadIdx.x; e < GK * GT; e += 256) {
            const int ll = e % GK, ii = e / GK;
            const int i = i0 + ii, l = l0 + ll;
            As[ll][ii] = (i < g.I && l < g.L) ? A[i * g.sAi + l * g.sAl] : 0.0;
        }
        for (int e = threadIdx.x; e < GK * GT; e += 256) {
            const int jj = e % GT, ll = e / GT;
            const int j = j0 + jj, l = l0 + ll;
            Bs[ll][jj] = (j < g.J && l < g.L) ? B[l * g.sBl + j * g.sBj] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int ll = 0; ll < GK; ++ll) {
            double a[4], bb[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) a[u] = As[ll][ty + 16 * u];
#pragma unroll
            for (int u = 0; u < 4; ++u) bb[u] = Bs[ll][tx + 16 * u];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], bb[v], acc[u][v]);
        }
        __syncthreads();
    }
    double* D = g.D + b * g.sDb;
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = i0 + ty + 16 * u, j = j0 + tx + 16 * v;
            if (i < g.I && j < g.J) D[i * g.sDi + j * g.sDj] = acc[u][v];
        }
}

static cudaError_t dgemm(const GemmDesc& g, int batch, cudaStream_t st) {
    dim3 grid((g.J + GT - 1) / GT, (g.I + GT - 1) / GT, batch);
    k_dgemm<<<grid, 256, 0, st>>>(g);
    return cudaGetLastError();
}

// Scale the dense octant in[kz][ky][kx] and store it in the block layout of
// greens_layout.h (zeros beyond kx = nx), one output element per step.
template <class R>
__global__ void k_scale_store(const double* __restrict__ in, int nx, int ny, int nz, double s, R* __restrict__ out) {
    constexpr int XW = greens_xw<R>();
    const long long n = greens_elems<R>(nx, ny, nz), bands = greens_bands<R>(nx);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long r = i / XW, blk = r / (nz + 1);
        const int kz = (int)(r - blk * (nz + 1)), ky = (int)(blk / bands);
        const int kx = (int)(blk - ky * bands) * XW + (int)(i - r * XW);
        out[i] = kx <= nx ? (R)(s * in[((long long)kz * (ny + 1) + ky) * (nx + 1) + kx]) : (R)0;
    }
}

static cudaError_t scale_store(const double* in, int nx, int ny, int nz, double s, float* of, double* od,
                               cudaStream_t st) {
    const long long n = of ? greens_elems<float>(nx, ny, nz) : greens_elems<double>(nx, ny, nz);
    const int blocks = (int)std::min<long long>((n + 255) / 256, 152LL * 16);
    if (of) k_scale_store<float><<<blocks, 256, 0, st>>>(in, nx, ny, nz, s, of);
    else k_scale_store<double><<<blocks, 256, 0, st>>>(in, nx, ny, nz, s, od);
    return cudaGetLastError();
}

#define PGB_TRY(x)                              \
    do {                                        \
        cudaError_t e_ = (x);                   \
        if (e_ != cudaSuccess) return e_;       \
    } while (0)

cudaError_t build_kernel_octant(int nx, int ny, int nz, double hx, double hy, double hz,
                                int r_near, double* out, cudaStream_t st) {
    const int ex = nx + 1, ey = ny + 1, ez = nz + 1;
    const long long total = (long long)ex * ey * ez;
    int blocks = (int)std::min<long long>((total + 255) / 256, 152LL * 16);
    k_kernel_octant<<<blocks, 256, 0, st>>>(out, ex, ey, ez, hx, hy, hz, r_near);
    return cudaGetLastError();
}

cudaError_t build_greens(int nx, int ny, int nz, double hx, double hy, double hz, int r_near,
                         double scale, float* out_f32, double* out_f64, cudaStream_t st,
                         const double* user_octant) {
    const int ex = nx + 1, ey = ny + 1, ez = nz + 1;
    const long long total = (long long)ex * ey * ez;
    double *k0 = nullptr, *k1 = nullptr;
    cpx<double>* tw[3] = {nullptr, nullptr, nullptr};
    cudaError_t err = cudaSuccess;
    do {
        if ((err = cudaMalloc(&k0, total * sizeof(double))) != cudaSuccess) break;
        if ((err = cudaMalloc(&k1, total * sizeof(double))) != cudaSuccess) break;
        const int n[3] = {nx, ny, nz};
        for (int a = 0; a < 3 && err == cudaSuccess; ++a)
            err = cudaMalloc(&tw[a], dct1_twiddle_entries(n[a]) * sizeof(cpx<double>));
        if (err != cudaSuccess) break;
        if (user_octant) {  // a caller's kernel octant (host memory) instead of the Green's kernel
            if ((err = cudaMemcpyAsync(k0, user_octant, total * sizeof(double), cudaMemcpyHostToDevice, st)))
                break;
        } else if ((err = build_kernel_octant(nx, ny, nz, hx, hy, hz, r_near, k0, st))) {
            break;
        }
        if ((err = dct1_octant(k0, k1, tw, nx, ny, nz, st))) break;  // result in k1
        if ((err = scale_store(k1, nx, ny, nz, scale, out_f32, out_f64, st))) break;
        err = cudaStreamSynchronize(st);
    } while (0);
    if (err != cudaSuccess) cudaStreamSynchronize(st);  // no queued work may outlive the buffers
    cudaFree(k0);
    cudaFree(k1);
    for (int a = 0; a < 3; ++a) cudaFree(tw[a]);
    return err;
}

}  // namespace pgb

namespace pgb {

// The DCT-I transform and scaling of build_greens on caller-provided device
// buffers, with nothing allocated and nothing synchronised: kbuf holds the
// k(d) octant on entry and is overwritten, tmp has the same size, cx/cy/cz
// are the (n+1)^2 DCT-I matrices of the three axes, out receives the scaled
// FP32 octant (block layout of greens_layout.h).  All work is queued on st.
cudaError_t greens_transform_into(double* kbuf, double* tmp, const double* cx, const double* cy,
                                  const double* cz, int nx, int ny, int nz, double scale,
                                  float* out, cudaStream_t st) {
    const int ex = nx + 1, ey = ny + 1, ez = nz + 1;
    GemmDesc g{};
    g.A = kbuf; g.sAi = ex; g.sAl = 1;
    g.B = cx; g.sBl = 1; g.sBj = ex;
    g.D = tmp; g.sDi = ex; g.sDj = 1;
    g.I = ey * ez; g.J = ex; g.L = ex;
    PGB_TRY(dgemm(g, 1, st));
    g = GemmDesc{};
    g.A = cy; g.sAi = ey; g.sAl = 1;
    g.B = tmp; g.sBb = (long long)ey * ex; g.sBl = ex; g.sBj = 1;
    g.D = kbuf; g.sDb = (long long)ey * ex; g.sDi = ex; g.sDj = 1;
    g.I = ey; g.J = ex; g.L = ey;
    PGB_TRY(dgemm(g, ez, st));
    g = GemmDesc{};
    g.A = cz; g.sAi = ez; g.sAl = 1;
    g.B = kbuf; g.sBl = (long long)ey * ex; g.sBj = 1;
    g.D = tmp; g.sDi = (long long)ey * ex; g.sDj = 1;
    g.I = ez; g.J = ey * ex; g.L = ez;
    PGB_TRY(dgemm(g, 1, st));
    return scale_store(tmp, nx, ny, nz, scale, out, nullptr, st);
}

}  // namespace pgb
