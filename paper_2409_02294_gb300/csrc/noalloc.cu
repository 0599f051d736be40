// poisson_solve_noalloc: a complete small-grid solve that allocates nothing.
//
// Who needs it: callers that must not call cudaMalloc at the moment they
// solve.  Examples are code running under a framework whose caching
// allocator owns all device memory (a stray cudaMalloc can fail or fragment
// the pool), code with a fixed device-memory budget decided up front, and
// code that cannot afford the device-wide synchronisation that cudaMalloc and
// cudaFree may imply.  A plan (poisson_plan_create) allocates its workspace,
// Green's function and tables; this entry point instead keeps all of them in
// one fixed device array that is part of the library image, so a solve needs
// only the caller's input and output buffers.
//
// The scratch array: kNoAllocScratchBytes (16 MiB) of device memory, declared
// at file scope below.  Every GPU that loads the library holds it until the
// process exits.  It is shared by every call on a device and keeps the last
// call's contents; nothing in it has to start at zero, because each call
// writes every value it later reads.  Calls whose GPU work overlaps in time
// (e.g. on two streams) race on it: issue them on one stream or serialise.
//
// Set-up: the first call on each device looks up the array's device address
// with cudaGetSymbolAddress (in host code the array's name is only a
// host-side stand-in, not a device address) and caches it per device,
// together with the identity of the CUDA context it was taken in; a call in
// a new context on that device (after cudaDeviceReset, say) looks it up
// again.  Make the first call on each device, and the first after a device
// reset, before any stream capture begins.
//
// Per call (all on the caller's stream): FP64 Green's kernel octant, its
// DCT-I along x, y, z and scaling to an FP32 octant, the twiddle tables, then
// the same five passes as poisson_solve.  The Green's function is rebuilt on
// every call; this entry point trades that cost for needing no plan.
#include <cudaTypedefs.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "configs.cuh"
#include "internal.h"
#include "poisson.h"

namespace {

constexpr size_t kNoAllocScratchBytes = 16u << 20;  // 16 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};
unsigned long long g_scratch_ctx[kMaxDevices] = {};  // context id the address belongs to

// Unique id of the calling thread's current CUDA context (driver entry
// points, no link against libcuda); 0 if it cannot be read.
unsigned long long current_context_id() {
    static std::once_flag once;
    static PFN_cuCtxGetCurrent_v4000 get_current = nullptr;
    static PFN_cuCtxGetId_v12000 get_id = nullptr;
    std::call_once(once, [] {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 4000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<PFN_cuCtxGetCurrent_v4000>(fn);
        fn = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &fn, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<PFN_cuCtxGetId_v12000>(fn);
    });
    if (!get_current || !get_id) return 0;
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Byte offsets of every buffer inside the scratch array for one grid.
struct Layout {
    size_t tw[3];      // axis twiddle tables (float2): W_2n^j, then the stage tables
    size_t ghat;       // greens_elems<float>(nx, ny, nz) floats (block layout)
    size_t work;       // union of {k octant, tmp, DCT-I matrices} (double) and {W1, W2} (float2)
    size_t dct[3];     // (n+1)^2 DCT-I matrices (double), one per axis, inside the work region
    size_t w2;         // offset of W2 inside the work region
    size_t ktmp;       // offset of the second k buffer inside the work region
    size_t total;
    long long sx;      // complex row stride of W1/W2
};

Layout make_layout(int nx, int ny, int nz) {
    Layout L{};
    const int n[3] = {nx, ny, nz};
    size_t off = 0;
    for (int a = 0; a < 3; ++a) {
        L.tw[a] = off;
        off += align256((size_t)pgb::axis_tw_list<float>(n[a], a == 0).total * sizeof(float2));
    }
    const size_t oct = (size_t)(nx + 1) * (ny + 1) * (nz + 1);
    L.ghat = off;
    off += align256((size_t)pgb::greens_elems<float>(nx, ny, nz) * sizeof(float));
    L.sx = ((long long)(nx + 1) + 15) / 16 * 16;
    const size_t w1 = (size_t)nz * ny * L.sx * sizeof(float2);
    const size_t kb = align256(oct * sizeof(double));
    L.work = off;
    L.w2 = align256(w1);
    L.ktmp = kb;
    // the DCT-I matrices are needed only while the Green's function is
    // built, before W1/W2 are written
    size_t build = 2 * kb;
    for (int a = 0; a < 3; ++a) {
        L.dct[a] = off + build;
        build += align256((size_t)(n[a] + 1) * (n[a] + 1) * sizeof(double));
    }
    const size_t work = std::max(L.w2 + 2 * w1, build);
    L.total = off + align256(work);
    return L;
}

// W_2n^j = exp(-i pi j / n), j < 2n, from the FP64 sincospi, rounded once.
__global__ void k_noalloc_twiddles(float2* __restrict__ tw, int n) {
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < 2 * n; j += gridDim.x * blockDim.x) {
        double s, c;
        sincospi((double)j / (double)n, &s, &c);
        tw[j] = make_float2((float)c, (float)-s);
    }
}

// C[q][d] = w_d cos(pi (q d mod 2n) / n), w_0 = w_n = 1, else 2.
__global__ void k_noalloc_dct(double* __restrict__ C, int n) {
    const int e = n + 1;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < e * e; i += gridDim.x * blockDim.x) {
        const int q = i / e, d = i % e;
        const long long r = ((long long)q * d) % (2LL * n);
        const double w = (d == 0 || d == n) ? 1.0 : 2.0;
        C[i] = w * cospi((double)r / (double)n);
    }
}

poisson_status to_status(cudaError_t e) {
    if (e == cudaSuccess) return POISSON_OK;
    if (e == cudaErrorMemoryAllocation) return POISSON_ERR_ALLOC;
    return POISSON_ERR_CUDA;
}

// Device address of the scratch array on the current device (set up once
// per device and context).
cudaError_t scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    // before the first CUDA call of the process there may be no current
    // context (id 0): the lookup then runs, initialises the device's primary
    // context, and the id is read again after it
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    const unsigned long long ctx = current_context_id();
    if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = p;
        g_scratch_ctx[dev] = current_context_id();
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return cudaSuccess;
}

}  // namespace

extern "C" poisson_status poisson_solve_noalloc(int nx, int ny, int nz, double hx, double hy,
                                                double hz, double G, const void* rho_dev,
                                                void* phi_dev, void* cuda_stream) {
    using namespace pgb;
    if (!rho_dev || !phi_dev) return POISSON_ERR_ARG;
    if (((reinterpret_cast<uintptr_t>(rho_dev) | reinterpret_cast<uintptr_t>(phi_dev)) & 15u) != 0)
        return POISSON_ERR_ARG;
    if (!(hx > 0.0) || !(hy > 0.0) || !(hz > 0.0) || !std::isfinite(hx) || !std::isfinite(hy) ||
        !std::isfinite(hz) || !std::isfinite(G))
        return POISSON_ERR_ARG;
    if (nx <= 0 || ny <= 0 || nz <= 0) return POISSON_ERR_ARG;
    if (!size_supported(nx) || !size_supported(ny) || !size_supported(nz)) return POISSON_ERR_UNSUPPORTED;
    const Layout L = make_layout(nx, ny, nz);
    if (L.total > kNoAllocScratchBytes) return POISSON_ERR_ARG;  // grid too large for the array

    unsigned char* base = nullptr;
    cudaError_t e = scratch_address(&base);
    if (e != cudaSuccess) return to_status(e);
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int n[3] = {nx, ny, nz};

    float2* tw[3];
    double* dct[3];
    for (int a = 0; a < 3; ++a) {
        tw[a] = reinterpret_cast<float2*>(base + L.tw[a]);
        dct[a] = reinterpret_cast<double*>(base + L.dct[a]);
        k_noalloc_twiddles<<<(2 * n[a] + 255) / 256, 256, 0, st>>>(tw[a], n[a]);
        if ((e = fill_stage_twiddles<float>(reinterpret_cast<cpx<float>*>(tw[a]), n[a], a == 0, st)) != cudaSuccess)
            return to_status(e);
        const int e2 = (n[a] + 1) * (n[a] + 1);
        k_noalloc_dct<<<(e2 + 255) / 256, 256, 0, st>>>(dct[a], n[a]);
    }
    if ((e = cudaGetLastError()) != cudaSuccess) return to_status(e);

    float* ghat = reinterpret_cast<float*>(base + L.ghat);
    double* kbuf = reinterpret_cast<double*>(base + L.work);
    double* ktmp = reinterpret_cast<double*>(base + L.work + L.ktmp);
    if ((e = build_kernel_octant(nx, ny, nz, hx, hy, hz, POISSON_R_NEAR_DEFAULT, kbuf, st)) != cudaSuccess)
        return to_status(e);
    const double scale = -G * hx * hy * hz / (8.0 * (double)nx * (double)ny * (double)nz);
    if ((e = greens_transform_into(kbuf, ktmp, dct[0], dct[1], dct[2], nx, ny, nz, scale, ghat, st)) !=
        cudaSuccess)
        return to_status(e);

    // the five passes; W1/W2 reuse the k buffers' region (stream-ordered)
    void* w1 = base + L.work;
    void* w2 = base + L.work + L.w2;
    for (int pass = 0; pass < 5; ++pass) {
        PassParams<float> p{};
        p.nx = nx;
        p.ny = ny;
        p.nz = nz;
        p.sx = L.sx;
        p.greens = ghat;
        int N = 0;
        switch (pass) {
            case 0: p.in = rho_dev; p.out = w1; N = nx; p.tw = reinterpret_cast<const cpx<float>*>(tw[0]); break;
            case 1: p.in = w1; p.out = w2; N = ny; p.tw = reinterpret_cast<const cpx<float>*>(tw[1]); break;
            case 2: p.in = w2; p.out = w2; N = nz; p.tw = reinterpret_cast<const cpx<float>*>(tw[2]); break;
            case 3: p.in = w2; p.out = w1; N = ny; p.tw = reinterpret_cast<const cpx<float>*>(tw[1]); break;
            default: p.in = w1; p.out = phi_dev; N = nx; p.tw = reinterpret_cast<const cpx<float>*>(tw[0]); break;
        }
        if ((e = launch_pass_f32(N, pass, (pass == 0 || pass == 4) ? kRowVarPlain : kColVarPlain, p, ny * nz,
                                 st)) != cudaSuccess)
            return to_status(e);
    }
    return POISSON_OK;
}
