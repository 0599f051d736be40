// Batched solve of many independent fields of uneven sizes, replayed from a
// CUDA graph, in one of two executions (the first call times both on the
// caller's data and keeps the faster; POISSON_BATCH_MODE=0/1 forces one):
//
//  mode 0: ONE persistent kernel over the tiles of all fields (below);
//  mode 1: every field's own five kernels (each plan's own, possibly
//          autotuned, variants), captured once into a graph whose branches
//          spread the fields over four streams (largest fields first, each
//          to the least loaded stream), so small fields run side by side;
//  mode 2: the same graph with the variants plans use untuned: variants
//          tuned for a field alone on the GPU are not always the best ones
//          when fields share it.
//
// Work items are runs of up to GROUP consecutive tiles of one pass of one
// field (fewer for small passes, so that every pass still splits into many
// items).  The queue is laid out pass-major (all x-forward items, then all
// y-forward items, ...) with larger fields first inside a pass.  CTAs claim
// items with an atomic counter; an item of pass p of field f first waits
// until every tile of pass p-1 of field f has finished (per-(field, pass)
// completion counters, counted in tiles), and publishes its own tiles with
// one release after the last of them.  A
// wait only ever targets items earlier in the queue, which were claimed by
// CTAs that are already running, so the scheme cannot deadlock however many
// CTAs are resident.  Every wait is bounded: after `spin_limit` polls it sets
// the timeout bit in the status word of the first plan, raises an abort flag
// that makes every other CTA stop, and the kernel returns.
//
// Data produced inside the launch is read with L1-bypassing loads (the tile
// functions' CG = true instantiation); completion is published by one
// thread with a device-scope fence after the CTA barrier and before the
// counter increment, and observed with an acquire load.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "configs.cuh"
#include "internal.h"
#include "plan.h"

namespace pgb {

constexpr int BATCH_THREADS = 128;
using BatchVar = Var<2, BATCH_THREADS>;  // both halves of a line per thread, as the standalone kernels

struct BatchField {
    PassParams<float> p[5];
    int N[5];        // transform length of each pass
    int ntiles[5];
    int rows;        // ny * nz (row passes)
};

struct BatchSeg {
    int field, pass;
    int begin;   // first work item of the segment
    int ntiles;  // tiles of this pass of this field
    int group;   // tiles per work item (the last item may hold fewer)
};

// Tiles per work item for a pass of `ntiles` tiles: up to 8, while keeping
// at least about a thousand items in the pass.
inline int seg_group(int ntiles) { return std::max(1, std::min(8, ntiles / 1024)); }

struct BatchArgs {
    const BatchField* fields;
    const BatchSeg* segs;
    int nseg;
    int total;
    unsigned* ctl;           // [0] work counter, [1] abort flag, [2..] done counters
    unsigned* status;        // status word of the first plan (bit 1: timeout)
    long long spin_limit;    // polls before a dependency wait gives up
    int hold_field;          // test hook: this field's pass-0 count is never enough (-1: off)
};

template <int N> struct BatchShape {
    using C = typename SizeCfg<float, N>::C;      // column tiles
    using RC = typename RowSizeCfg<float, N>::C;  // row tiles
    static constexpr int S = var_slots<C, BatchVar>();
    static constexpr int P = var_pairs<RC, BatchVar>();
    static_assert(col_threads<C, S, 2>() == BATCH_THREADS, "column tile must use BATCH_THREADS threads");
    static_assert(row_threads<RC, P, 2>() == BATCH_THREADS, "row tile must use BATCH_THREADS threads");
    static constexpr size_t smem = col_smem_z<C, S>() > row_smem<RC, P>() ? col_smem_z<C, S>() : row_smem<RC, P>();
};

template <int N>
__device__ __noinline__ void batch_tile(int pass, const PassParams<float>& p, int rows, int tile,
                                           unsigned char* sm) {
    using C = typename BatchShape<N>::C;
    using RC = typename BatchShape<N>::RC;
    constexpr int S = BatchShape<N>::S, P = BatchShape<N>::P;
    switch (pass) {
        case 0: tile_x_fwd<RC, P, 2, true>(p, rows, tile, sm); break;
        case 1: tile_y_fwd<C, S, 2, true>(p, tile, sm); break;
        case 2: tile_z_conv<C, S, 2, true>(p, tile, sm); break;
        case 3: tile_y_inv<C, S, 2, true>(p, tile, sm); break;
        default: tile_x_inv<RC, P, 2, true>(p, rows, tile, sm); break;
    }
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Bounded wait for *ctr >= target.  Returns false on timeout or abort.
__device__ bool wait_count(const unsigned* ctr, unsigned target, const BatchArgs& a) {
    for (long long it = 0; it < a.spin_limit; ++it) {
        if (ld_acquire_u32(ctr) >= target) return true;
        if (ld_acquire_u32(a.ctl + 1) != 0u) return false;
        __nanosleep(128);
    }
    atomicOr(a.status, 2u);
    atomicExch(a.ctl + 1, 1u);
    return false;
}

// Thread 0 claims the CTA's next item while the current one runs (a claim
// only ever comes after the CTA's current item in the queue, so the
// argument above still holds), and remembers the last (field, pass)
// dependency it saw complete, so the following tiles of that pass skip the
// poll.
__global__ void __launch_bounds__(BATCH_THREADS, 3) k_batched(BatchArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item, s_ok;
    unsigned next = 0;  // thread 0: the item claimed for after the current one
    int dep_done = -1;  // thread 0: field * 5 + pass of the last counter seen complete
    if (threadIdx.x == 0) next = atomicAdd(a.ctl, 1u);
    for (;;) {
        __syncthreads();  // the previous tile is done with shared memory
        if (threadIdx.x == 0) s_item = (int)next;
        __syncthreads();
        const int w = s_item;
        if (w >= a.total) return;
        if (threadIdx.x == 0) next = atomicAdd(a.ctl, 1u);
        // segment holding work item w (segments are sorted by begin)
        int lo = 0, hi = a.nseg - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (a.segs[mid].begin <= w) lo = mid;
            else hi = mid - 1;
        }
        const BatchSeg sg = a.segs[lo];
        const BatchField& f = a.fields[sg.field];
        const int t_first = (w - sg.begin) * sg.group;
        const int t_count = min(sg.group, sg.ntiles - t_first);
        if (threadIdx.x == 0) {
            bool ok = true;
            const int key = sg.field * 5 + sg.pass - 1;
            if (sg.pass > 0 && key != dep_done) {
                unsigned target = (unsigned)f.ntiles[sg.pass - 1];
                const bool held = sg.field == a.hold_field && sg.pass == 1;
                if (held) target += 1u;  // test hook
                ok = wait_count(a.ctl + 2 + key, target, a);
                if (ok && !held) dep_done = key;
            }
            s_ok = ok ? 1 : 0;
        }
        __syncthreads();
        if (!s_ok) return;  // timeout or abort: the whole CTA leaves together
        const PassParams<float>& p = f.p[sg.pass];
        for (int i = 0; i < t_count; ++i) {
            if (i > 0) __syncthreads();  // the previous tile is done with shared memory
            const int tile = t_first + i;
            switch (f.N[sg.pass]) {
                case 16: batch_tile<16>(sg.pass, p, f.rows, tile, smem_raw); break;
                case 32: batch_tile<32>(sg.pass, p, f.rows, tile, smem_raw); break;
                case 48: batch_tile<48>(sg.pass, p, f.rows, tile, smem_raw); break;
                case 64: batch_tile<64>(sg.pass, p, f.rows, tile, smem_raw); break;
                case 96: batch_tile<96>(sg.pass, p, f.rows, tile, smem_raw); break;
                case 128: batch_tile<128>(sg.pass, p, f.rows, tile, smem_raw); break;
                case 192: batch_tile<192>(sg.pass, p, f.rows, tile, smem_raw); break;
                case 256: batch_tile<256>(sg.pass, p, f.rows, tile, smem_raw); break;
                case 384: batch_tile<384>(sg.pass, p, f.rows, tile, smem_raw); break;
                default: batch_tile<512>(sg.pass, p, f.rows, tile, smem_raw); break;
            }
        }
        // release: the barrier orders every thread's stores before thread 0's
        // device-scope fence, which orders them before the count update
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(a.ctl + 2 + sg.field * 5 + sg.pass, (unsigned)t_count);
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
namespace {

// shared memory of the largest tile among the edge lengths present
size_t shape_smem(int N) {
    switch (N) {
        case 16: return BatchShape<16>::smem;
        case 32: return BatchShape<32>::smem;
        case 48: return BatchShape<48>::smem;
        case 64: return BatchShape<64>::smem;
        case 96: return BatchShape<96>::smem;
        case 128: return BatchShape<128>::smem;
        case 192: return BatchShape<192>::smem;
        case 256: return BatchShape<256>::smem;
        case 384: return BatchShape<384>::smem;
        default: return BatchShape<512>::smem;
    }
}
size_t batch_smem(const std::vector<poisson_plan_t>& plans) {
    size_t m = 0;
    for (const poisson_plan_s* pl : plans)
        m = std::max({m, shape_smem(pl->nx), shape_smem(pl->ny), shape_smem(pl->nz)});
    return m;
}

template <int N> int tiles_n(int pass, int nx, int ny, int nz) {
    constexpr int S = BatchShape<N>::S, P = BatchShape<N>::P;
    if (pass == 0 || pass == 4) return (ny * nz + 2 * P - 1) / (2 * P);
    return col_grid<float, S>(nx + 1, pass == 2 ? 2 * ny : nz);
}
int tiles_for(int N, int pass, int nx, int ny, int nz) {
    switch (N) {
        case 16: return tiles_n<16>(pass, nx, ny, nz);
        case 32: return tiles_n<32>(pass, nx, ny, nz);
        case 48: return tiles_n<48>(pass, nx, ny, nz);
        case 64: return tiles_n<64>(pass, nx, ny, nz);
        case 96: return tiles_n<96>(pass, nx, ny, nz);
        case 128: return tiles_n<128>(pass, nx, ny, nz);
        case 192: return tiles_n<192>(pass, nx, ny, nz);
        case 256: return tiles_n<256>(pass, nx, ny, nz);
        case 384: return tiles_n<384>(pass, nx, ny, nz);
        default: return tiles_n<512>(pass, nx, ny, nz);
    }
}

constexpr int BATCH_STREAMS = 4;

struct BatchState {
    std::vector<poisson_plan_t> plans;
    int hold_field = -1;
    int mode = -1;                   // 0 persistent kernel, 1/2 per-field launches, -1 undecided
    cudaStream_t side[BATCH_STREAMS] = {};
    cudaEvent_t fork = nullptr, join[BATCH_STREAMS] = {};
    cudaGraphExec_t lexec[2] = {};   // mode 1 and mode 2 graphs, for the pointers in lrho/lphi
    std::vector<const void*> lrho[2];
    std::vector<void*> lphi[2];
    int device = 0;
    BatchField* h_fields = nullptr;  // pinned mirror of d_fields
    BatchField* d_fields = nullptr;
    BatchSeg* d_segs = nullptr;
    unsigned* d_ctl = nullptr;
    size_t ctl_bytes = 0;
    cudaEvent_t copied = nullptr;    // last mirror -> device copy
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool have_ptrs = false;
};

std::mutex g_mu;
std::vector<BatchState*> g_cache;

void destroy_state(BatchState* b) {
    if (!b) return;
    for (int k = 0; k < 2; ++k)
        if (b->lexec[k]) cudaGraphExecDestroy(b->lexec[k]);
    for (int k = 0; k < BATCH_STREAMS; ++k) {
        if (b->side[k]) cudaStreamDestroy(b->side[k]);
        if (b->join[k]) cudaEventDestroy(b->join[k]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->copied) cudaEventDestroy(b->copied);
    cudaFreeHost(b->h_fields);
    cudaFree(b->d_fields);
    cudaFree(b->d_segs);
    cudaFree(b->d_ctl);
    delete b;
}

PassParams<float> pass_params(const poisson_plan_s* pl, int pass) {
    PassParams<float> p{};
    p.nx = pl->nx;
    p.ny = pl->ny;
    p.nz = pl->nz;
    p.sx = pl->sx;
    p.status = pl->status;
    p.greens = static_cast<const float*>(pl->greens);
    p.check_finite = pass == 4 && (pl->flags & POISSON_FLAG_CHECK_FINITE) != 0;
    switch (pass) {
        case 0: p.in = nullptr; p.out = pl->w1; p.tw = static_cast<const cpx<float>*>(pl->tw[0]); break;
        case 1: p.in = pl->w1; p.out = pl->w2; p.tw = static_cast<const cpx<float>*>(pl->tw[1]); break;
        case 2: p.in = pl->w2; p.out = pl->w2; p.tw = static_cast<const cpx<float>*>(pl->tw[2]); break;
        case 3: p.in = pl->w2; p.out = pl->w1; p.tw = static_cast<const cpx<float>*>(pl->tw[1]); break;
        default: p.in = pl->w1; p.out = nullptr; p.tw = static_cast<const cpx<float>*>(pl->tw[0]); break;
    }
    return p;
}

cudaError_t build_state(BatchState* b) {
    const int n = (int)b->plans.size();
    cudaError_t e;
    if ((e = cudaMallocHost(&b->h_fields, n * sizeof(BatchField)))) return e;
    if ((e = cudaMalloc(&b->d_fields, n * sizeof(BatchField)))) return e;
    if ((e = cudaEventCreateWithFlags(&b->copied, cudaEventDisableTiming))) return e;
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) {
        const poisson_plan_s* pl = b->plans[i];
        BatchField& f = b->h_fields[i];
        std::memset(&f, 0, sizeof(f));
        const int axisN[5] = {pl->nx, pl->ny, pl->nz, pl->ny, pl->nx};
        for (int pass = 0; pass < 5; ++pass) {
            f.p[pass] = pass_params(pl, pass);
            f.N[pass] = axisN[pass];
            f.ntiles[pass] = tiles_for(axisN[pass], pass, pl->nx, pl->ny, pl->nz);
        }
        f.rows = pl->ny * pl->nz;
        order[i] = i;
    }
    // larger fields first inside each pass
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const poisson_plan_s* a = b->plans[x];
        const poisson_plan_s* c = b->plans[y];
        return (long long)a->nx * a->ny * a->nz > (long long)c->nx * c->ny * c->nz;
    });
    std::vector<BatchSeg> segs;
    int total = 0;
    for (int pass = 0; pass < 5; ++pass)
        for (int i : order) {
            const int nt = b->h_fields[i].ntiles[pass];
            if (nt <= 0) continue;
            const BatchSeg s{i, pass, total, nt, seg_group(nt)};
            segs.push_back(s);
            total += (nt + s.group - 1) / s.group;  // work items of the segment
        }
    if ((e = cudaMalloc(&b->d_segs, segs.size() * sizeof(BatchSeg)))) return e;
    if ((e = cudaMemcpy(b->d_segs, segs.data(), segs.size() * sizeof(BatchSeg), cudaMemcpyHostToDevice)))
        return e;
    b->ctl_bytes = (size_t)(2 + 5 * n) * sizeof(unsigned);
    if ((e = cudaMalloc(&b->d_ctl, b->ctl_bytes))) return e;

    // launch shape: as many CTAs as fit on the GPU at once
    const size_t smem = batch_smem(b->plans);
    if ((e = cudaFuncSetAttribute(k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
        return e;
    int per_sm = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched, BATCH_THREADS, smem))) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device))) return e;
    const int grid = std::max(1, std::min(total, std::max(1, per_sm) * sms));

    BatchArgs args{};
    args.fields = b->d_fields;
    args.segs = b->d_segs;
    args.nseg = (int)segs.size();
    args.total = total;
    args.ctl = b->d_ctl;
    args.status = b->plans[0]->status;
    args.hold_field = b->hold_field;
    args.spin_limit = b->hold_field >= 0 ? 4096 : (1LL << 23);

    // graph: reset the control block, then the persistent kernel
    if ((e = cudaGraphCreate(&b->graph, 0))) return e;
    cudaGraphNode_t mset, kern;
    cudaMemsetParams mp{};
    mp.dst = b->d_ctl;
    mp.value = 0;
    mp.elementSize = sizeof(unsigned);
    mp.width = b->ctl_bytes / sizeof(unsigned);
    mp.height = 1;
    mp.pitch = b->ctl_bytes;
    if ((e = cudaGraphAddMemsetNode(&mset, b->graph, nullptr, 0, &mp))) return e;
    void* kargs[] = {&args};
    cudaKernelNodeParams kp{};
    kp.func = reinterpret_cast<void*>(k_batched);
    kp.gridDim = dim3(grid);
    kp.blockDim = dim3(BATCH_THREADS);
    kp.sharedMemBytes = (unsigned)smem;
    kp.kernelParams = kargs;
    if ((e = cudaGraphAddKernelNode(&kern, b->graph, &mset, 1, &kp))) return e;
    return cudaGraphInstantiate(&b->exec, b->graph, 0);
}

bool same_plans(const BatchState* b, poisson_plan_t const* plans, int count, int hold) {
    if ((int)b->plans.size() != count || b->hold_field != hold) return false;
    for (int i = 0; i < count; ++i)
        if (b->plans[i] != plans[i]) return false;
    return true;
}

// Queue every field's five kernels, spread over the side streams (forked
// from and joined back to `st`); usable eagerly or under stream capture.
cudaError_t enqueue_fields(BatchState* b, const void* const* rho, void* const* phi, cudaStream_t st,
                           bool defaults) {
    cudaError_t e;
    const int n = (int)b->plans.size();
    if (!b->fork) {
        if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming))) return e;
        for (int k = 0; k < BATCH_STREAMS; ++k) {
            if ((e = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking))) return e;
            if ((e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming))) return e;
        }
    }
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    auto cells = [&](int i) {
        const poisson_plan_s* p = b->plans[i];
        return (double)p->nx * p->ny * p->nz;
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cells(x) > cells(y); });
    double load[BATCH_STREAMS] = {0, 0, 0, 0};
    if ((e = cudaEventRecord(b->fork, st))) return e;
    for (int k = 0; k < BATCH_STREAMS; ++k)
        if ((e = cudaStreamWaitEvent(b->side[k], b->fork, 0))) return e;
    for (int i : order) {
        int k = 0;
        for (int j = 1; j < BATCH_STREAMS; ++j)
            if (load[j] < load[k]) k = j;
        load[k] += cells(i);
        for (int pass = 0; pass < 5; ++pass) {
            const int var = defaults ? plan_default_variant(b->plans[i], pass) : -1;
            if ((e = plan_run_pass(b->plans[i], pass, rho[i], phi[i], b->side[k], var))) return e;
        }
    }
    for (int k = 0; k < BATCH_STREAMS; ++k) {
        if ((e = cudaEventRecord(b->join[k], b->side[k]))) return e;
        if ((e = cudaStreamWaitEvent(st, b->join[k], 0))) return e;
    }
    return cudaSuccess;
}

// (Re)build the mode-1 graph for these buffers.
cudaError_t build_launch_graph(BatchState* b, const void* const* rho, void* const* phi, int mode) {
    cudaError_t e;
    const int k = mode - 1;
    if (b->lexec[k]) {
        cudaGraphExecDestroy(b->lexec[k]);
        b->lexec[k] = nullptr;
    }
    cudaStream_t cs;
    if ((e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking))) return e;
    // warm the kernels (attributes, module loading) outside the capture
    e = enqueue_fields(b, rho, phi, cs, mode == 2);
    if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
    cudaGraph_t g = nullptr;
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t e2 = enqueue_fields(b, rho, phi, cs, mode == 2);
        e = cudaStreamEndCapture(cs, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->lexec[k], g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    const int n = (int)b->plans.size();
    b->lrho[k].assign(rho, rho + n);
    b->lphi[k].assign(phi, phi + n);
    return e;
}

}  // namespace

poisson_status batch_mode(poisson_plan_t const* plans, int count, int set_to, int* get) {
    std::lock_guard<std::mutex> lock(g_mu);
    for (BatchState* c : g_cache) {
        if (!same_plans(c, plans, count, -1)) continue;
        if (get) *get = c->mode;
        if (set_to >= -1) c->mode = set_to;
        return POISSON_OK;
    }
    if (get) *get = -1;
    return set_to >= -1 ? POISSON_ERR_ARG : POISSON_OK;
}

void batch_forget_plan(poisson_plan_t plan) {
    std::lock_guard<std::mutex> lock(g_mu);
    for (size_t i = 0; i < g_cache.size();) {
        BatchState* b = g_cache[i];
        if (std::find(b->plans.begin(), b->plans.end(), plan) != b->plans.end()) {
            destroy_state(b);
            g_cache.erase(g_cache.begin() + i);
        } else {
            ++i;
        }
    }
}

poisson_status batched_solve(poisson_plan_t const* plans, int count, const void* const* rho,
                             void* const* phi, cudaStream_t st) {
    if (count == 0) return POISSON_OK;
    for (int i = 0; i < count; ++i)
        if (plans[i]->prec != POISSON_FP32 || plans[i]->device != plans[0]->device)
            return POISSON_ERR_UNSUPPORTED;
    // test hook: hold field 0's second pass on a count that never completes
    const char* hook = std::getenv("POISSON_TEST_BATCH_HOLD");
    const int hold = (hook && hook[0] == '1') ? 0 : -1;

    std::lock_guard<std::mutex> lock(g_mu);
    BatchState* b = nullptr;
    for (BatchState* c : g_cache)
        if (same_plans(c, plans, count, hold)) b = c;
    cudaError_t e;
    if (!b) {
        b = new BatchState();
        b->plans.assign(plans, plans + count);
        b->hold_field = hold;
        b->device = plans[0]->device;
        if ((e = build_state(b)) != cudaSuccess) {
            destroy_state(b);
            return e == cudaErrorMemoryAllocation ? POISSON_ERR_ALLOC : POISSON_ERR_CUDA;
        }
        g_cache.push_back(b);
    }
    // refresh the field table when the caller's buffers changed
    bool changed = !b->have_ptrs;
    for (int i = 0; i < count && !changed; ++i)
        changed = b->h_fields[i].p[0].in != rho[i] || b->h_fields[i].p[4].out != phi[i];
    if (changed) {
        if ((e = cudaEventSynchronize(b->copied))) return POISSON_ERR_CUDA;  // mirror free to edit
        for (int i = 0; i < count; ++i) {
            b->h_fields[i].p[0].in = rho[i];
            b->h_fields[i].p[4].out = phi[i];
        }
        if ((e = cudaMemcpyAsync(b->d_fields, b->h_fields, count * sizeof(BatchField),
                                 cudaMemcpyHostToDevice, st)))
            return POISSON_ERR_CUDA;
        if ((e = cudaEventRecord(b->copied, st))) return POISSON_ERR_CUDA;
        b->have_ptrs = true;
    }
    // modes 1 and 2 need a graph captured for exactly these buffers
    auto launch = [&](int m) -> cudaError_t {
        if (m == 0) return cudaGraphLaunch(b->exec, st);
        const int k = m - 1;
        bool same = b->lexec[k] != nullptr;
        for (int i = 0; i < count && same; ++i) same = b->lrho[k][i] == rho[i] && b->lphi[k][i] == phi[i];
        if (!same && (e = build_launch_graph(b, rho, phi, m))) return e;
        return cudaGraphLaunch(b->lexec[k], st);
    };
    if (b->mode < 0) {
        const char* forced = std::getenv("POISSON_BATCH_MODE");
        if (hold >= 0) {
            b->mode = 0;
        } else if (forced && forced[0] >= '0' && forced[0] <= '2') {
            b->mode = forced[0] - '0';
        } else {
            // time the three executions on the caller's data (twice each,
            // keep the second) and keep the fastest
            cudaEvent_t t0, t1;
            if ((e = cudaEventCreate(&t0)) || (e = cudaEventCreate(&t1))) return POISSON_ERR_CUDA;
            float ms[3] = {0.f, 0.f, 0.f};
            for (int m = 0; m < 3 && e == cudaSuccess; ++m)
                for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {
                    if ((e = cudaEventRecord(t0, st))) break;
                    if ((e = launch(m))) break;
                    if ((e = cudaEventRecord(t1, st))) break;
                    if ((e = cudaEventSynchronize(t1))) break;
                    e = cudaEventElapsedTime(&ms[m], t0, t1);
                }
            cudaEventDestroy(t0);
            cudaEventDestroy(t1);
            if (e != cudaSuccess) return POISSON_ERR_CUDA;
            int best = 0;
            for (int m = 1; m < 3; ++m)
                if (ms[m] < ms[best]) best = m;
            b->mode = best;
            return POISSON_OK;  // the timing runs already produced the result
        }
    }
    e = launch(b->mode);
    return e == cudaSuccess ? POISSON_OK : POISSON_ERR_CUDA;
}

}  // namespace pgb
