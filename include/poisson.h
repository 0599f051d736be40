/*
 * libpoisson: free-space Poisson solve Phi = G * rho on one GB300 GPU by
 * zero-padded FFT convolution.
 *
 * The operation is the potential-field solve of the paper's case study
 * (arXiv 2409.02294, Section 3: "the convolution method for solving
 * potential fields on nested grids", one N^3 array per mesh level, FFTs as
 * the performance-critical part, Section 1).  The paper does not print the
 * discretisation; this library computes, for a cell-centred grid of
 * n = (nx, ny, nz) cells with spacing h = (hx, hy, hz),
 *
 *     Phi[i] = -G V sum_{j in [0,n)} k(i - j) rho[j],   V = hx hy hz,
 *
 * where k(d) is the mean of 1/|r| over the source cell for |d|_inf <= r_near
 * (closed form) and the point value 1/|d h| beyond.  It does so by padding
 * to M = 2n per axis, a forward 3-D FFT, a pointwise multiply by the
 * transformed Green's function, an inverse FFT and a crop.
 *
 * Conventions shared by every entry point:
 *  - Arrays are dense, x fastest: element (x, y, z) at (z*ny + y)*nx + x.
 *  - Device pointers are caller-owned CUDA device memory on the plan's
 *    device, 16-byte aligned, holding float (POISSON_FP32) or double
 *    (POISSON_FP64) values.  Host pointers are caller-owned host memory
 *    (pinned memory gives full copy bandwidth, pageable memory works).
 *  - cuda_stream is a cudaStream_t (NULL = legacy default stream).  Device
 *    calls are asynchronous on that stream; host-buffer calls return after
 *    the result is in the host buffer.
 *  - Errors are reported by return value only; argument errors are detected
 *    before any work is queued.  Nothing is thrown across this boundary.
 *  - Supported edge lengths per axis: 16, 32, 48, 64, 96, 128, 192, 256,
 *    384, 512 (2^a or 3 * 2^a); the padded transform length is 2n.
 */
#ifndef POISSON_H
#define POISSON_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct poisson_plan_s* poisson_plan_t;

typedef enum {
    POISSON_OK = 0,
    POISSON_ERR_ARG = 1,         /* bad argument (null, size, alignment, ...) */
    POISSON_ERR_ALLOC = 2,       /* device or host allocation failed */
    POISSON_ERR_CUDA = 3,        /* a CUDA runtime call or launch failed */
    POISSON_ERR_UNSUPPORTED = 4, /* valid but not implemented (size, precision) */
    POISSON_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    POISSON_ERR_NUMERIC = 6      /* non-finite output (POISSON_FLAG_CHECK_FINITE) */
} poisson_status;

typedef enum {
    POISSON_FP64 = 0,      /* FP64 data path */
    POISSON_FP32 = 1,      /* FP32 data path, FP64-built Green's function */
    POISSON_TC_FP16X2 = 2, /* FP32 data path with split FP16 tensor-core DFT stages */
    POISSON_TC_BF16X2 = 3  /* FP32 data path with split BF16 tensor-core DFT stages */
} poisson_precision;

/* plan flags */
#define POISSON_FLAG_CHECK_FINITE 0x1u /* solves set POISSON_ERR_NUMERIC on NaN/Inf output */
#define POISSON_FLAG_AUTOTUNE 0x2u     /* tune in plan creation (or reuse this process's result for the shape) */

/* Default Chebyshev radius (in cells) inside which k(d) is the cell average. */
#define POISSON_R_NEAR_DEFAULT 8

/*
 * Create a plan for an nx x ny x nz grid.
 * Passage: Section 3 (the convolution method for potential fields on nested
 * grids, one N^3 array per mesh level) fixes the operation; everything the
 * method computes once per mesh level -- the Green's function k(d), its
 * transform, the twiddle tables -- is built here, so that a solve is only
 * the FFT passes the paper names as the performance-critical part
 * (Section 1).  The plan's buffers are allocated once and then reused by
 * every solve, the device-memory analogue of the paper's link-once pointer
 * set-up (Section 2.2, host memory: the address is taken once at start-up
 * and both sides keep using the same array).
 *  out         receives the plan handle (caller destroys it with
 *              poisson_plan_destroy).
 *  hx, hy, hz  cell spacing (> 0).   G  gravitational constant (any finite).
 *  prec        data-path precision.  flags  POISSON_FLAG_* bits.
 *  cuda_stream stream for the one-time set-up work (the Green's function is
 *              generated and transformed in FP64 on the GPU); the call
 *              synchronises that stream before returning.
 * The plan owns its workspace, transformed Green's function (an octant of
 * (nx+1)(ny+1)(nz+1) values, by its real even symmetry) and twiddle tables,
 * all on the current CUDA device.
 * Errors: POISSON_ERR_ARG (null out, non-positive spacing, non-finite G),
 * POISSON_ERR_UNSUPPORTED (edge length or precision), POISSON_ERR_ALLOC,
 * POISSON_ERR_CUDA.  *out is NULL on error.
 */
poisson_status poisson_plan_create(poisson_plan_t* out, int nx, int ny, int nz,
                                   double hx, double hy, double hz, double G,
                                   poisson_precision prec, unsigned flags,
                                   void* cuda_stream);

/* As poisson_plan_create with an explicit near-field radius r_near >= 0. */
poisson_status poisson_plan_create_ex(poisson_plan_t* out, int nx, int ny, int nz,
                                      double hx, double hy, double hz, double G,
                                      poisson_precision prec, unsigned flags,
                                      int r_near, void* cuda_stream);

/*
 * Plan for a caller-supplied real kernel that is even along every axis (a
 * generalisation of the Green's function of Section 3: screened or softened
 * potentials, smoothing kernels):
 *     Phi[i] = scale * sum_j k(|i - j|) rho[j],  i, j in [0, n)^3,
 * where k_octant holds k on the octant, FP64, host memory, dense
 * [dz][dy][dx] with 0 <= d <= n per axis ((nz+1)(ny+1)(nx+1) values; the
 * entries at d = n only sit at the padded grid's wrapped index M/2 and never
 * reach a kept output, but keep the transform real).  The plan copies and
 * transforms it once (FP64 on the GPU); the caller's array can be freed on
 * return.  Everything else (precisions, solves, adjoint = the same solve
 * since the kernel is even, batching, autotuning) is as for
 * poisson_plan_create; the plan's info reports h = 1, G = 0.
 * Errors: POISSON_ERR_ARG (null pointers, non-finite values, bad sizes),
 * POISSON_ERR_UNSUPPORTED (edge length or precision), POISSON_ERR_ALLOC,
 * POISSON_ERR_CUDA.
 */
poisson_status poisson_plan_create_kernel(poisson_plan_t* out, int nx, int ny, int nz, const double* k_octant,
                                          double scale, poisson_precision prec, unsigned flags,
                                          void* cuda_stream);

/*
 * Phi = G * rho.  Passage: Section 3, the convolution method of the case
 * study (zero-padded FFT convolution: forward 3-D FFT of the padded density,
 * multiply by the transformed Green's function, inverse FFT, crop).  The
 * caller owns both buffers and passes their device addresses; the library
 * neither copies nor keeps them, in the spirit of the paper's pointer
 * linking (Section 2.2) and its C-bound interface between separately built
 * codes (Appendix A).
 * rho_dev: nx*ny*nz input values; phi_dev: nx*ny*nz outputs.
 * rho_dev and phi_dev may be the same buffer (rho is fully consumed before
 * phi is written).  Asynchronous on cuda_stream.  A plan holds one
 * workspace, so solves on one plan must not overlap in time (issue them on
 * one stream).  Errors: POISSON_ERR_ARG (null/unaligned pointer, null plan),
 * POISSON_ERR_CUDA (launch failure).
 */
poisson_status poisson_solve(poisson_plan_t plan, const void* rho_dev, void* phi_dev,
                             void* cuda_stream);

/*
 * Adjoint solve.  Passage: Section 3's convolution method read backwards --
 * the paper prints no adjoint; it is the transpose of the same linear map.
 * grad = K^T w, the gradient of L = sum(w * Phi) with
 * respect to rho (the correlation of w with the Green's function: the same
 * padded pipeline with the conjugated transform, which for this real, even
 * kernel equals the forward one).  Same layout, aliasing and error rules as
 * poisson_solve.
 */
poisson_status poisson_solve_adjoint(poisson_plan_t plan, const void* w_dev, void* grad_dev,
                                     void* cuda_stream);

/*
 * Solve `count` independent fields.  Passage: Section 3, where every mesh
 * level of the nested grid is one independent N^3 convolution solve (one
 * level per image, and one GPU per level in the fully parallel runs); here
 * the levels, or any list of fields, share one GPU.  plans[i] is applied to
 * rho_dev[i] -> phi_dev[i].  Plans may have different sizes but must share the device
 * and precision (FP32); each plan appears at most once (a plan owns one
 * workspace and the fields run at the same time: use one plan per field, or
 * poisson_solve_host_levels, which serialises repeats).  Three executions exist, each replayed from a CUDA
 * graph: (0) one persistent kernel over the tiles of all fields, with
 * bounded per-field dependency waits; (1) every field's own five kernels
 * with each plan's own (possibly autotuned) variants, captured into one
 * graph that spreads the fields over four streams; (2) the same with the
 * variants plans use untuned (a field's best variants alone on the GPU are
 * not always the best when fields share it).  The first call with a given
 * plan list builds all three, times them on the caller's data
 * (synchronising cuda_stream) and keeps the fastest; the environment
 * variable POISSON_BATCH_MODE=0, 1 or 2 forces one.  Later calls replay the
 * chosen graph (modes 1 and 2 re-capture when the buffers change).  The arrays of
 * pointers are host arrays.  Errors: POISSON_ERR_ARG (also for a repeated
 * plan), POISSON_ERR_UNSUPPORTED
 * (mixed precision or devices), POISSON_ERR_CUDA, POISSON_ERR_TIMEOUT
 * (reported by poisson_plan_sync_status on plans[0]).
 */
poisson_status poisson_solve_batched(poisson_plan_t const* plans, int count,
                                     const void* const* rho_dev, void* const* phi_dev,
                                     void* cuda_stream);

/*
 * Kernel launches one poisson_solve of this plan makes in its current
 * configuration (variants and execution mode), counted by capturing a solve
 * into a CUDA graph on a private stream (nothing is executed).  Memset and
 * event nodes are not counted.  Errors: POISSON_ERR_ARG, POISSON_ERR_CUDA.
 */
poisson_status poisson_plan_launch_count(poisson_plan_t plan, int* launches);

/*
 * Execution mode of the batch cached for this plan list (after a first
 * poisson_solve_batched call with it): 0 persistent kernel, 1 per-field
 * launches with each plan's variants, 2 per-field launches with the untuned
 * variants, -1 not decided yet.  set_mode = -1 makes the next call time both
 * again.  Errors: POISSON_ERR_ARG (bad arguments, or set_mode on a plan list
 * that has no cached batch yet).
 */
poisson_status poisson_batch_get_mode(poisson_plan_t const* plans, int count, int* mode);
poisson_status poisson_batch_set_mode(poisson_plan_t const* plans, int count, int mode);

/*
 * End-to-end solve through host buffers: copies rho_host (nx*ny*nz values)
 * to plan-owned device memory, solves, copies Phi back to phi_host, and
 * returns once phi_host holds the result.  The device staging buffers are
 * allocated on the first call.  Errors as poisson_solve plus
 * POISSON_ERR_ALLOC.
 */
poisson_status poisson_solve_host(poisson_plan_t plan, const void* rho_host, void* phi_host,
                                  void* cuda_stream);

/*
 * Solve count independent fields (e.g. the levels of a nested grid, Section
 * 3) from host buffers, overlapping the transfers with the solves: level
 * i's host-to-device copy runs on a copy stream while earlier levels solve
 * on cuda_stream, and its device-to-host copy on a second copy stream while
 * later levels solve (the paper stages every level through host memory and
 * measures those transfers, Section 4).  rho_host[i] / phi_host[i] hold
 * plans[i]'s grid, dense [z][y][x] in the plan's precision; page-locked host
 * memory is needed for the copies to overlap (pageable memory works but
 * serialises).  A plan may appear more than once (e.g. a stream of fields
 * of one size): its occurrences alternate between two device staging pairs,
 * so one level's copies overlap the neighbouring levels' solves.  Returns when every
 * phi_host[i] is written.  All plans on one device.  Errors: POISSON_ERR_ARG,
 * POISSON_ERR_UNSUPPORTED, POISSON_ERR_CUDA, POISSON_ERR_ALLOC.
 */
poisson_status poisson_solve_host_levels(poisson_plan_t const* plans, int count, const void* const* rho_host,
                                         void* const* phi_host, void* cuda_stream);

/*
 * Launch one pass of poisson_solve (pass 0..4: x forward, y forward, z
 * convolve, y inverse, x inverse).  Calling passes 0..4 in order on one
 * stream is exactly poisson_solve; used to time passes individually.
 * Errors: POISSON_ERR_ARG (bad pass id or pointers), POISSON_ERR_CUDA.
 */
poisson_status poisson_solve_pass(poisson_plan_t plan, int pass, const void* rho_dev,
                                  void* phi_dev, void* cuda_stream);

/*
 * The plain FP32 pipeline, kept as a yardstick for the fused passes.
 * Passage: Section 3's convolution method in its straightforward form, with
 * this library's own line transforms: the padded Mx x My x Mz grid (M = 2n
 * per axis) is materialised as complex FP32 values, transformed by full
 * length-M FFTs along x, y and z in three separate passes, multiplied by the
 * transformed Green's function in a pass of its own, transformed back along
 * z, y and x, and cropped to phi.  Nothing is pruned or fused.  Same
 * arguments, layout and result as poisson_solve; FP32 plans only.  The
 * first call allocates the plan's 8 Mx My Mz-byte padded buffer and its
 * twiddle tables (kept until poisson_plan_destroy); later calls allocate
 * nothing.  Asynchronous on cuda_stream.  Errors: POISSON_ERR_ARG (null or
 * unaligned pointer, null plan), POISSON_ERR_UNSUPPORTED (not an FP32 plan),
 * POISSON_ERR_ALLOC, POISSON_ERR_CUDA.
 */
poisson_status poisson_solve_unfused(poisson_plan_t plan, const void* rho_dev, void* phi_dev,
                                     void* cuda_stream);

/* Release every device resource of the plan (synchronises the device).
 * Passage: the end of the plan's lifetime of Section 2.2's link-once
 * set-up; after this call the handle must not be used again.
 * Errors: POISSON_ERR_ARG (null plan). */
poisson_status poisson_plan_destroy(poisson_plan_t plan);

typedef struct {
    int nx, ny, nz;          /* user grid */
    int mx, my, mz;          /* padded transform lengths (2n) */
    double hx, hy, hz, G;
    int precision;           /* poisson_precision */
    int r_near;
    unsigned flags;
    size_t workspace_bytes;  /* W1 + W2 complex work buffers */
    size_t greens_bytes;     /* device bytes of the transformed Green's function octant (kx padded to 64 bytes) */
    long long row_stride;    /* complex elements per work-buffer row */
    int variant[5];          /* kernel variant in use per pass */
    int variant_count[5];    /* variants available per pass */
    int fused;               /* execution mode: 0 five launches, 1-2 fused kernel, 3-4 banded */
} poisson_plan_info;

/* Fill *info.  Errors: POISSON_ERR_ARG. */
poisson_status poisson_plan_get_info(poisson_plan_t plan, poisson_plan_info* info);

/*
 * Autotuner: for each of the five passes, time every compiled kernel variant
 * (lines per thread, CTA shape, register cap, persistent TMA column kernels)
 * on the plan's own buffers (two warm-up and five timed launches each, CUDA
 * events on cuda_stream) and keep the fastest, then time the execution modes
 * (five launches; FP32: banded streams; cubic FP32: the fused persistent
 * kernel) and keep the fastest.  The result is also recorded for the plan's
 * shape, precision and device: a later plan created with
 * POISSON_FLAG_AUTOTUNE for the same shape in this process takes it without
 * timing again.  Synchronises cuda_stream; allocates two temporary
 * grid-sized buffers.  Errors: POISSON_ERR_ARG, POISSON_ERR_ALLOC,
 * POISSON_ERR_CUDA.
 */
poisson_status poisson_plan_autotune(poisson_plan_t plan, void* cuda_stream);

/* Select kernel variant `variant` for `pass` (0..4) explicitly (for tests
 * and experiments).  pass = 5 selects the execution mode: 0 = five kernel
 * launches per solve, 1 or 2 = one persistent kernel that overlaps the
 * passes through tile-level dependencies, compiled for 3 or 2 resident CTAs
 * per SM (cubic FP32 grids of edge 64, 128, 192, 256, 384 or 512), 3 or 4 =
 * "banded": the column passes of 4 or 8 bands of kx columns run as staggered
 * chains on plan-owned streams forked from and joined back to cuda_stream
 * (FP32 plans); unsupported combinations return POISSON_ERR_UNSUPPORTED.
 * The autotuner picks the fastest mode available.  Errors: POISSON_ERR_ARG (out of range),
 * POISSON_ERR_UNSUPPORTED, POISSON_ERR_CUDA. */
poisson_status poisson_plan_set_variant(poisson_plan_t plan, int pass, int variant);

/*
 * Copy the plan's transformed Green's function octant to host memory as
 * doubles: host_out[(kz*(ny+1) + ky)*(nx+1) + kx] = Ghat(kx, ky, kz), the
 * DFT over the padded M^3 grid of -G V k, including the 1/(Mx My Mz) factor
 * of the inverse transform.  count must be >= (nx+1)(ny+1)(nz+1).
 * Synchronous.  Errors: POISSON_ERR_ARG, POISSON_ERR_CUDA.
 */
poisson_status poisson_plan_copy_greens(poisson_plan_t plan, double* host_out, size_t count);

/*
 * Read and clear the plan's device status word (written by checked solves
 * and bounded waits).  Synchronises cuda_stream.  Returns POISSON_OK,
 * POISSON_ERR_NUMERIC or POISSON_ERR_TIMEOUT.
 */
poisson_status poisson_plan_sync_status(poisson_plan_t plan, void* cuda_stream);

/*
 * Allocation-free solve for small FP32 grids, without a plan.  (The paper has
 * no counterpart; this exists for callers of the library.)
 *
 * For callers that must not call cudaMalloc when they solve: code inside a
 * framework whose caching allocator owns device memory, code with a fixed
 * memory budget, or code that cannot take the device synchronisation that
 * allocating and freeing may cause.  Instead of plan-owned buffers, this call
 * uses one fixed 16 MiB device array built into the library (held on every
 * GPU that loads the library until the process exits); it allocates nothing
 * and calls no allocating routine.  The caller passes only the FP32 input
 * rho_dev and output phi_dev (nx*ny*nz values each, 16-byte aligned device
 * memory); spacing, G and the result are as for a FP32 plan with the default
 * near-field radius.  The Green's function is rebuilt on every call.
 *
 * Limits: the grid's Green's function, tables and work buffers must fit the
 * 16 MiB array: 64^3 fits, and so does nx = 128 with ny = nz = 64 (a long x
 * axis is the only anisotropic shape with a 128 edge that fits, because the
 * x axis' spectrum keeps only nx + 1 bins); ny = 128 or nz = 128 with the
 * other two at 64 does not, nor does 128^3; larger grids
 * return POISSON_ERR_ARG before any work is queued.  Unsupported edge lengths
 * return POISSON_ERR_UNSUPPORTED.
 * Set-up: the first call on each device looks up the array's device address;
 * make that first call before any stream capture starts.
 * Sharing: all calls on a device share the array and it keeps the last call's
 * contents (nothing in it needs to start at zero).  Calls whose GPU work
 * overlaps in time race on it: issue them on one stream or serialise them.
 * Asynchronous on cuda_stream.  Errors: POISSON_ERR_ARG, POISSON_ERR_UNSUPPORTED,
 * POISSON_ERR_CUDA.
 */
poisson_status poisson_solve_noalloc(int nx, int ny, int nz, double hx, double hy, double hz,
                                     double G, const void* rho_dev, void* phi_dev,
                                     void* cuda_stream);

/* Static text for a status code (never NULL). */
const char* poisson_status_string(poisson_status status);

/* 1 if an edge length is supported, else 0. */
int poisson_supported_size(int n);

#ifdef __cplusplus
}
#endif

#endif /* POISSON_H */
