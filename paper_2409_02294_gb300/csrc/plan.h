// The plan object behind poisson_plan_t (shared by the library's units).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "poisson.h"

struct poisson_plan_s {
    int nx, ny, nz;
    double hx, hy, hz, G;
    poisson_precision prec;
    unsigned flags;
    int r_near;
    int device;
    long long sx;         // complex row stride of W1/W2
    size_t csize;         // bytes per complex element
    size_t rsize;         // bytes per real element
    void* w1;             // nz * ny * sx complex
    void* w2;             // nz * 2ny * sx complex
    void* greens;         // (nx+1)(ny+1)(nz+1) real
    void* tw[3];          // W_{2n}^j tables for x, y, z
    unsigned* status;     // device status word
    void* stage_in;       // device staging for poisson_solve_host
    void* stage_out;
    void* stage_in2;      // second staging pair: repeated levels of one plan alternate
    void* stage_out2;
    int var[5];           // kernel variant per pass (autotuned or default)
    int use_fused;        // 1: one persistent dataflow kernel instead of five launches
    void* fused_order;    // its work queue ((pass, tile) pairs) and counters
    void* fused_ctl;
    int fused_total;
    int fused_ctl_words;
    cudaStream_t band_stream[8];  // banded execution: one stream per kx band
    cudaEvent_t band_ev_x, band_ev_y[8], band_ev_done[8];
    bool band_ready;
    void* unf_buf;        // poisson_solve_unfused: the padded complex grid (made on first use)
    void* unf_tw[3];      // its per-axis W_2M tables
};

namespace pgb {
// Drop every cached batched-solve graph that refers to `plan` (called when
// the plan is destroyed).
void batch_forget_plan(poisson_plan_t plan);
// One pass (0..4) of the five-launch solve with the plan's kernel variants.
// One pass of a plan's solve, with the plan's variant (var < 0) or var.
cudaError_t plan_run_pass(const poisson_plan_s* pl, int pass, const void* rho, void* phi, cudaStream_t st,
                          int var = -1);
// The variant a plan uses for a pass when it is not autotuned.
int plan_default_variant(const poisson_plan_s* pl, int pass);
// Single-field fused dataflow solve (fused.cu).
template <class R> struct PassParams;
bool fused_supported(const poisson_plan_s* pl);
cudaError_t fused_prepare(poisson_plan_s* pl, cudaStream_t st);
cudaError_t fused_solve(const poisson_plan_s* pl, const PassParams<float> (&p)[5], cudaStream_t st);
// Get (get != NULL) and/or set (set_to >= -1) the execution mode of the
// cached batch for this plan list; set_to = -2 leaves it unchanged.
poisson_status batch_mode(poisson_plan_t const* plans, int count, int set_to, int* get);
// The batched solve (poisson_solve_batched after argument checks).
poisson_status batched_solve(poisson_plan_t const* plans, int count, const void* const* rho,
                             void* const* phi, cudaStream_t st);
}  // namespace pgb
