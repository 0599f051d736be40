// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace pgb {

template <class R> struct PassParams;

// One pass (0..4) of the five-pass solve for transform length N, kernel
// variant `var` (0 <= var < pass_variants(precision, pass)).
cudaError_t launch_pass_f32(int N, int pass, int var, const PassParams<float>& p, int rows, cudaStream_t st);
cudaError_t launch_pass_f64(int N, int pass, int var, const PassParams<double>& p, int rows, cudaStream_t st);
int pass_variants(bool fp64, int pass);
// per-group entry points (one translation unit each)
cudaError_t launch_row_f32(int N, int pass, int var, const PassParams<float>& p, int rows, cudaStream_t st);
cudaError_t launch_y_f32(int N, int pass, int var, const PassParams<float>& p, cudaStream_t st);
cudaError_t launch_z_f32(int N, int pass, int var, const PassParams<float>& p, cudaStream_t st);

// Build the transformed Green's function octant on the device (FP64
// throughout), scaled by `scale`, written as float (out_f32) or double
// (out_f64; exactly one of the two is non-null).  With user_octant (host,
// (nz+1)(ny+1)(nx+1) FP64 values k[dz][dy][dx]) that kernel is transformed
// instead of the Green's kernel (h and r_near are then unused).
cudaError_t build_greens(int nx, int ny, int nz, double hx, double hy, double hz, int r_near,
                         double scale, float* out_f32, double* out_f64, cudaStream_t st,
                         const double* user_octant = nullptr);

// Raw Green's kernel k(d) octant (FP64, (nx+1)(ny+1)(nz+1)), for tests.
cudaError_t build_kernel_octant(int nx, int ny, int nz, double hx, double hy, double hz,
                                int r_near, double* out, cudaStream_t st);

// z pass with tensor-core radix-16 stages (split FP16 or BF16 operands)
bool z_tc_supported(int N);
cudaError_t launch_z_tc(int N, bool bf16, const PassParams<float>& p, cudaStream_t st);

// DCT-I transform + scaling of a k(d) octant on caller-provided buffers
// (no allocation, no synchronisation); see greens.cu.
cudaError_t greens_transform_into(double* kbuf, double* tmp, const double* cx, const double* cy,
                                  const double* cz, int nx, int ny, int nz, double scale,
                                  float* out, cudaStream_t st);

}  // namespace pgb
