// Plan-time DCT-I of a Green's kernel octant by FP64 line FFTs
// (greens_dct.cu), shared by the plan's Green's function builder.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "fft_core.cuh"

namespace pgb {

// FP64 complex entries of one axis' twiddle table for an edge of n.
size_t dct1_twiddle_entries(int n);

// DCT-I of a k(d) octant along x, y and z: k holds the octant
// ((nx+1)(ny+1)(nz+1) doubles, x fastest) and is used as scratch, the result
// is left in tmp (same size); tw[a] has room for dct1_twiddle_entries(n_a)
// entries.  Queued on st.
cudaError_t dct1_octant(double* k, double* tmp, cpx<double>* const tw[3], int nx, int ny, int nz, cudaStream_t st);

}  // namespace pgb
