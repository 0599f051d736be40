// FP32 instantiations: x forward and x inverse passes.
#include "configs.cuh"
#include "internal.h"

namespace pgb {
cudaError_t launch_row_f32(int N, int pass, int var, const PassParams<float>& p, int rows, cudaStream_t st) {
    return launch_group<float, GROUP_ROW>(N, pass, var, p, rows, st);
}
}  // namespace pgb
