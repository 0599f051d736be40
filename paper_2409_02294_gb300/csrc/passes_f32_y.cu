// FP32 instantiations: y forward and y inverse passes.
#include "configs.cuh"
#include "internal.h"

namespace pgb {
cudaError_t launch_y_f32(int N, int pass, int var, const PassParams<float>& p, cudaStream_t st) {
    return launch_group<float, GROUP_Y>(N, pass, var, p, 0, st);
}
}  // namespace pgb
