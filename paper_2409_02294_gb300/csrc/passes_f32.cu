// FP32 instantiations of the five passes.
#include "configs.cuh"
#include "internal.h"

namespace pgb {
cudaError_t launch_pass_f32(int N, int pass, const PassParams<float>& p, int rows, cudaStream_t st) {
    return launch_pass_t<float>(N, pass, p, rows, st);
}
}  // namespace pgb
