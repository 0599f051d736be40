// FP32 instantiations: z convolution pass, plus the FP32 pass dispatcher.
#include "configs.cuh"
#include "internal.h"

namespace pgb {
cudaError_t launch_z_f32(int N, int pass, int var, const PassParams<float>& p, cudaStream_t st) {
    return launch_group<float, GROUP_Z>(N, pass, var, p, 0, st);
}

cudaError_t launch_pass_f32(int N, int pass, int var, const PassParams<float>& p, int rows, cudaStream_t st) {
    switch (pass_group(pass)) {
        case GROUP_ROW: return launch_row_f32(N, pass, var, p, rows, st);
        case GROUP_Y: return launch_y_f32(N, pass, var, p, st);
        default: return launch_z_f32(N, pass, var, p, st);
    }
}

int pass_variants(bool fp64, int pass) {
    return fp64 ? num_variants<double>(pass) : num_variants<float>(pass);
}
}  // namespace pgb
