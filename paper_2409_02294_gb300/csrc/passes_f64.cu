// FP64 instantiations of the five passes.
#include "configs.cuh"
#include "internal.h"

namespace pgb {
cudaError_t launch_pass_f64(int N, int pass, int var, const PassParams<double>& p, int rows, cudaStream_t st) {
    switch (pass_group(pass)) {
        case GROUP_ROW: return launch_group<double, GROUP_ROW>(N, pass, var, p, rows, st);
        case GROUP_Y: return launch_group<double, GROUP_Y>(N, pass, var, p, rows, st);
        default: return launch_group<double, GROUP_Z>(N, pass, var, p, rows, st);
    }
}
}  // namespace pgb
