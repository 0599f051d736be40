// FP64 instantiations of the five passes.
#include "configs.cuh"
#include "internal.h"

namespace pgb {
cudaError_t launch_pass_f64(int N, int pass, const PassParams<double>& p, int rows, cudaStream_t st) {
    return launch_pass_t<double>(N, pass, p, rows, st);
}
}  // namespace pgb
