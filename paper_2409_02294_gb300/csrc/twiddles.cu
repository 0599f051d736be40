// Stage twiddle tables: gathered on the device from an axis' W_2n^j table
// into the per-stage layout the line transforms read (see stage_tw_size).
#include "configs.cuh"

namespace pgb {

template <class R> __global__ void k_stage_twiddles(cpx<R>* __restrict__ tw, int n, StageTwList L) {
    const int stride = gridDim.x * blockDim.x;
    for (int s = 0; s < L.count; ++s) {
        const int ns = L.ns[s], rad = L.rad[s];
        const int size = rad == 2 ? ns : ns * rad;
        const long long c = 2LL * n / ((long long)ns * rad);  // W_{ns rad} = W_2n^c
        for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < size; e += stride) {
            int r, k;
            if (rad == 2) {
                r = 1;
                k = e;
            } else {
                const int q = e >> 1;
                r = 2 * (q / ns) + 1 + (e & 1);
                k = q % ns;
            }
            tw[L.off[s] + e] = tw[((long long)r * k * c) % (2LL * n)];
        }
    }
}

template <class R> cudaError_t fill_stage_twiddles(cpx<R>* tw, int n, bool row, cudaStream_t st) {
    const StageTwList L = axis_tw_list<R>(n, row);
    if (L.total == 0) return cudaErrorInvalidValue;
    if (L.count == 0) return cudaSuccess;
    k_stage_twiddles<R><<<8, 256, 0, st>>>(tw, n, L);
    return cudaGetLastError();
}

cudaError_t fill_stage_twiddles_list(cpx<float>* tw, int n, const StageTwList& L, cudaStream_t st) {
    if (L.count == 0) return cudaSuccess;
    k_stage_twiddles<float><<<8, 256, 0, st>>>(tw, n, L);
    return cudaGetLastError();
}

template cudaError_t fill_stage_twiddles<float>(cpx<float>*, int, bool, cudaStream_t);
template cudaError_t fill_stage_twiddles<double>(cpx<double>*, int, bool, cudaStream_t);

}  // namespace pgb
