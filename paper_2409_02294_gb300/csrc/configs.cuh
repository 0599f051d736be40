// Per-size line-transform configurations: elements per thread (E) and the
// Stockham radix sequence.  Every radix divides E; radices multiply to N.
#pragma once

#include "passes.cuh"

namespace pgb {

template <class R, int N> struct SizeCfg;

// FP32: E up to 24 complex values per line, two lines (even/odd halves) per
// thread.
template <> struct SizeCfg<float, 16>  { using C = LineCfg<float, 16, 16, Radices<16>>; };
template <> struct SizeCfg<float, 32>  { using C = LineCfg<float, 32, 8, Radices<8, 4>>; };
template <> struct SizeCfg<float, 48>  { using C = LineCfg<float, 48, 12, Radices<12, 4>>; };
template <> struct SizeCfg<float, 64>  { using C = LineCfg<float, 64, 8, Radices<8, 8>>; };
template <> struct SizeCfg<float, 96>  { using C = LineCfg<float, 96, 24, Radices<24, 4>>; };
template <> struct SizeCfg<float, 128> { using C = LineCfg<float, 128, 16, Radices<16, 8>>; };
template <> struct SizeCfg<float, 192> { using C = LineCfg<float, 192, 24, Radices<24, 8>>; };
template <> struct SizeCfg<float, 256> { using C = LineCfg<float, 256, 16, Radices<16, 16>>; };
template <> struct SizeCfg<float, 384> { using C = LineCfg<float, 384, 24, Radices<24, 8, 2>>; };
template <> struct SizeCfg<float, 512> { using C = LineCfg<float, 512, 16, Radices<16, 16, 2>>; };

// FP64: smaller E (twice the registers per value).
template <> struct SizeCfg<double, 16>  { using C = LineCfg<double, 16, 8, Radices<8, 2>>; };
template <> struct SizeCfg<double, 32>  { using C = LineCfg<double, 32, 8, Radices<8, 4>>; };
template <> struct SizeCfg<double, 48>  { using C = LineCfg<double, 48, 12, Radices<12, 4>>; };
template <> struct SizeCfg<double, 64>  { using C = LineCfg<double, 64, 8, Radices<8, 8>>; };
template <> struct SizeCfg<double, 96>  { using C = LineCfg<double, 96, 12, Radices<12, 4, 2>>; };
template <> struct SizeCfg<double, 128> { using C = LineCfg<double, 128, 8, Radices<8, 8, 2>>; };
template <> struct SizeCfg<double, 192> { using C = LineCfg<double, 192, 12, Radices<12, 4, 4>>; };
template <> struct SizeCfg<double, 256> { using C = LineCfg<double, 256, 8, Radices<8, 8, 4>>; };
template <> struct SizeCfg<double, 384> { using C = LineCfg<double, 384, 12, Radices<12, 4, 4, 2>>; };
template <> struct SizeCfg<double, 512> { using C = LineCfg<double, 512, 8, Radices<8, 8, 8>>; };

inline bool size_supported(int n) {
    switch (n) {
        case 16: case 32: case 48: case 64: case 96: case 128:
        case 192: case 256: case 384: case 512: return true;
        default: return false;
    }
}

// Dispatch one pass for edge length N (the pass's transform axis).
template <class R, int N>
cudaError_t launch_pass_n(int pass, const PassParams<R>& p, int rows, cudaStream_t st) {
    using C = typename SizeCfg<R, N>::C;
    if (pass == 0 || pass == 4) return launch_row<C>(pass, p, rows, st);
    return launch_col<C>(pass, p, st);
}

template <class R>
cudaError_t launch_pass_t(int N, int pass, const PassParams<R>& p, int rows, cudaStream_t st) {
    switch (N) {
        case 16: return launch_pass_n<R, 16>(pass, p, rows, st);
        case 32: return launch_pass_n<R, 32>(pass, p, rows, st);
        case 48: return launch_pass_n<R, 48>(pass, p, rows, st);
        case 64: return launch_pass_n<R, 64>(pass, p, rows, st);
        case 96: return launch_pass_n<R, 96>(pass, p, rows, st);
        case 128: return launch_pass_n<R, 128>(pass, p, rows, st);
        case 192: return launch_pass_n<R, 192>(pass, p, rows, st);
        case 256: return launch_pass_n<R, 256>(pass, p, rows, st);
        case 384: return launch_pass_n<R, 384>(pass, p, rows, st);
        case 512: return launch_pass_n<R, 512>(pass, p, rows, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pgb
