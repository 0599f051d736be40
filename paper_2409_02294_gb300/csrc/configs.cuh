// Per-size line-transform configurations: elements per thread (E) and the
// Stockham radix sequence.  Every radix divides E; radices multiply to N.
#pragma once

#include <tuple>
#include <type_traits>

#include "passes_pk.cuh"

namespace pgb {

template <class R, int N> struct SizeCfg;

// FP32: E up to 32 complex values per thread (one line per thread).
template <> struct SizeCfg<float, 16>  { using C = LineCfg<float, 16, 16, Radices<16>>; };
template <> struct SizeCfg<float, 32>  { using C = LineCfg<float, 32, 8, Radices<8, 4>>; };
template <> struct SizeCfg<float, 48>  { using C = LineCfg<float, 48, 12, Radices<12, 4>>; };
template <> struct SizeCfg<float, 64>  { using C = LineCfg<float, 64, 8, Radices<8, 8>>; };
template <> struct SizeCfg<float, 96>  { using C = LineCfg<float, 96, 24, Radices<24, 4>>; };
template <> struct SizeCfg<float, 128> { using C = LineCfg<float, 128, 16, Radices<16, 8>>; };
template <> struct SizeCfg<float, 192> { using C = LineCfg<float, 192, 24, Radices<24, 8>>; };
template <> struct SizeCfg<float, 256> { using C = LineCfg<float, 256, 16, Radices<16, 16>>; };
template <> struct SizeCfg<float, 384> { using C = LineCfg<float, 384, 24, Radices<24, 8, 2>>; };
template <> struct SizeCfg<float, 512> { using C = LineCfg<float, 512, 32, Radices<32, 16>>; };

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
template <> struct SizeCfg<double, 512> { using C = LineCfg<double, 512, 16, Radices<16, 16, 2>>; };

inline bool size_supported(int n) {
    switch (n) {
        case 16: case 32: case 48: case 64: case 96: case 128:
        case 192: case 256: case 384: case 512: return true;
        default: return false;
    }
}

// The row passes (x axis) use RowSizeCfg: SizeCfg except where fewer values
// per thread suit the row tiles (FP32 512: radices 16-16-2, 32 threads per
// line; the column tiles keep 32-16, whose 16 threads per line give wider
// column tiles).
template <class R, int N> struct RowSizeCfg { using C = typename SizeCfg<R, N>::C; };
template <> struct RowSizeCfg<float, 512> { using C = LineCfg<float, 512, 16, Radices<16, 16, 2>>; };

// Twiddle-table layout of an axis of edge n: the row configuration's radix
// sequence for the x axis (row = true), the column configuration's for y and
// z (every kernel that transforms lines of an axis uses that configuration).
template <class R, int N> inline StageTwList axis_tw_list_n(bool row) {
    return row ? stage_tw_list<N>(typename RowSizeCfg<R, N>::C::Rads{})
               : stage_tw_list<N>(typename SizeCfg<R, N>::C::Rads{});
}
template <class R> inline StageTwList axis_tw_list(int n, bool row) {
    switch (n) {
        case 16: return axis_tw_list_n<R, 16>(row);
        case 32: return axis_tw_list_n<R, 32>(row);
        case 48: return axis_tw_list_n<R, 48>(row);
        case 64: return axis_tw_list_n<R, 64>(row);
        case 96: return axis_tw_list_n<R, 96>(row);
        case 128: return axis_tw_list_n<R, 128>(row);
        case 192: return axis_tw_list_n<R, 192>(row);
        case 256: return axis_tw_list_n<R, 256>(row);
        case 384: return axis_tw_list_n<R, 384>(row);
        case 512: return axis_tw_list_n<R, 512>(row);
        default: return StageTwList{};
    }
}

// Fill the stage tables described by L of a table whose first 2n entries
// (W_2n^j) are already on the device (async on st), FP32.
cudaError_t fill_stage_twiddles_list(cpx<float>* tw, int n, const StageTwList& L, cudaStream_t st);

// Fill the stage tables of an axis table whose first 2n entries (W_2n^j)
// are already on the device (async on st); row as for axis_tw_list.
template <class R> cudaError_t fill_stage_twiddles(cpx<R>* tw, int n, bool row, cudaStream_t st);

// Variants the autotuner chooses from (per pass and edge length).
//   column passes (y forward, z convolve, y inverse): lines per thread and
//   CTA threads; row passes (x forward, x inverse) likewise.
template <class R> struct Variants;
template <> struct Variants<float> {
    // (the persistent TMA variants stay last: their Nyquist-column tiles
    // need a second, plain launch; the last two double-buffer, the one
    // before them single-buffers its 16-column tiles)
    using Col = std::tuple<Var<2, 128>, Var<2, 256>, Var<1, 256>, Var<1, 512>, Var<2, 64>,
                           Var<2, 128, 3>, Var<2, 64, 5>, Var<2, 128, 1, 0, true>,
                           Var<2, 256, 1, 0, true>, Var<2, 128, 3, 0, true>,
                           Var<2, 256, 1, 1>, Var<2, 128, 3, 2>, Var<1, 256, 2, 2>>;
    using Row = std::tuple<Var<2, 256>, Var<1, 256>, Var<2, 128>, Var<1, 256, 3>, Var<2, 64>, Var<2, 128, 4>>;
};
template <> struct Variants<double> {
    using Col = std::tuple<Var<1, 256>>;
    using Row = std::tuple<Var<1, 256>>;
};
// Plain variants (one tile per CTA, two lines per thread, 256-thread CTAs,
// no register cap, no TMA): a fixed, shape-independent choice for callers
// that do not autotune and create no tensor maps.
constexpr int kRowVarPlain = 0;
constexpr int kColVarPlain = 1;
static_assert(std::is_same<std::tuple_element<kRowVarPlain, Variants<float>::Row>::type, Var<2, 256>>::value,
              "kRowVarPlain must name the plain 256-thread row variant");
static_assert(std::is_same<std::tuple_element<kColVarPlain, Variants<float>::Col>::type, Var<2, 256>>::value,
              "kColVarPlain must name the plain 256-thread column variant");

template <class R> constexpr int num_variants(int pass) {
    return (pass == 0 || pass == 4) ? (int)std::tuple_size<typename Variants<R>::Row>::value
                                    : (int)std::tuple_size<typename Variants<R>::Col>::value;
}

enum PassGroup { GROUP_ROW = 0, GROUP_Y = 1, GROUP_Z = 2 };
inline int pass_group(int pass) { return (pass == 0 || pass == 4) ? GROUP_ROW : (pass == 2 ? GROUP_Z : GROUP_Y); }

template <class C, class Tuple, int I = 0>
cudaError_t launch_row_var(int var, int pass, const PassParams<typename C::R>& p, int rows, cudaStream_t st) {
    if constexpr (I < (int)std::tuple_size<Tuple>::value) {
        if (var == I) return launch_row<C, typename std::tuple_element<I, Tuple>::type>(pass, p, rows, st);
        return launch_row_var<C, Tuple, I + 1>(var, pass, p, rows, st);
    } else {
        return cudaErrorInvalidValue;
    }
}
template <class C, class Tuple, int I = 0>
cudaError_t launch_col_var(int var, int pass, const PassParams<typename C::R>& p, cudaStream_t st) {
    if constexpr (I < (int)std::tuple_size<Tuple>::value) {
        using V = typename std::tuple_element<I, Tuple>::type;
        if (var == I) {
            if constexpr (V::PK) {
                if constexpr (std::is_same<typename C::R, float>::value)
                    return launch_col_pk<C, var_slots<C, V>(), V::MINB>(pass, p, st);
                else
                    return cudaErrorInvalidValue;
            } else {
                return launch_col<C, V>(pass, p, st);
            }
        }
        return launch_col_var<C, Tuple, I + 1>(var, pass, p, st);
    } else {
        return cudaErrorInvalidValue;
    }
}

// Tile width (SLOTS) of column variant `var` for transform length N (host).
template <class R, int N, class Tuple, int I = 0> int col_slots_var(int var) {
    if constexpr (I < (int)std::tuple_size<Tuple>::value) {
        if (var == I) return var_slots<typename SizeCfg<R, N>::C, typename std::tuple_element<I, Tuple>::type>();
        return col_slots_var<R, N, Tuple, I + 1>(var);
    } else {
        return 0;
    }
}
template <class R> int col_slots_for(int N, int var) {
    using T = typename Variants<R>::Col;
    switch (N) {
        case 16: return col_slots_var<R, 16, T>(var);
        case 32: return col_slots_var<R, 32, T>(var);
        case 48: return col_slots_var<R, 48, T>(var);
        case 64: return col_slots_var<R, 64, T>(var);
        case 96: return col_slots_var<R, 96, T>(var);
        case 128: return col_slots_var<R, 128, T>(var);
        case 192: return col_slots_var<R, 192, T>(var);
        case 256: return col_slots_var<R, 256, T>(var);
        case 384: return col_slots_var<R, 384, T>(var);
        case 512: return col_slots_var<R, 512, T>(var);
        default: return 0;
    }
}

// Dispatch one pass of group GROUP for edge length N (the pass's axis).
template <class R, int GROUP, int N>
cudaError_t launch_group_n(int pass, int var, const PassParams<R>& p, int rows, cudaStream_t st) {
    if constexpr (GROUP == GROUP_ROW) {
        using C = typename RowSizeCfg<R, N>::C;
        return launch_row_var<C, typename Variants<R>::Row>(var, pass, p, rows, st);
    } else {
        using C = typename SizeCfg<R, N>::C;
        return launch_col_var<C, typename Variants<R>::Col>(var, pass, p, st);
    }
}

template <class R, int GROUP>
cudaError_t launch_group(int N, int pass, int var, const PassParams<R>& p, int rows, cudaStream_t st) {
    switch (N) {
        case 16: return launch_group_n<R, GROUP, 16>(pass, var, p, rows, st);
        case 32: return launch_group_n<R, GROUP, 32>(pass, var, p, rows, st);
        case 48: return launch_group_n<R, GROUP, 48>(pass, var, p, rows, st);
        case 64: return launch_group_n<R, GROUP, 64>(pass, var, p, rows, st);
        case 96: return launch_group_n<R, GROUP, 96>(pass, var, p, rows, st);
        case 128: return launch_group_n<R, GROUP, 128>(pass, var, p, rows, st);
        case 192: return launch_group_n<R, GROUP, 192>(pass, var, p, rows, st);
        case 256: return launch_group_n<R, GROUP, 256>(pass, var, p, rows, st);
        case 384: return launch_group_n<R, GROUP, 384>(pass, var, p, rows, st);
        case 512: return launch_group_n<R, GROUP, 512>(pass, var, p, rows, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace pgb
