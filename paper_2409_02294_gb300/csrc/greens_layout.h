// Device layout of the transformed Green's function octant Ghat(kx, ky, kz),
// kx <= nx, ky <= ny, kz <= nz (real; the plan's data-path precision).
//
// A z-pass column tile needs, for one ky, the values of a band of
// consecutive kx (16 floats or 8 doubles: 64 bytes) at every kz.  With the
// octant stored row by row ([kz][ky][kx]) each of those reads is a 64-byte
// piece of a row, and DRAM delivers the whole 128-byte line around it (the
// other half belongs to the next band, whose tiles run much later): twice
// the octant's bytes.  So the octant is stored in blocks: block (ky, b) holds
// kx = b XW .. b XW + XW - 1 (XW = 64 bytes of values) for kz = 0..nz as
// [kz][XW], contiguous, and a tile reads its block front to back:
//   index(kx, ky, kz) = ((ky * bands + kx / XW) * (nz + 1) + kz) * XW + kx % XW,
//   bands = ceil((nx + 1) / XW).
// Columns beyond nx in the last band are zero and never read by the passes.
#pragma once

namespace pgb {

template <class R> __host__ __device__ constexpr int greens_xw() { return 64 / (int)sizeof(R); }
template <class R> __host__ __device__ constexpr long long greens_bands(int nx) {
    return ((long long)nx + greens_xw<R>()) / greens_xw<R>();  // ceil((nx + 1) / XW)
}
// offset of (kx, ky, kz = 0); kz advances by greens_xw<R>()
template <class R> __host__ __device__ constexpr long long greens_base(int kx, int ky, int nx, int nz) {
    return ((long long)ky * greens_bands<R>(nx) + kx / greens_xw<R>()) * (nz + 1) * greens_xw<R>() +
           kx % greens_xw<R>();
}
template <class R> __host__ __device__ constexpr long long greens_index(int kx, int ky, int kz, int nx, int nz) {
    return greens_base<R>(kx, ky, nx, nz) + (long long)kz * greens_xw<R>();
}
template <class R> __host__ __device__ constexpr long long greens_elems(int nx, int ny, int nz) {
    return greens_bands<R>(nx) * greens_xw<R>() * (ny + 1) * (nz + 1);
}

}  // namespace pgb
