"""FP64 CPU oracle for the free-space Poisson solve (test infrastructure).

ONLY the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package.  The product library never does, and the two
share no code: the oracle's Green's function lives in ``oracle.c`` (plain C,
built with gcc), its convolutions are written out below in numpy.

The method (Section 3 of the paper: the convolution method for potential
fields, whose FFTs are the performance-critical part, Section 1) reaches the
plain free-space discrete convolution

    Phi[i] = -G V sum_j k(i - j) rho[j],   i, j in [0, n)^3,  V = hx hy hz,

exactly up to rounding, so the oracle is that definition, evaluated three
independent ways:

1. ``solve_direct``  - the pair sum itself (O(n^6)), tiny grids;
   ``sample_direct`` - the same sum at chosen target cells, any size;
   ``solve_direct_kernel`` - the pair sum with a caller's even kernel.
2. ``solve_dft``     - zero-pad to M = 2n per axis, apply a dense FP64 DFT
   matrix along each axis (a matmul), multiply by the transformed kernel,
   apply the inverse DFT matrix, crop.  DFT matrix entries are indexed by
   (j*k mod M) from one table of M roots of unity.
3. ``solve_fft``     - the same padded convolution with a library FP64 FFT
   (scipy.fft), for full fields at the large sizes; ``solve_fft_kernel``
   with a caller's even kernel; ``kernel_rfft`` + ``solve_fft_with`` split
   ``solve_fft`` into its grid-only part and its per-density part.

The kernel k(d) and the readings of the paper it rests on are described in
``oracle.c``.  Pins of every function here against values fixed by the
mathematics live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

R_NEAR_DEFAULT = 8


def build(force=False):
    """Compile oracle.c with gcc (-O2, OpenMP, IEEE arithmetic)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-fno-fast-math", "-ffp-contract=off", "-o", tmp, src, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _SO)
    return _SO


def build_planted(which, outdir):
    """Compile a deliberately wrong variant (ORACLE_PLANT=which) into
    `outdir`; used only by the tests that show the pins catch mistakes."""
    src = os.path.join(_HERE, "oracle.c")
    so = os.path.join(outdir, "liboracle_plant%d.so" % int(which))
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-fno-fast-math", "-ffp-contract=off",
                           "-DORACLE_PLANT=%d" % int(which), "-o", so, src, "-lm"])
    return so


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _load(_SO)
    return _lib


def _load(path):
    L = ctypes.CDLL(path)
    d = ctypes.c_double
    i = ctypes.c_int
    l = ctypes.c_long
    P = ctypes.c_void_p
    L.oracle_box_integral.restype = d
    L.oracle_box_integral.argtypes = [d, d, d, d, d, d]
    L.oracle_kernel.restype = d
    L.oracle_kernel.argtypes = [l, l, l, d, d, d, i]
    L.oracle_kernel_octant.restype = None
    L.oracle_kernel_octant.argtypes = [i, i, i, d, d, d, i, P]
    L.oracle_direct_sum.restype = None
    L.oracle_direct_sum.argtypes = [i, i, i, P, P, d, P]
    L.oracle_direct_sum_points.restype = None
    L.oracle_direct_sum_points.argtypes = [i, i, i, P, P, d, l, P, P]
    L.oracle_set_threads.restype = None
    L.oracle_set_threads.argtypes = [i]
    L.oracle_get_threads.restype = i
    L.oracle_get_threads.argtypes = []
    return L


def use_library(path):
    """Point the oracle at another build of oracle.c (planted-mistake
    tests); `None` restores the normal build."""
    global _lib
    with _lock:
        _lib = None if path is None else _load(path)


def set_threads(n):
    lib().oracle_set_threads(int(n))


def get_threads():
    return int(lib().oracle_get_threads())


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _h3(h):
    if np.isscalar(h):
        return (float(h),) * 3
    return tuple(float(v) for v in h)  # (hx, hy, hz)


# ----------------------------------------------------------------------------
# Green's function
# ----------------------------------------------------------------------------

def box_integral(x0, x1, y0, y1, z0, z1):
    """Closed-form integral of 1/|r| over an axis-aligned box."""
    return lib().oracle_box_integral(x0, x1, y0, y1, z0, z1)


def kernel(d, h=1.0, r_near=R_NEAR_DEFAULT):
    """k(d) for one integer offset d = (dx, dy, dz); units 1/length."""
    hx, hy, hz = _h3(h)
    return lib().oracle_kernel(int(d[0]), int(d[1]), int(d[2]), hx, hy, hz, int(r_near))


def kernel_octant(extent_xyz, h=1.0, r_near=R_NEAR_DEFAULT):
    """Array K[dz, dy, dx] = k(dx, dy, dz) for 0 <= d < extent (x, y, z)."""
    kx, ky, kz = (int(v) for v in extent_xyz)
    hx, hy, hz = _h3(h)
    out = np.empty((kz, ky, kx), dtype=np.float64)
    lib().oracle_kernel_octant(kx, ky, kz, hx, hy, hz, int(r_near), _ptr(out))
    return out


def wrapped_kernel(n_zyx, M_zyx=None, h=1.0, r_near=R_NEAR_DEFAULT):
    """k on the padded periodic grid: entry m (per axis) holds k(d) with
    d = m for m <= M/2 and d = m - M otherwise (k is even, so |d| is used).
    Default padding M = 2n per axis."""
    nz, ny, nx = n_zyx
    Mz, My, Mx = M_zyx if M_zyx is not None else (2 * nz, 2 * ny, 2 * nx)
    oct_ = kernel_octant((Mx // 2 + 1, My // 2 + 1, Mz // 2 + 1), h, r_near)

    def fold(M):
        m = np.arange(M)
        return np.minimum(m, M - m)

    return oct_[np.ix_(fold(Mz), fold(My), fold(Mx))]


def greens_hat(n_zyx, h=1.0, G=1.0, r_near=R_NEAR_DEFAULT, M_zyx=None):
    """FFT of -G V k on the padded grid (FP64, complex, full M^3)."""
    hx, hy, hz = _h3(h)
    kw = wrapped_kernel(n_zyx, M_zyx, h, r_near)
    return np.fft.fftn(-G * hx * hy * hz * kw)


# ----------------------------------------------------------------------------
# Route 1: direct pair sums
# ----------------------------------------------------------------------------

def solve_direct(rho, h=1.0, G=1.0, r_near=R_NEAR_DEFAULT):
    """Phi[i] = -G V sum_j k(i-j) rho[j], every target, O(n^6)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    hx, hy, hz = _h3(h)
    koct = kernel_octant((nx, ny, nz), h, r_near)
    phi = np.empty_like(rho)
    lib().oracle_direct_sum(nx, ny, nz, _ptr(rho), _ptr(koct), -G * hx * hy * hz, _ptr(phi))
    return phi


def solve_direct_kernel(rho, k_octant, scale):
    """Phi[i] = scale sum_j k(|i - j|) rho[j] for a caller's per-axis even
    kernel given on the octant k_octant[dz, dy, dx], 0 <= d < n per axis
    (entries beyond are not used), O(n^6)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    koct = np.ascontiguousarray(np.asarray(k_octant, dtype=np.float64)[:nz, :ny, :nx])
    phi = np.empty_like(rho)
    lib().oracle_direct_sum(nx, ny, nz, _ptr(rho), _ptr(koct), float(scale), _ptr(phi))
    return phi


def solve_fft_kernel(rho, k_octant, scale, workers=-1):
    """The padded (M = 2n) FFT convolution with a caller's octant kernel,
    k_octant[dz, dy, dx] for 0 <= d <= n (entry n fills the wrapped index
    M/2, which reaches no kept output)."""
    import scipy.fft as sfft
    rho = np.asarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    M = (2 * nz, 2 * ny, 2 * nx)
    koct = np.asarray(k_octant, dtype=np.float64)

    def fold(m):
        a = np.arange(m)
        return np.minimum(a, m - a)

    kw = koct[np.ix_(fold(M[0]), fold(M[1]), fold(M[2]))] * float(scale)
    X = sfft.rfftn(rho, s=M, workers=workers)
    X *= sfft.rfftn(kw, workers=workers)
    phi = sfft.irfftn(X, s=M, workers=workers)
    return np.ascontiguousarray(phi[:nz, :ny, :nx])


def sample_direct(rho, targets, h=1.0, G=1.0, r_near=R_NEAR_DEFAULT, koct=None):
    """Direct sums at target cells (flat indices into rho, x fastest)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    hx, hy, hz = _h3(h)
    if koct is None:
        koct = kernel_octant((nx, ny, nz), h, r_near)
    t = np.ascontiguousarray(targets, dtype=np.int64)
    out = np.empty(len(t), dtype=np.float64)
    lib().oracle_direct_sum_points(nx, ny, nz, _ptr(rho), _ptr(koct), -G * hx * hy * hz,
                                   len(t), _ptr(t), _ptr(out))
    return out


# ----------------------------------------------------------------------------
# Route 2: dense DFT matrices
# ----------------------------------------------------------------------------

def dft_matrix(M, inverse=False):
    """F[k, m] = exp(-+2 pi i (k m mod M) / M), entries from one FP64 table."""
    idx = np.arange(M)
    table = np.exp((2j if inverse else -2j) * np.pi * np.arange(M) / M)
    return table[np.outer(idx, idx) % M]


def _apply_axis(F, a, axis):
    """Apply the matrix F along `axis` of a (out[..k..] = sum_m F[k,m] a[..m..])."""
    a = np.moveaxis(a, axis, -1)
    out = a @ F.T
    return np.moveaxis(out, -1, axis)


def solve_dft(rho, h=1.0, G=1.0, r_near=R_NEAR_DEFAULT, M_zyx=None):
    """Zero-pad, DFT along each axis by matrix product, multiply by the
    transformed kernel, inverse DFT by matrix product, crop."""
    rho = np.asarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    Mz, My, Mx = M_zyx if M_zyx is not None else (2 * nz, 2 * ny, 2 * nx)
    hx, hy, hz = _h3(h)
    pad = np.zeros((Mz, My, Mx), dtype=np.complex128)
    pad[:nz, :ny, :nx] = rho
    kw = -G * hx * hy * hz * wrapped_kernel((nz, ny, nx), (Mz, My, Mx), h, r_near)
    fwd = [dft_matrix(Mz), dft_matrix(My), dft_matrix(Mx)]
    inv = [dft_matrix(Mz, True), dft_matrix(My, True), dft_matrix(Mx, True)]
    X = pad
    K = kw.astype(np.complex128)
    for ax in range(3):
        X = _apply_axis(fwd[ax], X, ax)
        K = _apply_axis(fwd[ax], K, ax)
    Y = X * K
    for ax in range(3):
        Y = _apply_axis(inv[ax], Y, ax)
    Y /= float(Mz) * My * Mx
    return Y[:nz, :ny, :nx].real.copy()


# ----------------------------------------------------------------------------
# Route 3: library FFT
# ----------------------------------------------------------------------------

def kernel_rfft(n_zyx, h=1.0, G=1.0, r_near=R_NEAR_DEFAULT, M_zyx=None, workers=-1):
    """The real FFT (scipy.fft.rfftn, FP64) of -G V k on the padded grid:
    the part of ``solve_fft`` that depends only on the grid, computed once
    when many densities of one grid are solved."""
    import scipy.fft as sfft
    nz, ny, nx = n_zyx
    M = M_zyx if M_zyx is not None else (2 * nz, 2 * ny, 2 * nx)
    hx, hy, hz = _h3(h)
    kw = wrapped_kernel((nz, ny, nx), M, h, r_near)
    kw *= -G * hx * hy * hz
    return sfft.rfftn(kw, workers=workers)


def solve_fft_with(rho, Kh, M_zyx=None, workers=-1):
    """The padded convolution of rho with the transformed kernel Kh of
    ``kernel_rfft`` (same grid, same padding): forward real FFT of the
    zero-padded density, multiply, inverse real FFT, crop."""
    import scipy.fft as sfft
    rho = np.asarray(rho, dtype=np.float64)
    nz, ny, nx = rho.shape
    M = M_zyx if M_zyx is not None else (2 * nz, 2 * ny, 2 * nx)
    X = sfft.rfftn(rho, s=M, workers=workers)
    X *= Kh
    phi = sfft.irfftn(X, s=M, workers=workers)
    return np.ascontiguousarray(phi[:nz, :ny, :nx])


def solve_fft(rho, h=1.0, G=1.0, r_near=R_NEAR_DEFAULT, M_zyx=None, workers=-1):
    """The padded convolution with scipy's FP64 real FFTs."""
    rho = np.asarray(rho, dtype=np.float64)
    Kh = kernel_rfft(rho.shape, h, G, r_near, M_zyx, workers)
    return solve_fft_with(rho, Kh, M_zyx, workers)


def solve_adjoint_direct(w, h=1.0, G=1.0, r_near=R_NEAR_DEFAULT):
    """Gradient of L = sum(w * Phi) with respect to rho, by the direct
    correlation g[j] = -G V sum_i k(i - j) w[i] (k(-d) used as written)."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    # k(i-j) = k(j-i) under the even reading, so the correlation sum is the
    # same pair sum with source and target swapped.
    return solve_direct(w, h, G, r_near)
