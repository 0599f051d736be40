"""Compile-time constants of the line transforms, checked on the host (CPU).

The pre- and post-multiplies of the padded transforms take W_2E^m =
exp(-i pi m / E) from cos_sin_pi_frac in csrc/fft_core.cuh, a compile-time
Taylor-series evaluation after exact integer range reduction.  A small host
program compiled with nvcc prints its values; they are compared here with
numpy's cos/sin at long double precision, and their FP32 roundings with the
FP32 roundings of the reference.  The Green's octant's block layout
(csrc/greens_layout.h) is checked for being a one-to-one map of the octant
into the stored array, with every tile segment 64-byte aligned.
"""
import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2409_02294_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include "fft_core.cuh"
#include "greens_layout.h"
int main() {
    for (int q = 1; q <= 64; ++q)
        for (int p = -2 * q; p <= 2 * q; ++p) {
            const pgb::CosSin w = pgb::cos_sin_pi_frac(p, q);
            std::printf("T %d %d %.17g %.17g\n", p, q, w.c, w.s);
        }
    const int shapes[][3] = {{16, 16, 16}, {48, 32, 16}, {512, 64, 32}, {96, 384, 16}};
    for (auto& s : shapes) {
        const int nx = s[0], ny = s[1], nz = s[2];
        std::printf("G %d %d %d %lld %lld %lld\n", nx, ny, nz, pgb::greens_elems<float>(nx, ny, nz),
                    pgb::greens_elems<double>(nx, ny, nz), pgb::greens_bands<float>(nx));
        for (int kz = 0; kz <= nz; ++kz)
            for (int ky = 0; ky <= ny; ++ky)
                for (int kx = 0; kx <= nx; ++kx)
                    std::printf("I %lld %lld\n", pgb::greens_index<float>(kx, ky, kz, nx, nz),
                                pgb::greens_index<double>(kx, ky, kz, nx, nz));
    }
    return 0;
}
"""


@pytest.fixture(scope="module")
def host_output():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "consts.cu")
        exe = os.path.join(d, "consts")
        with open(src, "w") as f:
            f.write(PROGRAM)
        subprocess.run([nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-I" + CSRC, "-o", exe, src],
                       check=True, capture_output=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    return out.splitlines()


def test_compile_time_cos_sin_of_rational_multiples_of_pi(host_output):
    rows = [l.split() for l in host_output if l.startswith("T ")]
    assert len(rows) > 8000
    p = np.array([int(r[1]) for r in rows], dtype=np.longdouble)
    q = np.array([int(r[2]) for r in rows], dtype=np.longdouble)
    c = np.array([float(r[3]) for r in rows])
    s = np.array([float(r[4]) for r in rows])
    a = np.longdouble("3.14159265358979323846264338327950288") * p / q
    rc, rs = np.cos(a), np.sin(a)
    # within a few double ulps of the long double values
    assert np.max(np.abs(c - rc.astype(np.float64))) < 5e-16
    assert np.max(np.abs(s - rs.astype(np.float64))) < 5e-16
    # exact where the circle's symmetries make the value exact
    quarter = (2 * p) % q == 0
    assert np.all(np.isin(c[quarter], [-1.0, 0.0, 1.0])) and np.all(np.isin(s[quarter], [-1.0, 0.0, 1.0]))
    # the FP32 constants the kernels use round like the reference
    tiny = 1e-15
    for got, ref in ((c, rc), (s, rs)):
        big = np.abs(ref) > tiny
        assert np.array_equal(got[big].astype(np.float32), ref[big].astype(np.float64).astype(np.float32))


def test_greens_block_layout_is_one_to_one_and_aligned(host_output):
    lines = iter(host_output)
    seen = 0
    for line in lines:
        if not line.startswith("G "):
            continue
        nx, ny, nz, ef, ed, bands = map(int, line.split()[1:])
        n = (nx + 1) * (ny + 1) * (nz + 1)
        idx = np.array([list(map(int, next(lines).split()[1:])) for _ in range(n)])
        for col, elems, xw in ((0, ef, 16), (1, ed, 8)):
            i = idx[:, col]
            assert np.unique(i).size == n            # one-to-one
            assert i.min() >= 0 and i.max() < elems  # inside the stored array
        assert bands == (nx + 16) // 16
        kx = np.tile(np.arange(nx + 1), (nz + 1) * (ny + 1))
        # a tile's band of 16 (8) columns starts on a 64-byte boundary and is
        # contiguous; consecutive kz of one band are one 64-byte row apart
        first = kx % 16 == 0
        assert np.all((idx[first, 0] * 4) % 64 == 0)
        firstd = kx % 8 == 0
        assert np.all((idx[firstd, 1] * 8) % 64 == 0)
        seen += 1
    assert seen == 4
