"""Write the golden fixture direct_sum_blobs_48x16x32.txt with the FP64
oracle only (its direct pair sum, the plain definition of the free-space
discrete convolution of Section 3, under the readings stated in oracle.c).

    python tests/golden/make_golden.py

Input: 6 seeded Gaussian blobs (workloads.gaussian_blobs, seed 2409) on a
(nz, ny, nx) = (48, 16, 32) grid with spacing (hx, hy, hz) = (1.0, 0.75,
1.25) and G = 1.  Output: Phi at 96 seeded target cells, 17 significant
digits.  The fixture is test infrastructure: the CPU tests check that the
oracle still reproduces it, the GPU tests check the FP64 device solve
against it.
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import workloads  # noqa: E402

SHAPE = (48, 16, 32)
H = (1.0, 0.75, 1.25)
SEED = 2409
NTARGETS = 96
OUT = os.path.join(HERE, "direct_sum_blobs_48x16x32.txt")


def density():
    rho, _ = workloads.gaussian_blobs(SHAPE, count=6, seed=SEED)
    return rho


def targets():
    rng = np.random.default_rng(SEED + 1)
    return np.sort(rng.choice(int(np.prod(SHAPE)), size=NTARGETS, replace=False)).astype(np.int64)


def main():
    rho = density()
    t = targets()
    phi = oracle.sample_direct(rho, t, h=H, G=1.0)
    nz, ny, nx = SHAPE
    with open(OUT, "w") as f:
        f.write("# Phi = -G V sum_j k(i - j) rho[j] (direct pair sum, FP64 oracle), Section 3 convolution\n")
        f.write("# grid (nz, ny, nx) = %s, h = (hx, hy, hz) = %s, G = 1, r_near = %d\n"
                % (SHAPE, H, oracle.R_NEAR_DEFAULT))
        f.write("# density: workloads.gaussian_blobs(%s, count=6, seed=%d); written by make_golden.py\n"
                % (SHAPE, SEED))
        f.write("# columns: flat index (z*ny + y)*nx + x, z, y, x, Phi\n")
        for idx, v in zip(t, phi):
            z, rem = divmod(int(idx), ny * nx)
            y, x = divmod(rem, nx)
            f.write("%d %d %d %d %.17g\n" % (idx, z, y, x, v))


if __name__ == "__main__":
    main()
