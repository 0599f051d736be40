/*
 * FP64 CPU oracle for the free-space Poisson solve Phi = G * rho.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code with the CUDA path.
 *
 * What it computes (the plain definition of the discrete free-space
 * convolution that the paper's case-study solver evaluates with FFTs,
 * Section 3, "convolution method for solving potential fields"):
 *
 *     Phi[i] = -G * V * sum_{j in [0,n)^3} k(i - j) * rho[j]
 *
 * with V = hx*hy*hz and k(d) the Green's function of -1/|r| sampled on the
 * cell-centred grid.  The paper does not state its discretisation; the
 * reading used here (and by the GPU path, written separately) is:
 *
 *   |d|_inf <= r_near : k(d) = mean over the source cell (a box of size h
 *                       centred at d*h) of 1/|r|, by the closed-form
 *                       antiderivative of 1/r over a rectangular box;
 *   otherwise         : k(d) = 1/|d*h| (the cell-centre point value).
 *
 * Loops are plain and unblocked; OpenMP only splits the outer target loop.
 */
#include <math.h>
#include <stdlib.h>
/* ORACLE_PLANT (default 0) selects a deliberately wrong variant of one step;
 * the tests compile such variants on the CPU to show that the pins catch
 * each kind of mistake.  The normal build never defines it. */
#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif
#include <stdint.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* log(x + r) with r = sqrt(x^2+y^2+z^2), written without cancellation for
 * x < 0 (x + r = (y^2+z^2)/(r - x)). */
static double log_x_plus_r(double x, double y, double z, double r)
{
    if (x >= 0.0)
        return log(x + r);
    return log((y * y + z * z) / (r - x));
}

/* F(x,y,z) with d^3 F / (dx dy dz) = 1/r:
 *   F = y z ln(x+r) + z x ln(y+r) + x y ln(z+r)
 *       - x^2/2 atan(y z/(x r)) - y^2/2 atan(z x/(y r)) - z^2/2 atan(x y/(z r)).
 * Terms whose prefactor vanishes are dropped (their limit is 0). */
static double prism_antiderivative(double x, double y, double z)
{
    double r = sqrt(x * x + y * y + z * z);
    double f = 0.0;
    if (y != 0.0 && z != 0.0) f += y * z * log_x_plus_r(x, y, z, r);
    if (z != 0.0 && x != 0.0) f += z * x * log_x_plus_r(y, z, x, r);
    if (x != 0.0 && y != 0.0) f += x * y * log_x_plus_r(z, x, y, r);
#if ORACLE_PLANT == 1
    if (x != 0.0) f += 0.5 * x * x * atan((y * z) / (x * r)); /* planted: sign */
#else
    if (x != 0.0) f -= 0.5 * x * x * atan((y * z) / (x * r));
#endif
    if (y != 0.0) f -= 0.5 * y * y * atan((z * x) / (y * r));
    if (z != 0.0) f -= 0.5 * z * z * atan((x * y) / (z * r));
    return f;
}

/* Integral of 1/|r| over the box [x0,x1] x [y0,y1] x [z0,z1]: the sum of F
 * over the eight corners, each with the sign (+ for an upper, - for a lower
 * limit) multiplied over the three axes. */
double oracle_box_integral(double x0, double x1, double y0, double y1,
                           double z0, double z1)
{
    const double xs[2] = {x0, x1}, ys[2] = {y0, y1}, zs[2] = {z0, z1};
    double s = 0.0;
    for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b)
            for (int c = 0; c < 2; ++c) {
                double sign = ((a + b + c) % 2 == 1) ? 1.0 : -1.0;
#if ORACLE_PLANT == 2
                if (a == 1 && b == 0 && c == 0) sign = -sign; /* planted: corner */
#endif
                /* a+b+c = 3 (all upper) -> +, 2 -> -, 1 -> +, 0 -> - */
                s += sign * prism_antiderivative(xs[a], ys[b], zs[c]);
            }
    return s;
}

/* k(d) in units of 1/length (see header). */
double oracle_kernel(long dx, long dy, long dz, double hx, double hy, double hz,
                     int r_near)
{
    long ax = labs(dx), ay = labs(dy), az = labs(dz);
    long cheb = ax > ay ? ax : ay;
    if (az > cheb) cheb = az;
    if (cheb <= r_near) {
        double cx = (double)dx * hx, cy = (double)dy * hy, cz = (double)dz * hz;
#if ORACLE_PLANT == 3
        cx += 0.5 * hx; /* planted: off-by-half-cell source offset */
#endif
#if ORACLE_PLANT == 4
        { double t = hx; hx = hy; hy = t; } /* planted: transposed spacings */
#endif
        double v = oracle_box_integral(cx - 0.5 * hx, cx + 0.5 * hx,
                                       cy - 0.5 * hy, cy + 0.5 * hy,
                                       cz - 0.5 * hz, cz + 0.5 * hz);
        return v / (hx * hy * hz);
    }
    double x = (double)dx * hx, y = (double)dy * hy, z = (double)dz * hz;
    return 1.0 / sqrt(x * x + y * y + z * z);
}

/* out[(dz*(ky) + dy)*(kx) + dx] = k(dx,dy,dz) for 0 <= d < (kx,ky,kz). */
void oracle_kernel_octant(int kx, int ky, int kz, double hx, double hy, double hz,
                          int r_near, double *out)
{
    #pragma omp parallel for schedule(static)
    for (long dz = 0; dz < kz; ++dz)
        for (long dy = 0; dy < ky; ++dy)
            for (long dx = 0; dx < kx; ++dx)
                out[(dz * ky + dy) * kx + dx] = oracle_kernel(dx, dy, dz, hx, hy, hz, r_near);
}

/* Full direct pair sum.  koct is the octant table of k over offsets
 * [0,nx) x [0,ny) x [0,nz) (k is even in each axis under the reading above,
 * so k(d) = koct[|dz|][|dy|][|dx|]).  phi[i] = scale * sum_j k(i-j) rho[j]. */
void oracle_direct_sum(int nx, int ny, int nz, const double *rho,
                       const double *koct, double scale, double *phi)
{
    const long nxy = (long)nx * ny;
    #pragma omp parallel for schedule(dynamic, 1) collapse(2)
    for (long iz = 0; iz < nz; ++iz)
        for (long iy = 0; iy < ny; ++iy)
            for (long ix = 0; ix < nx; ++ix) {
                double acc = 0.0;
                for (long jz = 0; jz < nz; ++jz) {
                    long dz = labs(iz - jz);
                    for (long jy = 0; jy < ny; ++jy) {
                        long dy = labs(iy - jy);
                        const double *krow = koct + (dz * ny + dy) * nx;
                        const double *rrow = rho + jz * nxy + jy * nx;
                        for (long jx = 0; jx < nx; ++jx)
#if ORACLE_PLANT == 5
                            acc += krow[labs(ix - jx)] * rrow[nx - 1 - jx]; /* planted: index */
#else
                            acc += krow[labs(ix - jx)] * rrow[jx];
#endif
                    }
                }
                phi[iz * nxy + iy * nx + ix] = scale * acc;
            }
}

/* Direct sums at `count` target cells given as flat indices (z*ny + y)*nx + x. */
void oracle_direct_sum_points(int nx, int ny, int nz, const double *rho,
                              const double *koct, double scale, long count,
                              const int64_t *targets, double *out)
{
    const long nxy = (long)nx * ny;
    #pragma omp parallel for schedule(dynamic, 1)
    for (long t = 0; t < count; ++t) {
        long f = (long)targets[t];
        long iz = f / nxy, iy = (f / nx) % ny, ix = f % nx;
        double acc = 0.0;
        for (long jz = 0; jz < nz; ++jz) {
            long dz = labs(iz - jz);
            for (long jy = 0; jy < ny; ++jy) {
                long dy = labs(iy - jy);
                const double *krow = koct + (dz * ny + dy) * nx;
                const double *rrow = rho + jz * nxy + jy * nx;
                for (long jx = 0; jx < nx; ++jx)
                    acc += krow[labs(ix - jx)] * rrow[jx];
            }
        }
        out[t] = scale * acc;
    }
}

void oracle_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

int oracle_get_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
