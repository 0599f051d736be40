"""Seeded synthetic density fields for the free-space Poisson solve.

These generators are shared by the FP64 oracle (tests), the CUDA path's tests
and the benchmark.  They hold none of the solver's arithmetic: they only build
densities rho[z, y, x] (numpy float64, C order, x fastest) sampled at cell
centres.  Cell (ix, iy, iz) has its centre at (ix, iy, iz) in cell units.

The paper's case study solves potentials on nested meshes of N^3 cells with
N = 64 and 128 (Section 3); the shapes below stand in for those workloads with
the configurations the benchmark and tests use:

* gaussian_blobs  - a few seeded Gaussian blobs on a zero background
* plummer_spheres - seeded Plummer spheres plus a uniform background
* lognormal_field - a lognormal random field with a power-law spectrum
* uniform_sphere  - a constant-density ball (closed-form potential)
* batch_shapes    - seeded uneven field shapes for the batched solve
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "gaussian_blobs",
    "plummer_spheres",
    "lognormal_field",
    "uniform_sphere",
    "batch_shapes",
    "batch_densities",
    "random_weights",
]


def _axes(shape):
    nz, ny, nx = shape
    return (np.arange(nz, dtype=np.float64), np.arange(ny, dtype=np.float64),
            np.arange(nx, dtype=np.float64))


def _shape3(n):
    if np.isscalar(n):
        return (int(n),) * 3
    return tuple(int(v) for v in n)


def gaussian_blobs(n, count=4, seed=2409, centre_lo=None, centre_hi=None,
                   sigma=(2.0, 5.0), amplitude=(0.5, 2.0), truncate=6.0):
    """Sum of `count` Gaussian blobs A exp(-r^2 / (2 s^2)).

    Centres are uniform in [centre_lo, centre_hi) per axis (default: the
    middle half of the box, i.e. [8, 24) for a 32-cell edge), widths uniform
    in `sigma`, peak amplitudes uniform in `amplitude`.  Each blob is cut off
    beyond `truncate` widths per axis (relative size < exp(-18)), which keeps
    large batches cheap to build; `truncate=None` keeps the whole profile.
    Returns (rho, blobs) where blobs is a list of (centre_xyz, sigma, A).
    """
    shape = _shape3(n)
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    dims_xyz = np.array([nx, ny, nz], dtype=np.float64)
    lo = dims_xyz * 0.25 if centre_lo is None else np.broadcast_to(centre_lo, (3,))
    hi = dims_xyz * 0.75 if centre_hi is None else np.broadcast_to(centre_hi, (3,))
    rho = np.zeros(shape, dtype=np.float64)
    z, y, x = _axes(shape)
    blobs = []
    for _ in range(count):
        c = rng.uniform(lo, hi)
        s = rng.uniform(*sigma)
        a = rng.uniform(*amplitude)
        blobs.append((c, s, a))
        gx = np.exp(-((x - c[0]) ** 2) / (2 * s * s))
        gy = np.exp(-((y - c[1]) ** 2) / (2 * s * s))
        gz = np.exp(-((z - c[2]) ** 2) / (2 * s * s))
        if truncate is not None:
            gx[np.abs(x - c[0]) > truncate * s] = 0.0
            gy[np.abs(y - c[1]) > truncate * s] = 0.0
            gz[np.abs(z - c[2]) > truncate * s] = 0.0
        ix = np.nonzero(gx)[0]
        iy = np.nonzero(gy)[0]
        iz = np.nonzero(gz)[0]
        if len(ix) == 0 or len(iy) == 0 or len(iz) == 0:
            continue
        sl = (slice(iz[0], iz[-1] + 1), slice(iy[0], iy[-1] + 1), slice(ix[0], ix[-1] + 1))
        rho[sl] += a * (gz[sl[0], None, None] * gy[None, sl[1], None] * gx[None, None, sl[2]])
    return rho, blobs


def plummer_spheres(n, count=64, seed=2409, scale_radius=(2.0, 12.0),
                    mass=(1e-2, 1.0), background=0.01):
    """Sum of `count` Plummer spheres rho = 3M/(4 pi a^3) (1 + r^2/a^2)^(-5/2).

    Centres uniform in [0.09375 n, 0.90625 n) per axis ([24, 232) at n=256),
    scale radii a and masses M log-uniform over the given ranges, plus a
    uniform background equal to `background` times the mean of the sampled
    Plummer density.  Returns (rho, spheres) with spheres = [(c_xyz, a, M)].
    """
    shape = _shape3(n)
    rng = np.random.default_rng(seed)
    nz, ny, nx = shape
    dims_xyz = np.array([nx, ny, nz], dtype=np.float64)
    z, y, x = _axes(shape)
    import torch  # multithreaded elementwise work on the host cores
    rho_t = torch.zeros(shape, dtype=torch.float64)
    spheres = []
    for _ in range(count):
        c = rng.uniform(dims_xyz * 0.09375, dims_xyz * 0.90625)
        a = float(np.exp(rng.uniform(np.log(scale_radius[0]), np.log(scale_radius[1]))))
        m = float(np.exp(rng.uniform(np.log(mass[0]), np.log(mass[1]))))
        spheres.append((c, a, m))
        qz = torch.from_numpy(((z - c[2]) / a) ** 2)
        qy = torch.from_numpy(((y - c[1]) / a) ** 2)
        qx = torch.from_numpy(((x - c[0]) / a) ** 2)
        norm = 3.0 * m / (4.0 * np.pi * a ** 3)
        q = 1.0 + qz[:, None, None] + qy[None, :, None] + qx[None, None, :]
        rho_t += norm * q.pow_(-2.5)
        del q
    rho = rho_t.numpy()
    rho += background * rho.mean()
    return rho, spheres


def uniform_sphere(n, radius, centre=None, density=1.0):
    """Constant `density` inside a ball of `radius` cells (cell centres tested)."""
    shape = _shape3(n)
    nz, ny, nx = shape
    if centre is None:
        centre = ((nx - 1) / 2.0, (ny - 1) / 2.0, (nz - 1) / 2.0)
    z, y, x = _axes(shape)
    r2 = ((z - centre[2]) ** 2)[:, None, None] + ((y - centre[1]) ** 2)[None, :, None] \
        + ((x - centre[0]) ** 2)[None, None, :]
    return np.where(r2 <= radius * radius, density, 0.0)


def lognormal_field(n, seed=2409, sigma=1.5, slope=-3.0, sphere_radius=40.0,
                    sphere_density=1.0):
    """Lognormal field exp(sigma g - sigma^2/2) plus a uniform ball.

    g is a unit-variance Gaussian random field with power spectrum
    P(k) ~ |k|^slope (k = 0 removed), made by filtering seeded white noise
    with an FP64 FFT; the ball (radius `sphere_radius` cells, centred in the
    box) is added on top for a closed-form check of its excess potential.
    Returns (rho, sphere_only).
    """
    shape = _shape3(n)
    rng = np.random.default_rng(seed)
    try:
        import scipy.fft as sfft
        kw = {"workers": -1}
    except ImportError:  # pragma: no cover
        import numpy.fft as sfft
        kw = {}
    white = rng.standard_normal(shape)
    wk = sfft.rfftn(white, **kw)
    del white
    nz, ny, nx = shape
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.rfftfreq(nx)[None, None, :]
    k2 = kz * kz + ky * ky + kx * kx
    k2[0, 0, 0] = 1.0
    amp = k2 ** (slope / 4.0)
    amp[0, 0, 0] = 0.0
    wk *= amp
    del amp, k2
    g = sfft.irfftn(wk, s=shape, **kw)
    del wk
    g /= g.std()
    rho = np.exp(sigma * g - 0.5 * sigma * sigma)
    del g
    sphere = uniform_sphere(shape, sphere_radius, density=sphere_density)
    rho += sphere
    return rho, sphere


def batch_shapes(count=96, seed=2409, edges=(64, 96, 128, 192, 256, 384)):
    """Seeded uneven field shapes (nz, ny, nx) for the batched solve.

    Each field draws an edge e from `edges`; half are cubic (e, e, e) and half
    2:1 anisotropic (one long axis of e and two of e/2, the long axis drawn by
    seed).
    """
    rng = np.random.default_rng(seed)
    shapes = []
    for _ in range(count):
        e = int(rng.choice(edges))
        if rng.uniform() < 0.5:
            shapes.append((e, e, e))
        else:
            long_axis = int(rng.integers(0, 3))
            s = [e // 2] * 3
            s[long_axis] = e
            shapes.append(tuple(s))
    return shapes


def batch_densities(shapes, seed=2409, dtype=np.float32):
    """One seeded Gaussian-blob density (4-16 blobs, widths 3-10 % of the
    shortest edge) per shape, cast to `dtype`."""
    rng = np.random.default_rng(seed)
    out = []
    for i, shp in enumerate(shapes):
        count = int(rng.integers(4, 17))
        e = min(shp)
        rho, _ = gaussian_blobs(shp, count=count, seed=seed * 1000 + i,
                                sigma=(0.03 * e, 0.10 * e))
        out.append(rho.astype(dtype))
    return out


def random_weights(n, seed=2409):
    """Seeded weights w ~ U[-1, 1] of shape n (for the loss sum(w * Phi))."""
    rng = np.random.default_rng(seed)
    return rng.uniform(-1.0, 1.0, size=_shape3(n))
