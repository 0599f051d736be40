"""Pins of the FP64 oracle against values fixed by the mathematics (CPU only).

Each test checks the oracle against something other than itself: a closed
form, an independent quadrature, an identity of the discrete transform, a
brute-force sum, or a symmetry/invariant of the convolution.  The cases are
chosen so that a dropped term, a wrong sign, a wrong index or a transposed
operand in the oracle fails at least one of them (test_planted_mistakes
demonstrates that for mistakes planted into the oracle's C source).
"""
import math

import numpy as np
import pytest
from scipy.special import erf

import workloads

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


# --------------------------------------------------------------------------
# independent quadratures of 1/|r| over a box
# --------------------------------------------------------------------------

def _gl(npts, a, b):
    x, w = np.polynomial.legendre.leggauss(npts)
    return 0.5 * (b - a) * x + 0.5 * (b + a), 0.5 * (b - a) * w


def gauss_box(x0, x1, y0, y1, z0, z1, npts=24, split=4):
    """Tensor Gauss-Legendre on a box that does not contain the origin
    (smooth integrand); each axis split into `split` panels."""
    tot = 0.0
    ex = np.linspace(x0, x1, split + 1)
    ey = np.linspace(y0, y1, split + 1)
    ez = np.linspace(z0, z1, split + 1)
    for i in range(split):
        xs, wx = _gl(npts, ex[i], ex[i + 1])
        for j in range(split):
            ys, wy = _gl(npts, ey[j], ey[j + 1])
            for k in range(split):
                zs, wz = _gl(npts, ez[k], ez[k + 1])
                X, Y, Z = np.meshgrid(xs, ys, zs, indexing="ij")
                W = wx[:, None, None] * wy[None, :, None] * wz[None, None, :]
                tot += np.sum(W / np.sqrt(X * X + Y * Y + Z * Z))
    return tot


def corner_box_pyramids(a, b, c, npts=60):
    """Integral of 1/r over [0,a]x[0,b]x[0,c] (singular corner at the
    origin) by splitting into the three pyramids with apex at the origin
    and bases on the far faces; in each, (y, z) = x (s, t) turns the
    integral into a^2/2 * I(b/a, c/a) with I(p, q) the smooth integral of
    (1 + s^2 + t^2)^(-1/2) over [0,p] x [0,q]."""
    def I(p, q):
        s, ws = _gl(npts, 0.0, p)
        t, wt = _gl(npts, 0.0, q)
        S, T = np.meshgrid(s, t, indexing="ij")
        return np.sum(ws[:, None] * wt[None, :] / np.sqrt(1.0 + S * S + T * T))
    return 0.5 * a * a * I(b / a, c / a) + 0.5 * b * b * I(a / b, c / b) \
        + 0.5 * c * c * I(a / c, b / c)


# --------------------------------------------------------------------------
# Green's function
# --------------------------------------------------------------------------

def test_self_cell_unit_cube_closed_form(oracle_mod):
    # Potential at the centre of a uniform unit cube (textbook closed form):
    # integral of 1/r over [-1/2,1/2]^3 = 3 ln((sqrt3+1)/(sqrt3-1)) - pi/2.
    s3 = math.sqrt(3.0)
    exact = 3.0 * math.log((s3 + 1.0) / (s3 - 1.0)) - math.pi / 2.0
    assert oracle_mod.kernel((0, 0, 0)) == pytest.approx(exact, rel=1e-14)
    # scaling: k(0; h) = k(0; 1) / h for cubic cells
    assert oracle_mod.kernel((0, 0, 0), h=0.25) == pytest.approx(exact / 0.25, rel=1e-14)


@pytest.mark.parametrize("h", [(1.0, 1.0, 1.0), (1.0, 0.5, 2.0), (0.3, 0.7, 0.45)])
def test_self_cell_vs_pyramid_quadrature(oracle_mod, h):
    hx, hy, hz = h
    quad = 8.0 * corner_box_pyramids(hx / 2, hy / 2, hz / 2) / (hx * hy * hz)
    assert oracle_mod.kernel((0, 0, 0), h=h) == pytest.approx(quad, rel=1e-12)


@pytest.mark.parametrize("d", [(1, 0, 0), (0, 1, 0), (0, 0, 1), (1, 1, 0), (1, 1, 1),
                               (2, 0, 0), (3, -2, 1), (-5, 4, 2), (8, 8, 8), (0, 7, -8)])
@pytest.mark.parametrize("h", [(1.0, 1.0, 1.0), (1.0, 0.5, 2.0)])
def test_near_cells_vs_gauss_quadrature(oracle_mod, d, h):
    hx, hy, hz = h
    cx, cy, cz = d[0] * hx, d[1] * hy, d[2] * hz
    quad = gauss_box(cx - hx / 2, cx + hx / 2, cy - hy / 2, cy + hy / 2,
                     cz - hz / 2, cz + hz / 2) / (hx * hy * hz)
    assert oracle_mod.kernel(d, h=h) == pytest.approx(quad, rel=1e-11)


def test_far_cells_point_value_and_cube_average_limit(oracle_mod):
    # beyond r_near the reading takes the point value 1/|d h| ...
    for d in [(9, 0, 0), (9, 4, 1), (20, 13, 7)]:
        r = math.sqrt(sum(v * v for v in d))
        assert oracle_mod.kernel(d) == 1.0 / r
    # ... which the exact cube average approaches as |d|^-5 (relative
    # O(|d|^-4): the cube's second moment is isotropic and 1/r harmonic)
    errs = []
    for m in (4, 8, 16):
        avg = oracle_mod.kernel((m, 0, 0), r_near=64)
        errs.append(abs(avg - 1.0 / m))
    assert errs[0] / errs[1] == pytest.approx(32.0, rel=0.15)
    assert errs[1] / errs[2] == pytest.approx(32.0, rel=0.15)
    # with r_near = 8 the switch costs at most a few 1e-6 relative
    for d in [(9, 0, 0), (9, 4, 0), (9, 9, 9)]:
        exact = oracle_mod.kernel(d, r_near=64)
        assert abs(oracle_mod.kernel(d) / exact - 1.0) < 3e-6


def test_kernel_symmetries(oracle_mod):
    rng = np.random.default_rng(1)
    for _ in range(20):
        d = rng.integers(-9, 10, size=3)
        base = oracle_mod.kernel(d)
        for sx in (1, -1):
            for sy in (1, -1):
                for sz in (1, -1):
                    assert oracle_mod.kernel((sx * d[0], sy * d[1], sz * d[2])) == \
                        pytest.approx(base, rel=1e-13)
        for perm in [(1, 0, 2), (2, 1, 0), (0, 2, 1), (1, 2, 0), (2, 0, 1)]:
            assert oracle_mod.kernel(d[list(perm)]) == pytest.approx(base, rel=1e-12)
    # anisotropic spacing: swapping an offset and its spacing together
    h = (1.0, 0.5, 2.0)
    assert oracle_mod.kernel((2, 1, 0), h=h) == pytest.approx(
        oracle_mod.kernel((1, 2, 0), h=(0.5, 1.0, 2.0)), rel=1e-12)


def test_kernel_octant_layout(oracle_mod):
    K = oracle_mod.kernel_octant((5, 4, 3), h=(1.0, 0.5, 2.0))
    assert K.shape == (3, 4, 5)
    for dz in range(3):
        for dy in range(4):
            for dx in range(5):
                assert K[dz, dy, dx] == oracle_mod.kernel((dx, dy, dz), h=(1.0, 0.5, 2.0))


# --------------------------------------------------------------------------
# DFT matrices
# --------------------------------------------------------------------------

@pytest.mark.parametrize("M", [6, 16, 24, 64])
def test_dft_matrix_identities(oracle_mod, M):
    F = oracle_mod.dft_matrix(M)
    Fi = oracle_mod.dft_matrix(M, inverse=True)
    assert np.allclose(F @ Fi, M * np.eye(M), atol=1e-11)
    x = np.random.default_rng(M).standard_normal(M) + 1j * np.random.default_rng(M + 1).standard_normal(M)
    # Parseval: ||F x||^2 = M ||x||^2
    assert np.sum(np.abs(F @ x) ** 2) == pytest.approx(M * np.sum(np.abs(x) ** 2), rel=1e-13)
    # a shifted impulse transforms to a pure phase ramp
    e = np.zeros(M)
    e[1] = 1.0
    assert np.allclose(F @ e, np.exp(-2j * np.pi * np.arange(M) / M), atol=1e-14)


# --------------------------------------------------------------------------
# convolution routes
# --------------------------------------------------------------------------

@pytest.mark.parametrize("shape,h", [((8, 8, 8), 1.0), ((6, 10, 12), (1.0, 0.5, 2.0)),
                                      ((12, 6, 9), (0.7, 1.3, 0.9))])
def test_three_routes_agree(oracle_mod, shape, h):
    rng = np.random.default_rng(7)
    rho = rng.standard_normal(shape)
    a = oracle_mod.solve_direct(rho, h=h, G=1.7)
    b = oracle_mod.solve_dft(rho, h=h, G=1.7)
    c = oracle_mod.solve_fft(rho, h=h, G=1.7)
    scale = np.abs(a).max()
    assert np.abs(a - b).max() < 1e-13 * scale
    assert np.abs(a - c).max() < 1e-13 * scale


def test_routes_agree_32_cube_blobs(oracle_mod):
    rho, _ = workloads.gaussian_blobs(32, count=4, seed=2409)
    a = oracle_mod.solve_direct(rho)
    c = oracle_mod.solve_fft(rho)
    assert np.linalg.norm(a - c) / np.linalg.norm(a) < 1e-14
    idx = np.random.default_rng(3).choice(rho.size, 50, replace=False)
    s = oracle_mod.sample_direct(rho, idx)
    assert np.abs(s - a.reshape(-1)[idx]).max() < 1e-13 * np.abs(a).max()


@pytest.mark.parametrize("route", ["direct", "dft", "fft"])
def test_impulse_response(oracle_mod, route):
    # rho = delta at j gives Phi(i) = -G V k(i - j) exactly
    shape = (7, 6, 5)
    h = (1.0, 0.5, 2.0)
    V = 1.0 * 0.5 * 2.0
    solve = {"direct": oracle_mod.solve_direct, "dft": oracle_mod.solve_dft,
             "fft": oracle_mod.solve_fft}[route]
    for j in [(0, 0, 0), (6, 5, 4), (3, 2, 1)]:
        rho = np.zeros(shape)
        rho[j] = 1.0
        phi = solve(rho, h=h, G=2.0)
        for i in [(0, 0, 0), (6, 5, 4), (2, 4, 1), j]:
            d = (i[2] - j[2], i[1] - j[1], i[0] - j[0])  # (dx, dy, dz)
            assert phi[i] == pytest.approx(-2.0 * V * oracle_mod.kernel(d, h=h), rel=1e-12)
    # opposite corners of an n^3 box: far-corner value -G V / (h sqrt3 (n-1))
    n = 16
    rho = np.zeros((n, n, n))
    rho[0, 0, 0] = 1.0
    phi = solve(rho)
    assert phi[-1, -1, -1] == pytest.approx(-1.0 / (math.sqrt(3.0) * (n - 1)), rel=1e-12)


def test_fft_route_with_a_reused_kernel_transform(oracle_mod):
    # kernel_rfft once, then solve_fft_with for several densities of the
    # grid: each result is the direct pair sum of its own density (an
    # anisotropic grid, so a transposed kernel or spacing fails)
    shape, h, G = (6, 9, 7), (1.0, 0.5, 2.0), 1.3
    Kh = oracle_mod.kernel_rfft(shape, h=h, G=G)
    rng = np.random.default_rng(31)
    for _ in range(3):
        rho = rng.standard_normal(shape)
        a = oracle_mod.solve_direct(rho, h=h, G=G)
        b = oracle_mod.solve_fft_with(rho, Kh)
        assert np.linalg.norm(a - b) / np.linalg.norm(a) < 1e-13


def test_linearity_and_translation(oracle_mod):
    rng = np.random.default_rng(11)
    a = rng.standard_normal((10, 10, 10))
    b = rng.standard_normal((10, 10, 10))
    pa = oracle_mod.solve_fft(a)
    pb = oracle_mod.solve_fft(b)
    pab = oracle_mod.solve_fft(2.5 * a - 0.75 * b)
    assert np.abs(pab - (2.5 * pa - 0.75 * pb)).max() < 1e-12 * np.abs(pab).max()
    # translation: a blob shifted by s gives Phi shifted by s, on the overlap
    rho, _ = workloads.gaussian_blobs(24, count=1, seed=5, centre_lo=9, centre_hi=10, sigma=(1.5, 1.5))
    sh = np.roll(rho, (2, 3, 1), axis=(0, 1, 2))
    p0 = oracle_mod.solve_direct(rho)
    p1 = oracle_mod.solve_direct(sh)
    # exact when no density wraps: compare p1[i+s] with p0[i] on the overlap
    assert np.abs(p1 - p0).max() > 1e-3 * np.abs(p0).max()  # the shift matters
    # the shifted sum differs from p0 only through sources that crossed the
    # box edge (none here: the blob is far from the edges)
    assert np.abs(p1[2:, 3:, 1:] - p0[:-2, :-3, :-1]).max() < 1e-9 * np.abs(p0).max()


def _relabelling_holds(solve, rho, hx, hy, hz, tol):
    p = solve(rho, h=(hx, hy, hz))
    scale = np.abs(p).max()
    h_arr = (hz, hy, hx)  # spacing of array axes 0, 1, 2
    for perm in [(2, 1, 0), (1, 0, 2), (0, 2, 1), (1, 2, 0)]:
        h_new = tuple(h_arr[a] for a in perm)
        q = solve(np.ascontiguousarray(np.transpose(rho, perm)), h=(h_new[2], h_new[1], h_new[0]))
        if np.abs(q - np.transpose(p, perm)).max() >= tol * scale:
            return False
    return True


@pytest.mark.parametrize("route", ["solve_direct", "solve_fft"])
def test_reflection_and_axis_relabelling(oracle_mod, route):
    # the kernel is even along every axis: flipping rho along an axis flips
    # Phi.  The cell average depends on the offset and the spacings only
    # through the box they span, so relabelling the array axes together
    # with their spacings relabels Phi's axes: a spacing tied to the wrong
    # axis, or a transposed offset, breaks this on an anisotropic grid
    solve = getattr(oracle_mod, route)
    rng = np.random.default_rng(21)
    rho = rng.standard_normal((6, 10, 12))  # [z][y][x]
    hx, hy, hz = 0.7, 1.3, 0.9
    p = solve(rho, h=(hx, hy, hz))
    scale = np.abs(p).max()
    for ax in range(3):
        assert np.abs(solve(np.flip(rho, ax), h=(hx, hy, hz)) - np.flip(p, ax)).max() < 1e-12 * scale
    h_arr = (hz, hy, hx)  # spacing of array axes 0, 1, 2
    for perm in [(2, 1, 0), (1, 0, 2), (0, 2, 1), (1, 2, 0)]:
        h_new = tuple(h_arr[a] for a in perm)
        q = solve(np.ascontiguousarray(np.transpose(rho, perm)), h=(h_new[2], h_new[1], h_new[0]))
        assert np.abs(q - np.transpose(p, perm)).max() < 1e-12 * scale, perm
        # the same relabelling without its spacings is a different problem
        q_wrong = solve(np.ascontiguousarray(np.transpose(rho, perm)), h=(hx, hy, hz))
        assert np.abs(q_wrong - np.transpose(p, perm)).max() > 1e-3 * scale, perm


def test_padding_length_invariance(oracle_mod):
    # any M >= 2n - 1 per axis gives the same free-space result
    rng = np.random.default_rng(2)
    rho = rng.standard_normal((6, 7, 8))
    base = oracle_mod.solve_fft(rho)
    for M in [(11, 13, 15), (14, 16, 18), (18, 21, 24)]:
        other = oracle_mod.solve_fft(rho, M_zyx=M)
        assert np.abs(other - base).max() < 1e-12 * np.abs(base).max()
    other = oracle_mod.solve_dft(rho, M_zyx=(13, 14, 17))
    assert np.abs(other - base).max() < 1e-12 * np.abs(base).max()
    # too little padding wraps around (M = 2n - 2 happens to be masked by the
    # kernel's evenness, M = 2n - 4 is not)
    bad = oracle_mod.solve_fft(rho, M_zyx=(8, 10, 12))
    assert np.abs(bad - base).max() > 1e-6 * np.abs(base).max()


def test_self_adjoint(oracle_mod):
    rng = np.random.default_rng(4)
    rho = rng.standard_normal((9, 8, 7))
    w = rng.standard_normal((9, 8, 7))
    lhs = np.sum(w * oracle_mod.solve_fft(rho, h=(1.0, 0.5, 2.0)))
    rhs = np.sum(oracle_mod.solve_adjoint_direct(w, h=(1.0, 0.5, 2.0)) * rho)
    assert lhs == pytest.approx(rhs, rel=1e-12)
    # L = sum(w Phi) is linear in rho: a central difference is exact up to rounding
    g = oracle_mod.solve_adjoint_direct(w)
    e = np.zeros_like(rho)
    e[4, 3, 2] = 1.0
    fd = (np.sum(w * oracle_mod.solve_direct(rho + 1e-3 * e)) -
          np.sum(w * oracle_mod.solve_direct(rho - 1e-3 * e))) / 2e-3
    assert fd == pytest.approx(g[4, 3, 2], rel=1e-9)


# --------------------------------------------------------------------------
# closed-form potentials (discretisation-level tolerances)
# --------------------------------------------------------------------------

def _gauss_case(oracle_mod, n, s, A=1.3, c=(19.3, 20.1, 19.7), G=1.0):
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    rho = A * np.exp(-r ** 2 / (2 * s * s))
    phi = oracle_mod.solve_fft(rho, G=G)
    Mb = A * (2 * np.pi) ** 1.5 * s ** 3
    ex = -G * Mb * erf(r / (math.sqrt(2.0) * s)) / np.maximum(r, 1e-300)
    return np.linalg.norm(phi - ex) / np.linalg.norm(ex)


def test_gaussian_blob_closed_form_and_second_order(oracle_mod):
    # Phi = -G M erf(r / (sqrt2 s)) / r with M = A (2 pi)^(3/2) s^3
    e1 = _gauss_case(oracle_mod, 40, 2.5)
    e2 = _gauss_case(oracle_mod, 40, 3.5)
    assert e1 < 5e-3 and e2 < 3e-3
    # second-order convergence in h/s
    assert e1 / e2 == pytest.approx((3.5 / 2.5) ** 2, rel=0.3)
    # G scales linearly
    assert _gauss_case(oracle_mod, 40, 3.5, G=3.0) == pytest.approx(e2, rel=1e-9)


def test_uniform_sphere_closed_form(oracle_mod):
    n, R, rho0 = 40, 10.0, 1.0
    c = (19.5, 19.5, 19.5)
    rho = workloads.uniform_sphere(n, R, centre=c, density=rho0)
    phi = oracle_mod.solve_fft(rho)
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    r = np.sqrt((x - c[0]) ** 2 + (y - c[1]) ** 2 + (z - c[2]) ** 2)
    inside = r < 0.6 * R
    ex_in = -2.0 * math.pi * rho0 * (R * R - r[inside] ** 2 / 3.0)
    assert np.abs(phi[inside] - ex_in).max() < 2e-2 * np.abs(ex_in).max()
    # outside, with the staircased (discrete) mass: -G M / r
    mass = rho.sum()
    outside = r > 1.8 * R
    ex_out = -mass / r[outside]
    assert np.abs(phi[outside] / ex_out - 1.0).max() < 2e-3


def test_point_mass_far_field(oracle_mod):
    rho, blobs = workloads.gaussian_blobs(32, count=1, seed=9, centre_lo=3.5, centre_hi=4.5,
                                          sigma=(1.2, 1.2), amplitude=(1.0, 1.0), truncate=None)
    phi = oracle_mod.solve_fft(rho)
    c = blobs[0][0]
    M = rho.sum()
    for i in [(31, 31, 31), (31, 0, 31), (0, 31, 31), (20, 25, 30)]:
        r = math.sqrt((i[2] - c[0]) ** 2 + (i[1] - c[1]) ** 2 + (i[0] - c[2]) ** 2)
        assert phi[i] == pytest.approx(-M / r, rel=2e-4)


# --------------------------------------------------------------------------
# planted mistakes: each wrong variant of the oracle must fail a pin
# --------------------------------------------------------------------------

def _pins_pass(oracle_mod):
    """Run a compact subset of the pins above; True if all hold."""
    checks = []
    s3 = math.sqrt(3.0)
    exact0 = 3.0 * math.log((s3 + 1.0) / (s3 - 1.0)) - math.pi / 2.0
    checks.append(abs(oracle_mod.kernel((0, 0, 0)) / exact0 - 1) < 1e-12)
    h = (1.0, 0.5, 2.0)
    for d in [(1, 0, 0), (1, 1, 1), (3, -2, 1)]:
        cx, cy, cz = d[0] * h[0], d[1] * h[1], d[2] * h[2]
        quad = gauss_box(cx - h[0] / 2, cx + h[0] / 2, cy - h[1] / 2, cy + h[1] / 2,
                         cz - h[2] / 2, cz + h[2] / 2, npts=12, split=2) / (h[0] * h[1] * h[2])
        checks.append(abs(oracle_mod.kernel(d, h=h) / quad - 1) < 1e-9)
    rng = np.random.default_rng(7)
    rho = rng.standard_normal((6, 7, 8))
    a = oracle_mod.solve_direct(rho, h=h)
    c = oracle_mod.solve_fft(rho, h=h)
    checks.append(np.abs(a - c).max() < 1e-12 * np.abs(a).max())
    return all(checks)


@pytest.mark.parametrize("which", [1, 2, 3, 4, 5])
def test_planted_mistakes_fail_a_pin(oracle_mod, which, tmp_path):
    assert _pins_pass(oracle_mod)
    so = oracle_mod.build_planted(which, str(tmp_path))
    oracle_mod.use_library(so)
    try:
        assert not _pins_pass(oracle_mod), "planted mistake %d went unnoticed" % which
    finally:
        oracle_mod.use_library(None)
    assert _pins_pass(oracle_mod)


@pytest.mark.parametrize("which", [4, 5])
def test_relabelling_pin_alone_catches_axis_mistakes(oracle_mod, which, tmp_path):
    # transposed spacings (4) and a mirrored source index along x (5): the
    # relabelling pin by itself fails both (a mirrored index still passes
    # the reflection half, so it is the relabelling that catches it)
    rho = np.random.default_rng(21).standard_normal((6, 10, 12))
    assert _relabelling_holds(oracle_mod.solve_direct, rho, 0.7, 1.3, 0.9, 1e-12)
    so = oracle_mod.build_planted(which, str(tmp_path))
    oracle_mod.use_library(so)
    try:
        assert not _relabelling_holds(oracle_mod.solve_direct, rho, 0.7, 1.3, 0.9, 1e-9)
    finally:
        oracle_mod.use_library(None)


# ---------------------------------------------------------------------------
# caller-supplied even kernels (generalisation of the Green's function)
# ---------------------------------------------------------------------------

def _even_kernel(shape_zyx, seed):
    """A random octant k[dz, dy, dx] (any values: evenness is by construction)."""
    return np.random.default_rng(seed).standard_normal(shape_zyx)


def test_user_kernel_delta_and_constant_closed_forms(oracle_mod):
    rng = np.random.default_rng(11)
    rho = rng.standard_normal((5, 6, 7))
    delta = np.zeros((6, 7, 8))
    delta[0, 0, 0] = 1.0
    # k = delta: Phi = scale * rho exactly (direct) and to rounding (FFT)
    assert np.array_equal(oracle_mod.solve_direct_kernel(rho, delta, 2.5), 2.5 * rho)
    np.testing.assert_allclose(oracle_mod.solve_fft_kernel(rho, delta, 2.5), 2.5 * rho, rtol=0, atol=1e-13)
    # k = 1: Phi[i] = scale * sum(rho) at every cell
    ones = np.ones((6, 7, 8))
    want = np.full(rho.shape, -0.75 * rho.sum())
    np.testing.assert_allclose(oracle_mod.solve_direct_kernel(rho, ones, -0.75), want, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(oracle_mod.solve_fft_kernel(rho, ones, -0.75), want, rtol=1e-12, atol=1e-12)


def test_user_kernel_brute_force_and_route_agreement(oracle_mod):
    # brute force in plain Python loops on a tiny grid, then the two routes
    rng = np.random.default_rng(12)
    nz, ny, nx = 3, 4, 5
    rho = rng.standard_normal((nz, ny, nx))
    k = _even_kernel((nz + 1, ny + 1, nx + 1), 13)
    brute = np.zeros_like(rho)
    for iz in range(nz):
        for iy in range(ny):
            for ix in range(nx):
                s = 0.0
                for jz in range(nz):
                    for jy in range(ny):
                        for jx in range(nx):
                            s += k[abs(iz - jz), abs(iy - jy), abs(ix - jx)] * rho[jz, jy, jx]
                brute[iz, iy, ix] = 1.5 * s
    np.testing.assert_allclose(oracle_mod.solve_direct_kernel(rho, k, 1.5), brute, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(oracle_mod.solve_fft_kernel(rho, k, 1.5), brute, rtol=1e-12, atol=1e-12)
    # larger grid: direct sum = FFT route
    rho = rng.standard_normal((9, 10, 12))
    k = _even_kernel((10, 11, 13), 14)
    a = oracle_mod.solve_direct_kernel(rho, k, 0.5)
    b = oracle_mod.solve_fft_kernel(rho, k, 0.5)
    assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def test_user_kernel_with_the_greens_octant_is_the_poisson_solve(oracle_mod):
    rho = np.random.default_rng(15).standard_normal((6, 7, 8))
    h = (1.0, 0.5, 2.0)
    koct = oracle_mod.kernel_octant((9, 8, 7), h=h)  # extents x, y, z = n + 1
    a = oracle_mod.solve_direct_kernel(rho, koct, -1.0 * 1.0 * 0.5 * 2.0)
    b = oracle_mod.solve_direct(rho, h=h)
    assert np.abs(a - b).max() <= 1e-14 * np.abs(b).max()


# ---------------------------------------------------------------------------
# golden fixture (tests/golden): written by the oracle; pins it against change
# ---------------------------------------------------------------------------

def _golden():
    import importlib.util
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "make_golden.py")
    spec = importlib.util.spec_from_file_location("make_golden", path)
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    data = np.loadtxt(mg.OUT, comments="#")
    return mg, data[:, 0].astype(np.int64), data[:, 4]


def test_oracle_reproduces_the_golden_fixture(oracle_mod):
    mg, idx, phi = _golden()
    got = oracle_mod.sample_direct(mg.density(), idx, h=mg.H, G=1.0)
    assert np.abs(got - phi).max() <= 1e-13 * np.abs(phi).max()


def test_cell_averages_add_up_to_the_whole_box_integral(oracle_mod):
    # with r_near >= n every pair uses the exact cell average, so the direct
    # sum for a uniform density is the potential of the whole box: the
    # classical prism antiderivative over its 8 corners, written out here
    # independently and anchored by the textbook cube-centre value
    def F(u, v, w):
        r = math.sqrt(u * u + v * v + w * w)
        t = 0.0
        if r > 0:
            t += v * w * math.log(u + r) if u + r > 0 else 0.0
            t += w * u * math.log(v + r) if v + r > 0 else 0.0
            t += u * v * math.log(w + r) if w + r > 0 else 0.0
            if u != 0:
                t -= 0.5 * u * u * math.atan(v * w / (u * r))
            if v != 0:
                t -= 0.5 * v * v * math.atan(w * u / (v * r))
            if w != 0:
                t -= 0.5 * w * w * math.atan(u * v / (w * r))
        return t

    def box(x, y, z, a, b, c):
        tot = 0.0
        for i, u in ((0, a - x), (1, -x)):
            for j, v in ((0, b - y), (1, -y)):
                for k, w in ((0, c - z), (1, -z)):
                    tot += (-1) ** (i + j + k) * F(u, v, w)
        return tot

    s3 = math.sqrt(3.0)
    assert box(0.5, 0.5, 0.5, 1, 1, 1) == pytest.approx(3 * math.log((s3 + 1) / (s3 - 1)) - math.pi / 2, rel=1e-14)
    n, h = (16, 8, 12), (1.0, 0.75, 0.5)
    phi = oracle_mod.solve_direct(np.ones(n), h=h, G=1.0, r_near=16)
    for iz, iy, ix in [(0, 0, 0), (8, 4, 6), (15, 7, 11), (3, 5, 2), (10, 0, 9)]:
        want = -box((ix + 0.5) * h[0], (iy + 0.5) * h[1], (iz + 0.5) * h[2], n[2] * h[0], n[1] * h[1], n[0] * h[2])
        assert phi[iz, iy, ix] == pytest.approx(want, rel=1e-12)
