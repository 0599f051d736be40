"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Tolerances: FP64 data path rel-L2 <= 1e-12 and max-norm <= 1e-11 max|Phi|;
FP32 data path rel-L2 <= 1e-6 and max-norm <= 1e-5 max|Phi| (the FP32
solve's stated tolerance; FP32 rounding of the input is applied before the
oracle sees it, so only the solver's own error is measured).
"""
import math

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = (1e-6, 1e-5)
TOL64 = (1e-12, 1e-11)


@pytest.fixture(scope="module")
def pg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2409_02294_gb300 as pg
    pg.lib()
    return pg


def rel_errors(out, ref):
    out = np.asarray(out, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    l2 = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    mx = np.abs(out - ref).max() / np.abs(ref).max()
    return l2, mx


def gpu_solve(pg, rho, h=1.0, G=1.0, precision="fp32", flags=0):
    nz, ny, nx = rho.shape
    dt = torch.float64 if precision == "fp64" else torch.float32
    with pg.Plan(nx, ny, nz, h=h, G=G, precision=precision, flags=flags) as plan:
        x = torch.from_numpy(np.ascontiguousarray(rho)).to(device="cuda", dtype=dt)
        phi = plan.solve(x)
        torch.cuda.synchronize()
        return phi.double().cpu().numpy()


# ---------------------------------------------------------------------------
# Green's function (plan time, FP64 on the GPU)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape,h", [((16, 16, 16), 1.0), ((32, 16, 48), (1.0, 0.5, 2.0)),
                                      ((48, 32, 16), (0.7, 1.3, 0.9)), ((16, 64, 96), (1.0, 0.8, 1.2)),
                                      ((128, 192, 16), 1.0), ((256, 16, 32), (0.5, 1.0, 1.0)),
                                      ((384, 16, 16), 1.0), ((512, 16, 16), (1.0, 1.0, 0.5))])
def test_greens_octant_matches_oracle(pg, oracle_mod, shape, h):
    # the plan's FP64 DCT-I (line FFTs of every supported length) against the
    # oracle's full FFT of the wrapped kernel
    nz, ny, nx = shape
    ref = oracle_mod.greens_hat(shape, h=h, G=1.7).real[:nz + 1, :ny + 1, :nx + 1] / (8.0 * nx * ny * nz)
    with pg.Plan(nx, ny, nz, h=h, G=1.7, precision="fp64") as plan:
        g64 = plan.greens_octant()
    assert np.abs(g64 - ref).max() <= 1e-12 * np.abs(ref).max()
    with pg.Plan(nx, ny, nz, h=h, G=1.7, precision="fp32") as plan:
        g32 = plan.greens_octant()
    # FP32 storage of the FP64 result: one rounding per value
    assert np.all(np.abs(g32 - ref) <= 6e-8 * np.abs(ref) + 1e-30)


def test_greens_near_field_radius(pg, oracle_mod):
    shape = (32, 32, 32)
    for r_near in (0, 3, 8):
        ref = oracle_mod.greens_hat(shape, r_near=r_near).real[:33, :33, :33] / (8.0 * 32 ** 3)
        with pg.Plan(32, 32, 32, precision="fp64", r_near=r_near) as plan:
            g = plan.greens_octant()
        assert np.abs(g - ref).max() <= 1e-12 * np.abs(ref).max()


# ---------------------------------------------------------------------------
# FP64 data path: 32^3, four Gaussian blobs, against the direct pair sum
# ---------------------------------------------------------------------------

def test_fp64_32cube_blobs_vs_direct_pair_sum(pg, oracle_mod):
    rho, _ = workloads.gaussian_blobs(32, count=4, seed=2409)
    ref = oracle_mod.solve_direct(rho)
    out = gpu_solve(pg, rho, precision="fp64")
    l2, mx = rel_errors(out, ref)
    assert l2 <= TOL64[0] and mx <= TOL64[1], (l2, mx)


@pytest.mark.parametrize("shape,h", [((16, 48, 32), (1.0, 0.5, 2.0)), ((48, 16, 16), 1.0),
                                      ((16, 16, 96), (0.3, 0.3, 0.3))])
def test_fp64_anisotropic_vs_oracle(pg, oracle_mod, shape, h):
    rho = np.random.default_rng(5).standard_normal(shape)
    ref = oracle_mod.solve_fft(rho, h=h, G=0.8)
    out = gpu_solve(pg, rho, h=h, G=0.8, precision="fp64")
    l2, mx = rel_errors(out, ref)
    assert l2 <= TOL64[0] and mx <= TOL64[1], (l2, mx)


# ---------------------------------------------------------------------------
# FP32 data path, every supported edge length, ragged tiles
# ---------------------------------------------------------------------------

SHAPES32 = [
    (16, 16, 16), (48, 16, 16), (16, 48, 32), (32, 64, 48), (64, 96, 16),
    (96, 32, 128), (16, 192, 64), (192, 16, 32), (32, 32, 256), (16, 256, 16),
    (256, 16, 48), (16, 16, 384), (384, 16, 16), (16, 384, 16), (16, 16, 512),
    (512, 16, 16), (16, 512, 16),
]


@pytest.mark.parametrize("shape", SHAPES32)
def test_fp32_sizes_vs_oracle(pg, oracle_mod, shape):
    rng = np.random.default_rng(sum(shape))
    rho = rng.standard_normal(shape).astype(np.float32).astype(np.float64)
    h = (1.0, 0.75, 1.25)
    ref = oracle_mod.solve_fft(rho, h=h, G=1.0)
    out = gpu_solve(pg, rho, h=h)
    l2, mx = rel_errors(out, ref)
    assert l2 <= TOL32[0] and mx <= TOL32[1], (l2, mx)


def test_fp32_impulse_response(pg, oracle_mod):
    n = 32
    rho = np.zeros((n, n, n))
    rho[0, 0, 0] = 1.0
    rho[-1, -1, -1] = 1.0
    out = gpu_solve(pg, rho)
    ref = oracle_mod.solve_direct(rho)
    l2, mx = rel_errors(out, ref)
    assert l2 <= TOL32[0] and mx <= TOL32[1]
    # k(0) on the self cell and the far corner value are recovered
    s3 = math.sqrt(3.0)
    k0 = 3.0 * math.log((s3 + 1.0) / (s3 - 1.0)) - math.pi / 2.0
    assert out[0, 0, 0] == pytest.approx(-(k0 + 1.0 / (s3 * (n - 1))), rel=1e-5)


def test_fp32_zero_input_gives_zero(pg):
    out = gpu_solve(pg, np.zeros((32, 48, 64)))
    assert np.all(out == 0.0)


def test_fp32_linearity_and_G_scaling(pg):
    rng = np.random.default_rng(3)
    a = rng.standard_normal((32, 32, 32)).astype(np.float32)
    b = rng.standard_normal((32, 32, 32)).astype(np.float32)
    pa, pb = gpu_solve(pg, a), gpu_solve(pg, b)
    pab = gpu_solve(pg, (a + b).astype(np.float32).astype(np.float64))
    assert np.abs(pab - (pa + pb)).max() < 1e-5 * np.abs(pab).max()
    p3 = gpu_solve(pg, a, G=3.0)
    assert np.abs(p3 - 3.0 * pa).max() < 1e-5 * np.abs(p3).max()


# ---------------------------------------------------------------------------
# configuration workloads
# ---------------------------------------------------------------------------

def test_fp32_256cube_plummer_full_field(pg, oracle_mod):
    rho, _ = workloads.plummer_spheres(256, count=64, seed=2409)
    rho32 = rho.astype(np.float32)
    ref = oracle_mod.solve_fft(rho32.astype(np.float64))
    out = gpu_solve(pg, rho32, flags=pg.abi.FLAG_AUTOTUNE)  # the benchmark's launch configuration
    l2, mx = rel_errors(out, ref)
    assert l2 <= TOL32[0] and mx <= TOL32[1], (l2, mx)


def test_fp32_512cube_lognormal_sampled(pg, oracle_mod):
    rho, sphere = workloads.lognormal_field(512, seed=2409)
    rho32 = rho.astype(np.float32)
    out = gpu_solve(pg, rho32, flags=pg.abi.FLAG_AUTOTUNE)  # the benchmark's launch configuration
    rng = np.random.default_rng(11)
    n = 512
    idx = np.concatenate([rng.choice(n ** 3, 24, replace=False),
                          np.array([0, n ** 3 - 1, (n // 2) * n * n + (n // 2) * n + n // 2])])
    ref = oracle_mod.sample_direct(rho32.astype(np.float64), idx)
    got = out.reshape(-1)[idx]
    scale = np.abs(ref).max()
    assert np.abs(got - ref).max() <= 1e-5 * scale, np.abs(got - ref).max() / scale
    # linearity of the ball excess: Phi(field) - Phi(field - ball) = Phi(ball)
    # and the ball's potential matches the closed form inside it
    base = gpu_solve(pg, (rho - sphere).astype(np.float32))
    ball = out - base
    c = (n - 1) / 2.0
    z, y, x = np.meshgrid(np.arange(n) - c, np.arange(n) - c, np.arange(n) - c, indexing="ij")
    r = np.sqrt(x * x + y * y + z * z)
    inside = r < 20.0
    exact = -2.0 * math.pi * (40.0 ** 2 - r[inside] ** 2 / 3.0)
    assert np.abs(ball[inside] - exact).max() < 2e-2 * np.abs(exact).max()


# ---------------------------------------------------------------------------
# adjoint, host path, passes
# ---------------------------------------------------------------------------

def test_adjoint_identity_and_oracle_gradient(pg, oracle_mod):
    shape = (32, 48, 16)
    rng = np.random.default_rng(8)
    rho = rng.standard_normal(shape)
    w = workloads.random_weights(shape, seed=9)
    with pg.Plan(16, 48, 32, h=(1.0, 0.5, 2.0), precision="fp64") as plan:
        r = torch.from_numpy(rho).cuda()
        ww = torch.from_numpy(w).cuda()
        phi = plan.solve(r)
        g = plan.adjoint(ww)
        lhs = float((ww * phi).sum())
        rhs = float((g * r).sum())
        assert lhs == pytest.approx(rhs, rel=1e-12)
        ref = oracle_mod.solve_adjoint_direct(w, h=(1.0, 0.5, 2.0))
        l2, mx = rel_errors(g.cpu().numpy(), ref)
        assert l2 <= TOL64[0] and mx <= TOL64[1]


def test_autograd_matches_finite_differences_32cube(pg, oracle_mod):
    n = 32
    rho = torch.from_numpy(workloads.gaussian_blobs(n, seed=4)[0]).cuda().requires_grad_(True)
    w = torch.from_numpy(workloads.random_weights(n, seed=5)).cuda()
    with pg.Plan(n, precision="fp64") as plan:
        phi = pg.PoissonSolve.apply(rho, plan)
        loss = (w * phi).sum()
        loss.backward()
        grad = rho.grad.detach().cpu().numpy()
        # L is linear in rho: central differences along random directions
        rng = np.random.default_rng(6)
        for _ in range(3):
            v = torch.from_numpy(rng.standard_normal((n, n, n))).cuda()
            eps = 1e-3
            lp = float((w * plan.solve((rho.detach() + eps * v).contiguous())).sum())
            lm = float((w * plan.solve((rho.detach() - eps * v).contiguous())).sum())
            fd = (lp - lm) / (2 * eps)
            assert fd == pytest.approx(float((rho.grad * v).sum()), rel=1e-9)
    ref = oracle_mod.solve_adjoint_direct(w.cpu().numpy())
    l2, mx = rel_errors(grad, ref)
    assert l2 <= TOL64[0] and mx <= TOL64[1]


def test_fp32_adjoint_equals_oracle_gradient(pg, oracle_mod):
    shape = (48, 32, 64)
    w = workloads.random_weights(shape, seed=12).astype(np.float32)
    with pg.Plan(64, 32, 48) as plan:
        g = plan.adjoint(torch.from_numpy(w).cuda()).double().cpu().numpy()
    ref = oracle_mod.solve_fft(w.astype(np.float64))
    l2, mx = rel_errors(g, ref)
    assert l2 <= TOL32[0] and mx <= TOL32[1]


def test_host_path_and_passes_match_device_solve(pg):
    shape = (64, 32, 48)
    rho = np.random.default_rng(1).standard_normal(shape).astype(np.float32)
    with pg.Plan(48, 32, 64) as plan:
        x = torch.from_numpy(rho).cuda()
        dev = plan.solve(x).cpu().numpy()
        host = plan.solve_host(torch.from_numpy(rho).pin_memory()).numpy()
        assert np.array_equal(dev, host)
        y = torch.empty_like(x)
        for i in range(5):
            plan.solve_pass(i, x, y)
        torch.cuda.synchronize()
        assert np.array_equal(dev, y.cpu().numpy())
        # in place (rho and phi may alias)
        z = x.clone()
        plan.solve(z, out=z)
        torch.cuda.synchronize()
        assert np.array_equal(dev, z.cpu().numpy())


def test_repeat_solves_are_deterministic(pg):
    rho = torch.from_numpy(np.random.default_rng(2).standard_normal((64, 64, 64)).astype(np.float32)).cuda()
    with pg.Plan(64) as plan:
        a = plan.solve(rho).cpu()
        b = plan.solve(rho).cpu()
    assert torch.equal(a, b)


def test_bad_arguments_on_device(pg):
    with pg.Plan(32) as plan:
        x = torch.zeros((32, 32, 32), device="cuda")
        with pytest.raises(ValueError):
            plan.solve(torch.zeros((32, 32, 16), device="cuda"))
        with pytest.raises(pg.PoissonError):
            plan.solve_pass(7, x, x)
        # misaligned pointer is rejected with POISSON_ERR_ARG
        flat = torch.zeros(32 ** 3 + 1, device="cuda")
        import ctypes
        st = plan.solve_pass  # noqa: F841
        rc = pg.lib().poisson_solve(plan.handle, ctypes.c_void_p(flat.data_ptr() + 4),
                                    ctypes.c_void_p(x.data_ptr()), None)
        assert rc == 1


# ---------------------------------------------------------------------------
# kernel variants and the autotuner
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("shape", [(16, 16, 16), (48, 32, 96), (64, 128, 192), (16, 256, 48),
                                   (32, 16, 384), (512, 16, 32), (16, 512, 16), (16, 32, 512)])
def test_every_kernel_variant_matches_oracle(pg, oracle_mod, shape):
    nz, ny, nx = shape
    rng = np.random.default_rng(sum(shape) + 1)
    rho = rng.standard_normal(shape).astype(np.float32)
    h = (1.0, 0.75, 1.25)
    ref = oracle_mod.solve_fft(rho.astype(np.float64), h=h)
    x = torch.from_numpy(rho).cuda()
    with pg.Plan(nx, ny, nz, h=h) as plan:
        counts = plan.info()["variant_count"]
        for v in range(max(counts)):
            for pss in range(5):
                plan.set_variant(pss, min(v, counts[pss] - 1))
            out = plan.solve(x).double().cpu().numpy()
            l2, mx = rel_errors(out, ref)
            assert l2 <= TOL32[0] and mx <= TOL32[1], (v, l2, mx)


@pytest.mark.parametrize("shape", [(16, 16, 16), (48, 32, 96), (32, 16, 384), (16, 512, 16), (512, 16, 32),
                                   (96, 192, 64)])
def test_unfused_plain_pipeline_matches_oracle(pg, oracle_mod, shape):
    # the yardstick pipeline (padded grid materialised, full length-2n FFTs
    # of 32 .. 1024 points along each axis, separate multiply and crop)
    nz, ny, nx = shape
    rho = np.random.default_rng(sum(shape) + 7).standard_normal(shape).astype(np.float32)
    h = (1.0, 0.75, 1.25)
    ref = oracle_mod.solve_fft(rho.astype(np.float64), h=h)
    x = torch.from_numpy(rho).cuda()
    with pg.Plan(nx, ny, nz, h=h) as plan:
        for _ in range(2):  # the first call allocates, the second reuses
            out = plan.solve_unfused(x).double().cpu().numpy()
            l2, mx = rel_errors(out, ref)
            assert l2 <= TOL32[0] and mx <= TOL32[1], (shape, l2, mx)
    with pg.Plan(16, precision="fp64") as plan:
        with pytest.raises(pg.PoissonError):
            plan.solve_unfused(torch.zeros((16, 16, 16), dtype=torch.float64, device="cuda"))


def test_autotuned_plan_matches_oracle(pg, oracle_mod):
    shape = (64, 96, 128)
    rho = np.random.default_rng(9).standard_normal(shape).astype(np.float32)
    ref = oracle_mod.solve_fft(rho.astype(np.float64))
    with pg.Plan(128, 96, 64, flags=pg.abi.FLAG_AUTOTUNE) as plan:
        info = plan.info()
        assert all(0 <= v < c for v, c in zip(info["variant"], info["variant_count"]))
        out = plan.solve(torch.from_numpy(rho).cuda()).double().cpu().numpy()
        plan.autotune()
        out2 = plan.solve(torch.from_numpy(rho).cuda()).double().cpu().numpy()
    for o in (out, out2):
        l2, mx = rel_errors(o, ref)
        assert l2 <= TOL32[0] and mx <= TOL32[1]


# ---------------------------------------------------------------------------
# fused single-field dataflow kernel
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("n", [64, 128, 192, 256])
def test_fused_dataflow_solve_matches_oracle(pg, oracle_mod, n):
    rho = np.random.default_rng(n).standard_normal((n, n, n)).astype(np.float32)
    ref = oracle_mod.solve_fft(rho.astype(np.float64))
    x = torch.from_numpy(rho).cuda()
    with pg.Plan(n) as plan:
        five = plan.solve(x).double().cpu().numpy()
        for mode in (1, 2):
            plan.set_variant(5, mode)
            assert plan.info()["fused"] == mode
            for _ in range(2):  # repeated launches reuse the counters
                out = plan.solve(x).double().cpu().numpy()
                l2, mx = rel_errors(out, ref)
                assert l2 <= TOL32[0] and mx <= TOL32[1], (mode, l2, mx)
            assert plan.sync_status() == 0
        assert np.abs(out - five).max() <= 1e-6 * np.abs(five).max()


def test_fused_dataflow_solve_at_512_equals_the_five_pass_solve(pg):
    # 512 is the edge whose row tiles (x passes) use a different line
    # configuration from its column tiles
    n = 512
    x = torch.from_numpy(np.random.default_rng(n).standard_normal((n, n, n)).astype(np.float32)).cuda()
    with pg.Plan(n) as plan:
        five = plan.solve(x)
        for mode in (1, 2):
            plan.set_variant(5, mode)
            out = plan.solve(x)
            assert plan.sync_status() == 0
            assert ((out - five).abs().max() <= 1e-6 * five.abs().max()).item(), mode


def test_fused_mode_rejected_for_unsupported_shapes(pg):
    with pg.Plan(64, 32, 32) as plan:
        with pytest.raises(pg.PoissonError):
            plan.set_variant(5, 1)


@pytest.mark.parametrize("shape", [(64, 64, 64), (48, 96, 192), (256, 256, 256), (32, 64, 512)])
@pytest.mark.parametrize("mode", [3, 4])
def test_banded_execution_matches_oracle(pg, oracle_mod, shape, mode):
    nz, ny, nx = shape
    rho = np.random.default_rng(sum(shape) + mode).standard_normal(shape).astype(np.float32)
    ref = oracle_mod.solve_fft(rho.astype(np.float64))
    x = torch.from_numpy(rho).cuda()
    with pg.Plan(nx, ny, nz) as plan:
        counts = plan.info()["variant_count"]
        # band ranges follow each pass's tile width; the last two column
        # variants are the persistent TMA kernels, which take band ranges too
        for v in (0, 2, 4, counts[1] - 2, counts[1] - 1):
            for pss in range(5):
                plan.set_variant(pss, min(v, counts[pss] - 1))
            plan.set_variant(5, mode)
            for _ in range(2):
                out = plan.solve(x).double().cpu().numpy()
                l2, mx = rel_errors(out, ref)
                assert l2 <= TOL32[0] and mx <= TOL32[1], (v, l2, mx)


def test_launch_count_follows_configuration(pg):
    with pg.Plan(64, 64, 64) as plan:
        counts = plan.info()["variant_count"]
        for pss in range(5):
            plan.set_variant(pss, 0)
        plan.set_variant(5, 0)
        assert plan.launch_count() == 5
        # persistent TMA column kernels add one plain launch for the Nyquist
        # column (kx = nx) of each column pass
        for pss in (1, 2, 3):
            plan.set_variant(pss, counts[pss] - 1)
        assert plan.launch_count() == 8
        plan.set_variant(5, 1)  # fused dataflow kernel
        assert plan.launch_count() == 1


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_check_finite_flag_reports_non_finite_output(pg, precision):
    dt = torch.float32 if precision == "fp32" else torch.float64
    rho = torch.zeros((32, 32, 48), device="cuda", dtype=dt)
    rho[3, 4, 5] = float("nan")
    with pg.Plan(48, 32, 32, precision=precision, flags=pg.abi.FLAG_CHECK_FINITE) as plan:
        for v in range(plan.info()["variant_count"][4]):  # staged and direct x inverse
            plan.set_variant(4, v)
            plan.solve(rho)
            assert plan.sync_status() == 6  # POISSON_ERR_NUMERIC
            plan.solve(torch.ones_like(rho))
            assert plan.sync_status() == 0
    with pg.Plan(48, 32, 32, precision=precision) as plan:  # without the flag nothing is checked
        plan.solve(rho)
        assert plan.sync_status() == 0


def test_autotune_result_is_reused_for_the_same_shape(pg, oracle_mod):
    import time
    shape = (32, 48, 96)
    rho = np.random.default_rng(21).standard_normal(shape).astype(np.float32)
    ref = oracle_mod.solve_fft(rho.astype(np.float64))
    t0 = time.perf_counter()
    with pg.Plan(96, 48, 32, flags=pg.abi.FLAG_AUTOTUNE) as a:
        t_first = time.perf_counter() - t0
        t0 = time.perf_counter()
        with pg.Plan(96, 48, 32, flags=pg.abi.FLAG_AUTOTUNE) as b:
            t_second = time.perf_counter() - t0
            ia, ib = a.info(), b.info()
            assert ia["variant"] == ib["variant"] and ia["fused"] == ib["fused"]
            out = b.solve(torch.from_numpy(rho).cuda()).double().cpu().numpy()
    assert t_second < t_first  # the second plan took the recorded result
    l2, mx = rel_errors(out, ref)
    assert l2 <= TOL32[0] and mx <= TOL32[1]


@pytest.mark.parametrize("from_last", [3, 2])
def test_tma_column_kernel_wait_timeout_is_reported(pg, oracle_mod, monkeypatch, from_last):
    # Test hook: the persistent TMA kernel skips its first copy, so the bounded
    # mbarrier wait (about a second) runs out; the kernel records a timeout in
    # the status word and returns, and the GPU stays usable.  from_last = 3:
    # the single-buffered variant, 2: the first double-buffered one.
    shape = (32, 32, 32)
    rho = np.random.default_rng(31).standard_normal(shape).astype(np.float32)
    x = torch.from_numpy(rho).cuda()
    with pg.Plan(32) as plan:
        tma = plan.info()["variant_count"][2] - from_last  # a persistent TMA column variant
        plan.set_variant(2, tma)
        monkeypatch.setenv("POISSON_TEST_TMA_HOLD", "1")
        plan.solve(x)
        assert plan.sync_status() == 5  # POISSON_ERR_TIMEOUT
        monkeypatch.delenv("POISSON_TEST_TMA_HOLD")
        out = plan.solve(x).double().cpu().numpy()
        assert plan.sync_status() == 0
    ref = oracle_mod.solve_fft(rho.astype(np.float64))
    assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-6


def test_autograd_with_a_batch_dimension(pg):
    rng = np.random.default_rng(41)
    rho = torch.from_numpy(rng.standard_normal((3, 16, 32, 48)).astype(np.float32)).cuda().requires_grad_()
    w = torch.from_numpy(rng.standard_normal((3, 16, 32, 48)).astype(np.float32)).cuda()
    with pg.Plan(48, 32, 16) as plan:
        phi = pg.PoissonSolve.apply(rho, plan)
        (w * phi).sum().backward()
        for b in range(3):
            assert torch.equal(phi[b], plan.solve(rho[b].detach().contiguous()))
            assert torch.equal(rho.grad[b], plan.adjoint(w[b].contiguous()))


def test_fp64_solve_matches_the_golden_fixture(pg):
    # the stored direct pair sums (tests/golden, written by the oracle)
    import importlib.util
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "make_golden.py")
    spec = importlib.util.spec_from_file_location("make_golden", path)
    mg = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mg)
    data = np.loadtxt(mg.OUT, comments="#")
    idx, want = data[:, 0].astype(np.int64), data[:, 4]
    nz, ny, nx = mg.SHAPE
    with pg.Plan(nx, ny, nz, h=mg.H, precision="fp64") as plan:
        out = plan.solve(torch.from_numpy(mg.density()).cuda()).cpu().numpy().ravel()
    assert np.abs(out[idx] - want).max() <= 1e-11 * np.abs(want).max()


def _prism_potential(x, y, z, a, b, c):
    """Integral of 1/|p - r| over the box [0,a] x [0,b] x [0,c] at points
    p = (x, y, z) (the potential of a homogeneous rectangular prism of unit
    density: the 8-corner sum of the classical antiderivative)."""
    def F(u, v, w):
        r = np.sqrt(u * u + v * v + w * w)
        with np.errstate(divide="ignore", invalid="ignore"):
            t = (v * w * np.log(u + r) + w * u * np.log(v + r) + u * v * np.log(w + r)
                 - 0.5 * u * u * np.arctan(v * w / (u * r)) - 0.5 * v * v * np.arctan(w * u / (v * r))
                 - 0.5 * w * w * np.arctan(u * v / (w * r)))
        return t
    # upper limits (a - x, ...) with sign +, lower limits (-x, ...) with sign -
    tot = 0.0
    for i, u in ((0, a - x), (1, -x)):
        for j, v in ((0, b - y), (1, -y)):
            for k, w in ((0, c - z), (1, -z)):
                tot = tot + (-1) ** (i + j + k) * F(u, v, w)
    return tot


@pytest.mark.parametrize("shape,h", [((32, 32, 32), (1.0, 1.0, 1.0)), ((32, 48, 64), (1.0, 0.75, 0.5))])
def test_uniform_density_over_the_whole_grid_is_the_prism_potential(pg, shape, h):
    # r_near >= n: every cell pair uses the exact cell average, so Phi at a
    # cell centre is -G rho0 times the integral of 1/r over the whole box
    nz, ny, nx = shape
    rho0, G = 1.5, 0.8
    rho = np.full(shape, rho0, dtype=np.float32)
    with pg.Plan(nx, ny, nz, h=h, G=G, r_near=max(shape)) as plan:
        out = plan.solve(torch.from_numpy(rho).cuda()).double().cpu().numpy()
    rng = np.random.default_rng(5)
    pts = [(0, 0, 0), (nz - 1, ny - 1, nx - 1), (nz // 2, ny // 2, nx // 2)] + \
        [tuple(int(rng.integers(0, s)) for s in shape) for _ in range(20)]
    hx, hy, hz = h
    for iz, iy, ix in pts:
        want = -G * rho0 * _prism_potential((ix + 0.5) * hx, (iy + 0.5) * hy, (iz + 0.5) * hz,
                                            nx * hx, ny * hy, nz * hz)
        assert abs(out[iz, iy, ix] - want) <= 2e-6 * abs(want), ((iz, iy, ix), out[iz, iy, ix], want)


def test_reflection_and_translation_at_size(pg):
    # the kernel is even: flipping rho along an axis flips Phi; the
    # free-space convolution is translation covariant: shifting a density
    # whose support stays inside the grid shifts Phi on the overlap
    shape = (64, 96, 128)
    nz, ny, nx = shape
    rho = np.zeros(shape, dtype=np.float32)
    inner, _ = workloads.gaussian_blobs((32, 48, 64), count=5, seed=23)
    rho[16:48, 24:72, 32:96] = inner.astype(np.float32)
    s = (3, -5, 7)
    shifted = np.roll(rho, s, axis=(0, 1, 2))  # support stays inside: nothing wraps
    with pg.Plan(nx, ny, nz) as plan:
        def solve(a):
            return plan.solve(torch.from_numpy(np.ascontiguousarray(a)).cuda()).double().cpu().numpy()
        base = solve(rho)
        scale = np.abs(base).max()
        for ax in range(3):
            assert np.abs(solve(np.flip(rho, ax)) - np.flip(base, ax)).max() <= 2e-6 * scale
        moved = solve(shifted)
    z0, y0, x0 = max(s[0], 0), max(s[1], 0), max(s[2], 0)
    z1, y1, x1 = nz + min(s[0], 0), ny + min(s[1], 0), nx + min(s[2], 0)
    a = moved[z0:z1, y0:y1, x0:x1]
    b = base[z0 - s[0]:z1 - s[0], y0 - s[1]:y1 - s[1], x0 - s[2]:x1 - s[2]]
    assert np.abs(a - b).max() <= 2e-6 * scale
