"""Tensor-core precisions (split FP16 / BF16 radix-16 stages in the z pass,
FP32 accumulate) against the FP64 oracle, and their adjoint.

The stated tolerances come from the arithmetic: an FP16 hi+lo operand carries
22 significant bits and the products accumulate in FP32, so the error stays at
the FP32 path's level (rel-L2 <= 1e-6); a BF16 hi+lo operand carries 16 bits
(unit roundoff 2^-17 ~ 7.6e-6 per product, the dropped lo*lo term ~2^-16),
and one radix-16 stage of each z transform runs at that precision, so
rel-L2 <= 1e-5 and max-norm <= 2e-5 max|Phi| (measured on these fields: at
most 3.5e-6 and 4.5e-6).  Both forms scale each group by a power of two
before the split, so the bars hold for fields scaled by 1e-30 and 1e30.
"""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"tc_fp16x2": (1e-6, 1e-5), "tc_bf16x2": (1e-5, 2e-5)}


@pytest.fixture(scope="module")
def pg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2409_02294_gb300 as pg
    pg.lib()
    return pg


def _rel(out, ref):
    return (np.linalg.norm(out - ref) / np.linalg.norm(ref), np.abs(out - ref).max() / np.abs(ref).max())


@pytest.mark.parametrize("prec", ["tc_fp16x2", "tc_bf16x2"])
@pytest.mark.parametrize("shape", [(128, 32, 48), (256, 16, 32), (384, 32, 16), (512, 16, 16),
                                   (96, 32, 32)])
def test_tensor_core_precisions_vs_oracle(pg, oracle_mod, prec, shape):
    nz, ny, nx = shape
    rho = np.random.default_rng(sum(shape)).standard_normal(shape).astype(np.float32)
    ref = oracle_mod.solve_fft(rho.astype(np.float64), h=(1.0, 0.9, 1.1))
    with pg.Plan(nx, ny, nz, h=(1.0, 0.9, 1.1), precision=prec) as plan:
        out = plan.solve(torch.from_numpy(rho).cuda()).double().cpu().numpy()
    l2, mx = _rel(out, ref)
    assert l2 <= TOL[prec][0] and mx <= TOL[prec][1], (prec, shape, l2, mx)


@pytest.mark.parametrize("prec", ["tc_fp16x2", "tc_bf16x2"])
def test_tensor_core_plummer_and_scale_range(pg, oracle_mod, prec):
    # Plummer densities spanning several decades, and the same field scaled by
    # 1e-30 and 1e30: the per-group power-of-two scaling keeps both forms in range
    rho, _ = workloads.plummer_spheres((128, 64, 64), count=16, seed=7)
    rho = rho.astype(np.float32)
    ref = oracle_mod.solve_fft(rho.astype(np.float64))
    with pg.Plan(64, 64, 128, precision=prec) as plan:
        for f in (1.0, 1e-30, 1e30):
            x = torch.from_numpy((rho * np.float32(f)).astype(np.float32)).cuda()
            out = plan.solve(x).double().cpu().numpy() / f
            l2, mx = _rel(out, ref)
            assert l2 <= TOL[prec][0] and mx <= TOL[prec][1], (f, l2, mx)


@pytest.mark.parametrize("prec", ["fp32", "tc_fp16x2", "tc_bf16x2"])
def test_adjoint_directional_fd_on_subblock(pg, prec):
    # L(rho) = sum(w Phi) is linear, so a central difference along v (supported
    # on a 32^3 sub-block) equals <K^T w, v> up to rounding
    shape = (128, 96, 64)
    rng = np.random.default_rng(21)
    rho = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
    w = torch.from_numpy(workloads.random_weights(shape, seed=22).astype(np.float32)).cuda()
    v = torch.zeros(shape, device="cuda")
    v[40:72, 30:62, 10:42] = torch.from_numpy(rng.standard_normal((32, 32, 32)).astype(np.float32)).cuda()
    with pg.Plan(64, 96, 128, precision=prec) as plan:
        g = plan.adjoint(w)
        lp = float((w.double() * plan.solve((rho + v).contiguous()).double()).sum())
        lm = float((w.double() * plan.solve((rho - v).contiguous()).double()).sum())
        fd = (lp - lm) / 2.0
        an = float((g.double() * v.double()).sum())
    tol = {"fp32": 1e-5, "tc_fp16x2": 1e-5, "tc_bf16x2": 4e-5}[prec]
    assert fd == pytest.approx(an, rel=tol)


@pytest.mark.parametrize("prec", ["tc_fp16x2", "tc_bf16x2"])
def test_tensor_core_384cube_plummer_sampled(pg, oracle_mod, prec):
    # one field of the 8 x 384^3 tensor-core workload at full size, autotuned
    # as in the benchmark, against direct pair sums at sampled cells
    rho, _ = workloads.plummer_spheres(384, count=16, seed=2409)
    rho32 = rho.astype(np.float32)
    with pg.Plan(384, precision=prec, flags=pg.abi.FLAG_AUTOTUNE) as plan:
        out = plan.solve(torch.from_numpy(rho32).cuda()).double().cpu().numpy().reshape(-1)
    n = 384
    rng = np.random.default_rng(19)
    idx = np.concatenate([rng.choice(n ** 3, 20, replace=False),
                          np.array([0, n ** 3 - 1, (n // 2) * n * n + (n // 2) * n + n // 2])])
    ref = oracle_mod.sample_direct(rho32.astype(np.float64), idx)
    err = np.abs(out[idx] - ref).max() / np.abs(ref).max()
    assert err <= TOL[prec][1], (prec, err)
