"""Full-size parity: the benchmark workloads solved in the benchmark's launch
configuration and compared with the FP64 oracle element by element.

* 512^3 lognormal field + ball (autotuned FP32 plan) against the oracle's
  full-field FFT convolution: rel-L2 <= 1e-6, max-norm <= 1e-5 max|Phi|.
* every field of the 96-field uneven batch, in the execution mode the first
  batched call picks and in the persistent-kernel mode, against the oracle.
* one full 384^3 Plummer field per precision (FP32, FP16 hi+lo, BF16 hi+lo)
  against the oracle's full field.

The FP32 input is what the oracle sees (FP32 rounding of the density is not
counted as solver error).
"""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = (1e-6, 1e-5)
# rel-L2 and max-norm bars of the compensated tensor-core forms (see the
# tensor-core test module for how they follow from the arithmetic)
TOL_TC = {"tc_fp16x2": (1e-6, 1e-5), "tc_bf16x2": (2e-6, 5e-6)}


@pytest.fixture(scope="module")
def pg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2409_02294_gb300 as pg
    pg.lib()
    return pg


def _rel(out, ref):
    out = np.asarray(out, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return (float(np.linalg.norm(out - ref) / np.linalg.norm(ref)),
            float(np.abs(out - ref).max() / np.abs(ref).max()))


def test_fp32_512cube_lognormal_full_field(pg, oracle_mod):
    rho, _ = workloads.lognormal_field(512, seed=2409)
    rho32 = rho.astype(np.float32)
    del rho
    with pg.Plan(512, flags=pg.abi.FLAG_AUTOTUNE) as plan:  # the benchmark's launch configuration
        x = torch.from_numpy(rho32).cuda()
        out = plan.solve(x).cpu().numpy()
        del x
        torch.cuda.synchronize()
    ref = oracle_mod.solve_fft(rho32.astype(np.float64))
    l2, mx = _rel(out, ref)
    assert l2 <= TOL32[0] and mx <= TOL32[1], (l2, mx)


@pytest.fixture(scope="module")
def batch96(pg, oracle_mod):
    shapes = workloads.batch_shapes(96, seed=2409)
    dens = workloads.batch_densities(shapes, seed=2409)
    refs = [oracle_mod.solve_fft(d.astype(np.float64)) for d in dens]
    return shapes, dens, refs


@pytest.mark.parametrize("mode", ["chosen", "0"])
def test_batch96_every_field_vs_oracle(pg, batch96, mode, monkeypatch):
    shapes, dens, refs = batch96
    monkeypatch.delenv("POISSON_BATCH_MODE", raising=False)
    plans = [pg.Plan(s[2], s[1], s[0], flags=pg.abi.FLAG_AUTOTUNE) for s in shapes]
    try:
        rhos = [torch.from_numpy(d).cuda() for d in dens]
        phis = [torch.empty_like(r) for r in rhos]
        pg.solve_batched(plans, rhos, phis)  # the first call picks the mode
        if mode != "chosen":
            pg.batch_mode(plans, int(mode))
            for p in phis:
                p.fill_(float("nan"))
            pg.solve_batched(plans, rhos, phis)
        torch.cuda.synchronize()
        assert plans[0].sync_status() == 0
        for s, o, ref in zip(shapes, phis, refs):
            l2, mx = _rel(o.double().cpu().numpy(), ref)
            assert l2 <= TOL32[0] and mx <= TOL32[1], (s, l2, mx)
    finally:
        for p in plans:
            p.close()


@pytest.fixture(scope="module")
def plummer384(oracle_mod):
    rho, _ = workloads.plummer_spheres(384, count=16, seed=2409)
    rho32 = rho.astype(np.float32)
    return rho32, oracle_mod.solve_fft(rho32.astype(np.float64))


@pytest.mark.parametrize("prec", ["fp32", "tc_fp16x2", "tc_bf16x2"])
def test_384cube_plummer_full_field_every_precision(pg, plummer384, prec):
    rho32, ref = plummer384
    with pg.Plan(384, precision=prec, flags=pg.abi.FLAG_AUTOTUNE) as plan:
        out = plan.solve(torch.from_numpy(rho32).cuda()).double().cpu().numpy()
    l2, mx = _rel(out, ref)
    tol = TOL32 if prec == "fp32" else TOL_TC[prec]
    assert l2 <= tol[0] and mx <= tol[1], (prec, l2, mx)
