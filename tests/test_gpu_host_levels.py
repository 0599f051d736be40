"""Overlapped host-staged solve of several independent fields (the levels of
a nested grid): poisson_solve_host_levels must give exactly the results of
one poisson_solve_host per level, for pinned and pageable host memory and
with a plan that appears more than once."""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2409_02294_gb300 as pg
    pg.lib()
    return pg


@pytest.mark.parametrize("pinned", [True, False])
def test_levels_equal_one_host_solve_per_level(pg, oracle_mod, pinned):
    a, b, c = pg.Plan(64), pg.Plan(128, 64, 64), pg.Plan(32, 32, 32, precision="fp64")
    plans = [a, b, a, c, b]  # repeated plans reuse their staging buffers in order
    try:
        rhos = []
        for i, p in enumerate(plans):
            r = workloads.gaussian_blobs(p.shape, count=5, seed=300 + i)[0].astype(
                np.float64 if p.dtype == torch.float64 else np.float32)
            t = torch.from_numpy(r)
            rhos.append(t.pin_memory() if pinned else t)
        phis = pg.solve_host_levels(plans, rhos)
        for p, r, o in zip(plans, rhos, phis):
            ref = p.solve_host(r)
            assert torch.equal(o, ref)
        ref = oracle_mod.solve_fft(rhos[1].double().numpy())
        out = phis[1].double().numpy()
        assert np.linalg.norm(out - ref) / np.linalg.norm(ref) <= 1e-6
    finally:
        for p in (a, b, c):
            p.close()


def test_levels_reject_bad_arguments(pg):
    with pg.Plan(32) as p:
        x = torch.zeros((32, 32, 32))
        with pytest.raises(ValueError):
            pg.solve_host_levels([p], [x, x])
        with pytest.raises(ValueError):
            pg.solve_host_levels([p], [torch.zeros((16, 32, 32))])
    assert pg.solve_host_levels([], []) == []


def test_one_plan_repeated_alternates_staging(pg):
    # five fields through one plan: occurrences alternate between two staging
    # pairs and reuse each pair after the field two before it
    with pg.Plan(64, 32, 48) as p:
        rhos = [torch.from_numpy(workloads.gaussian_blobs(p.shape, count=4, seed=400 + i)[0]
                                 .astype(np.float32)).pin_memory() for i in range(5)]
        outs = [torch.empty_like(r).pin_memory() for r in rhos]
        pg.solve_host_levels([p] * 5, rhos, outs)
        for r, o in zip(rhos, outs):
            assert torch.equal(o, p.solve_host(r))
