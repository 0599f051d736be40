"""Batched solve: many fields of uneven sizes in one persistent, graph-replayed
launch (poisson_solve_batched), compared with the single-field solve and the
oracle; plus the bounded-wait failure path."""
import os

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(16, 16, 16), (32, 64, 48), (96, 48, 48), (64, 32, 32), (128, 64, 64),
          (16, 192, 96), (384, 16, 16), (16, 16, 512), (48, 96, 192), (256, 32, 16)]


@pytest.fixture(scope="module")
def pg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2409_02294_gb300 as pg
    pg.lib()
    return pg


def _rel(a, b):
    a = a.double().cpu().numpy() if hasattr(a, "cpu") else a
    b = b.double().cpu().numpy() if hasattr(b, "cpu") else b
    return (np.linalg.norm(a - b) / np.linalg.norm(b), np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("mode", ["0", "1", "2", "auto"])
def test_batched_matches_single_solves_and_oracle(pg, oracle_mod, mode, monkeypatch):
    if mode == "auto":
        monkeypatch.delenv("POISSON_BATCH_MODE", raising=False)
    else:
        monkeypatch.setenv("POISSON_BATCH_MODE", mode)
    plans = [pg.Plan(s[2], s[1], s[0], h=(1.0, 0.8, 1.2)) for s in SHAPES]
    try:
        for rep in range(3):  # first call builds the graphs, later ones replay
            rhos = [torch.from_numpy(workloads.gaussian_blobs(s, count=6, seed=10 * rep + i)[0]
                                     .astype(np.float32)).cuda() for i, s in enumerate(SHAPES)]
            phis = [torch.empty_like(r) for r in rhos]
            pg.solve_batched(plans, rhos, phis)
            torch.cuda.synchronize()
            assert plans[0].sync_status() == 0
            chosen = pg.batch_mode(plans)
            assert chosen in (0, 1, 2) and (mode == "auto" or chosen == int(mode))
            for i, (p, r, o) in enumerate(zip(plans, rhos, phis)):
                ref = p.solve(r)
                l2, mx = _rel(o, ref)
                assert l2 <= 1e-6 and mx <= 1e-5, (SHAPES[i], l2, mx)
            for i in (1, 5):
                ref = oracle_mod.solve_fft(rhos[i].double().cpu().numpy(), h=(1.0, 0.8, 1.2))
                l2, mx = _rel(phis[i].double().cpu().numpy(), ref)
                assert l2 <= 1e-6 and mx <= 1e-5
    finally:
        for p in plans:
            p.close()


def test_batch_mode_switch_keeps_results(pg, monkeypatch):
    monkeypatch.delenv("POISSON_BATCH_MODE", raising=False)
    shapes = SHAPES[:4]
    plans = [pg.Plan(s[2], s[1], s[0]) for s in shapes]
    for p in plans:  # non-default variants, so that modes 1 and 2 run different kernels
        for ps, v in ((0, 1), (1, 4), (2, 0), (3, 2), (4, 0)):
            p.set_variant(ps, v)
    try:
        with pytest.raises(pg.PoissonError):
            pg.batch_mode(plans, 0)  # no cached batch for this plan list yet
        assert pg.batch_mode(plans) == -1
        rhos = [torch.randn(s, device="cuda") for s in shapes]
        outs = []
        first = [torch.empty_like(r) for r in rhos]
        pg.solve_batched(plans, rhos, first)  # picks a mode by timing
        torch.cuda.synchronize()
        assert plans[0].sync_status() == 0
        for m in (0, 1, 2):
            phis = [torch.empty_like(r) for r in rhos]
            pg.batch_mode(plans, m)
            pg.solve_batched(plans, rhos, phis)
            torch.cuda.synchronize()
            assert plans[0].sync_status() == 0
            assert pg.batch_mode(plans) == m
            outs.append(phis)
        for other in outs[1:]:
            for a, b in zip(outs[0], other):
                assert _rel(a, b)[0] <= 1e-6
    finally:
        for p in plans:
            p.close()


def test_batched_rejects_mixed_precision_repeated_plans_and_empty(pg):
    with pg.Plan(32) as a, pg.Plan(32, precision="fp64") as b:
        x = torch.zeros((32, 32, 32), device="cuda")
        y = torch.zeros((32, 32, 32), device="cuda", dtype=torch.float64)
        with pytest.raises(pg.PoissonError):
            pg.solve_batched([a, b], [x, y], [torch.empty_like(x), torch.empty_like(y)])
        with pytest.raises(pg.PoissonError):  # one workspace per plan: no repeats
            pg.solve_batched([a, a], [x, x.clone()], [torch.empty_like(x), torch.empty_like(x)])
    pg.solve_batched([], [], [])


def test_batched_bounded_wait_reports_timeout(pg, monkeypatch):
    # Test hook: field 0's second pass waits on a completion count that is
    # never reached; the bounded wait must give up, flag the timeout in the
    # status word, stop the other CTAs and return, leaving the GPU usable.
    plans = [pg.Plan(32), pg.Plan(64, 32, 32)]
    try:
        rhos = [torch.randn(32, 32, 32, device="cuda"), torch.randn(32, 32, 64, device="cuda")]
        phis = [torch.empty_like(r) for r in rhos]
        monkeypatch.setenv("POISSON_TEST_BATCH_HOLD", "1")
        pg.solve_batched(plans, rhos, phis)
        torch.cuda.synchronize()
        assert plans[0].sync_status() == 5  # POISSON_ERR_TIMEOUT
        monkeypatch.delenv("POISSON_TEST_BATCH_HOLD")
        pg.solve_batched(plans, rhos, phis)
        torch.cuda.synchronize()
        assert plans[0].sync_status() == 0
        for p, r, o in zip(plans, rhos, phis):
            l2, mx = _rel(o, p.solve(r))
            assert l2 <= 1e-6
    finally:
        for p in plans:
            p.close()
