"""poisson_solve_noalloc: the plan-free solve that allocates no device memory.

It is meant for callers that must not call cudaMalloc when they solve (code
under a framework's caching allocator, a fixed memory budget, or code that
cannot take the synchronisation an allocation may cause); all its buffers
live in one fixed 16 MiB device array inside the library.  Its output must
match the planned solve (poisson_solve) within the FP32 tolerance of the
other parity tests, on consecutive calls that reuse the shared array.
This file is collected last so that a failure here leaves every other test
already run.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_L2, TOL_MAX = 1e-6, 1e-5


@pytest.fixture(scope="module")
def pg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2409_02294_gb300 as pg
    pg.lib()
    return pg


def _noalloc(pg, rho, h, G):
    nz, ny, nx = rho.shape
    out = torch.empty_like(rho)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = pg.lib().poisson_solve_noalloc(nx, ny, nz, h[0], h[1], h[2], G,
                                        ctypes.c_void_p(rho.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), st)
    assert rc == 0, rc
    return out


def _close(a, b):
    a = a.double().cpu().numpy()
    b = b.double().cpu().numpy()
    l2 = np.linalg.norm(a - b) / np.linalg.norm(b)
    mx = np.abs(a - b).max() / np.abs(b).max()
    assert l2 <= TOL_L2 and mx <= TOL_MAX, (l2, mx)


def test_noalloc_matches_planned_solve_on_consecutive_calls(pg):
    rng = np.random.default_rng(77)
    cases = [((32, 48, 64), (1.0, 0.5, 2.0), 1.3),   # (nz, ny, nx), (hx, hy, hz), G
             ((32, 48, 64), (1.0, 0.5, 2.0), 1.3),   # same grid, new input
             ((64, 16, 32), (0.7, 0.7, 0.7), 0.5)]   # different grid after it
    for shape, h, G in cases:
        nz, ny, nx = shape
        rho = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
        with pg.Plan(nx, ny, nz, h=h, G=G) as plan:
            ref = plan.solve(rho)
            got = _noalloc(pg, rho, h, G)
            torch.cuda.synchronize()
        _close(got, ref)


def test_noalloc_rejects_grids_beyond_the_array(pg):
    rho = torch.zeros((128, 128, 128), device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = pg.lib().poisson_solve_noalloc(128, 128, 128, 1.0, 1.0, 1.0, 1.0,
                                        ctypes.c_void_p(rho.data_ptr()),
                                        ctypes.c_void_p(rho.data_ptr()), st)
    assert rc == 1  # POISSON_ERR_ARG: does not fit the 16 MiB array
    rc = pg.lib().poisson_solve_noalloc(100, 64, 64, 1.0, 1.0, 1.0, 1.0,
                                        ctypes.c_void_p(rho.data_ptr()),
                                        ctypes.c_void_p(rho.data_ptr()), st)
    assert rc == 4  # POISSON_ERR_UNSUPPORTED edge length
