"""poisson_solve_noalloc: the plan-free solve that allocates no device memory.

It is meant for callers that must not call cudaMalloc when they solve (code
under a framework's caching allocator, a fixed memory budget, or code that
cannot take the synchronisation an allocation may cause); all its buffers
live in one fixed 16 MiB device array inside the library.  Its output must
match the planned solve (poisson_solve) and the FP64 oracle within the FP32
tolerance of the other parity tests, on consecutive calls that reuse the
shared array, and a run of calls must leave the device's free memory and
torch's allocator untouched.  This file is collected last so that a failure
here leaves every other test already run.
"""
import ctypes

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL_L2, TOL_MAX = 1e-6, 1e-5
ERR_ARG, ERR_UNSUPPORTED = 1, 4


@pytest.fixture(scope="module")
def pg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2409_02294_gb300 as pg
    pg.lib()
    return pg


def _call(pg, nx, ny, nz, h, G, rho_ptr, out_ptr):
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return pg.lib().poisson_solve_noalloc(nx, ny, nz, h[0], h[1], h[2], G, ctypes.c_void_p(rho_ptr),
                                          ctypes.c_void_p(out_ptr), st)


def _noalloc(pg, rho, h, G, out=None):
    nz, ny, nx = rho.shape
    out = torch.empty_like(rho) if out is None else out
    rc = _call(pg, nx, ny, nz, h, G, rho.data_ptr(), out.data_ptr())
    assert rc == 0, rc
    return out


def _close(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    l2 = np.linalg.norm(a - b) / np.linalg.norm(b)
    mx = np.abs(a - b).max() / np.abs(b).max()
    assert l2 <= TOL_L2 and mx <= TOL_MAX, (l2, mx)


@pytest.mark.parametrize("shape,h,G", [
    ((32, 48, 64), (1.0, 0.5, 2.0), 1.3),   # (nz, ny, nx), (hx, hy, hz), G
    ((96, 64, 64), (1.0, 1.0, 1.0), 1.0),   # radix-3 edge along z
    ((64, 64, 128), (0.5, 1.0, 1.0), 2.0),  # nx = 128, ny = nz = 64: the long-x shape that fits
])
def test_noalloc_matches_planned_solve_and_oracle_on_consecutive_calls(pg, shape, h, G):
    rng = np.random.default_rng(77 + shape[0])
    nz, ny, nx = shape
    with pg.Plan(nx, ny, nz, h=h, G=G) as plan:
        for _ in range(2):  # two calls in a row on the shared array, new input each time
            rho_h = rng.standard_normal(shape).astype(np.float32)
            rho = torch.from_numpy(rho_h).cuda()
            ref = plan.solve(rho)
            got = _noalloc(pg, rho, h, G)
            torch.cuda.synchronize()
            got_h = got.double().cpu().numpy()
            _close(got_h, ref.double().cpu().numpy())
            _close(got_h, oracle.solve_fft(rho_h.astype(np.float64), h=h, G=G))


def test_noalloc_allocates_no_device_memory(pg):
    rng = np.random.default_rng(5)
    shape, h, G = (48, 32, 64), (1.0, 1.0, 1.0), 1.0
    rho = torch.from_numpy(rng.standard_normal(shape).astype(np.float32)).cuda()
    out = torch.empty_like(rho)
    _noalloc(pg, rho, h, G, out)  # warm-up: loads the kernels and looks up the array
    first = out.clone()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    stats0 = torch.cuda.memory_stats()
    for _ in range(5):
        _noalloc(pg, rho, h, G, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    stats1 = torch.cuda.memory_stats()
    for key in ("allocation.all.allocated", "segment.all.allocated", "reserved_bytes.all.current"):
        assert stats1.get(key, 0) == stats0.get(key, 0), key
    assert torch.equal(out, first)  # same input, same shared array state: same result


def test_noalloc_rejects_grids_beyond_the_array(pg):
    rho = torch.zeros((128, 128, 128), device="cuda")
    p = rho.data_ptr()
    h = (1.0, 1.0, 1.0)
    assert _call(pg, 128, 128, 128, h, 1.0, p, p) == ERR_ARG     # 128^3 does not fit 16 MiB
    assert _call(pg, 64, 128, 64, h, 1.0, p, p) == ERR_ARG       # ny = 128 does not fit
    assert _call(pg, 64, 64, 128, h, 1.0, p, p) == ERR_ARG       # nz = 128 does not fit
    assert _call(pg, 100, 64, 64, h, 1.0, p, p) == ERR_UNSUPPORTED  # edge length
    assert _call(pg, 64, 64, 64, (0.0, 1.0, 1.0), 1.0, p, p) == ERR_ARG


def test_noalloc_binding_checks_the_output_tensor(pg):
    rho = torch.zeros((32, 32, 32), device="cuda")
    for bad in (torch.empty((32, 32, 16), device="cuda"),
                torch.empty((32, 32, 32), device="cuda", dtype=torch.float16),
                torch.empty((32, 32, 64), device="cuda")[:, :, :32],
                torch.empty((32, 32, 32))):
        with pytest.raises(ValueError):
            pg.solve_noalloc(rho, out=bad)
    out = pg.solve_noalloc(rho)
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0
