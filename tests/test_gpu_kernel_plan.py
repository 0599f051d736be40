"""Plans for a caller-supplied even kernel (poisson_plan_create_kernel):
parity with the oracle's kernel convolution, closed forms, and agreement
with the Green's-function plan when given the Green's kernel."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = (1e-6, 1e-5)


@pytest.fixture(scope="module")
def pg():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_2409_02294_gb300 as pg
    pg.lib()
    return pg


def _rel(a, b):
    return (np.linalg.norm(a - b) / np.linalg.norm(b), np.abs(a - b).max() / np.abs(b).max())


def _yukawa_octant(nz, ny, nx, lam=6.0):
    """exp(-r/lam)/r with a finite self value: a screened potential."""
    dz, dy, dx = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    r = np.sqrt(dx ** 2 + dy ** 2 + dz ** 2.0)
    r[0, 0, 0] = 0.5
    return np.exp(-r / lam) / r


@pytest.mark.parametrize("shape", [(32, 48, 64), (96, 16, 48), (64, 64, 64)])
def test_screened_kernel_matches_oracle(pg, oracle_mod, shape):
    nz, ny, nx = shape
    k = _yukawa_octant(nz, ny, nx)
    rho = np.random.default_rng(sum(shape)).standard_normal(shape).astype(np.float32)
    ref = oracle_mod.solve_fft_kernel(rho.astype(np.float64), k, -0.3)
    with pg.Plan.from_kernel(k, scale=-0.3) as plan:
        x = torch.from_numpy(rho).cuda()
        out = plan.solve(x).double().cpu().numpy()
        adj = plan.adjoint(x).double().cpu().numpy()
    l2, mx = _rel(out, ref)
    assert l2 <= TOL32[0] and mx <= TOL32[1], (l2, mx)
    assert np.array_equal(out, adj)  # even kernel: the adjoint is the same solve


def test_delta_kernel_is_a_scaled_copy(pg):
    k = np.zeros((33, 17, 49))
    k[0, 0, 0] = 1.0
    rho = np.random.default_rng(3).standard_normal((32, 16, 48)).astype(np.float32)
    with pg.Plan.from_kernel(k, scale=2.0) as plan:
        out = plan.solve(torch.from_numpy(rho).cuda()).double().cpu().numpy()
    l2, mx = _rel(out, 2.0 * rho.astype(np.float64))
    assert l2 <= 1e-6 and mx <= 1e-5


def test_greens_octant_reproduces_the_poisson_plan(pg, oracle_mod):
    shape = (16, 32, 48)
    nz, ny, nx = shape
    h = (1.0, 0.75, 1.25)
    koct = oracle_mod.kernel_octant((nx + 1, ny + 1, nz + 1), h=h)
    rho = np.random.default_rng(5).standard_normal(shape)
    x = torch.from_numpy(rho).cuda()
    with pg.Plan.from_kernel(koct, scale=-h[0] * h[1] * h[2], precision="fp64") as a, \
            pg.Plan(nx, ny, nz, h=h, precision="fp64") as b:
        oa = a.solve(x).cpu().numpy()
        ob = b.solve(x).cpu().numpy()
    assert np.abs(oa - ob).max() <= 1e-12 * np.abs(ob).max()
    ref = oracle_mod.solve_direct(rho, h=h)
    assert np.linalg.norm(oa - ref) / np.linalg.norm(ref) <= 1e-12


def test_kernel_plan_rejects_bad_input(pg):
    k = np.ones((17, 17, 17))
    k[3, 2, 1] = np.nan
    with pytest.raises(pg.PoissonError):
        pg.Plan.from_kernel(k)
    with pytest.raises(pg.PoissonError):
        pg.Plan.from_kernel(np.ones((18, 17, 17)))  # edge 17 is not a supported size
    with pytest.raises(pg.PoissonError):
        pg.Plan.from_kernel(np.ones((17, 17, 17)), scale=float("inf"))
