"""GB300-native free-space Poisson solver: Python binding over libpoisson.

Argument marshalling only.  Every step of a solve runs in the CUDA kernels of
``libpoisson.so`` (built from ``csrc/`` by ``build.py``); PyTorch supplies
device memory and streams.  There is no CPU fallback: if the library cannot
be loaded, importing ``paper_2409_02294_gb300.abi`` raises.

Public entry points mirror the C-ABI of ``include/poisson.h``:

* ``Plan(nx, ny, nz, h=1.0, G=1.0, precision="fp32")`` -
  ``poisson_plan_create``; ``.solve(rho)``, ``.adjoint(w)``,
  ``.solve_host(rho_host)``, ``.solve_pass(i, rho, phi)``,
  ``.solve_unfused(rho)``, ``.greens_octant()``, ``.info()``, ``.close()``
* ``solve_batched(plans, rhos, phis)`` - ``poisson_solve_batched``
* ``solve_host_levels(plans, rhos_host)`` - ``poisson_solve_host_levels``
* ``solve_noalloc(rho, h, G)`` - ``poisson_solve_noalloc`` (no device allocation)
* ``PoissonSolve`` - torch.autograd.Function (forward solve, backward adjoint)
"""
from . import abi  # noqa: F401
from .abi import (  # noqa: F401
    Plan,
    PoissonError,
    batch_mode,
    PoissonSolve,
    lib,
    solve_batched,
    solve_host_levels,
    solve_noalloc,
    supported_size,
)

__all__ = ["Plan", "PoissonError", "PoissonSolve", "batch_mode", "lib", "solve_batched", "solve_host_levels",
           "solve_noalloc", "supported_size"]
