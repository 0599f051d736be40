"""ctypes binding to libpoisson.so (names follow include/poisson.h)."""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpoisson.so")

POISSON_OK = 0
STATUS_NAMES = {
    0: "POISSON_OK", 1: "POISSON_ERR_ARG", 2: "POISSON_ERR_ALLOC", 3: "POISSON_ERR_CUDA",
    4: "POISSON_ERR_UNSUPPORTED", 5: "POISSON_ERR_TIMEOUT", 6: "POISSON_ERR_NUMERIC",
}
PRECISIONS = {"fp64": 0, "fp32": 1, "tc_fp16x2": 2, "tc_bf16x2": 3}
FLAG_CHECK_FINITE = 0x1
FLAG_AUTOTUNE = 0x2


class PoissonError(RuntimeError):
    def __init__(self, status, where):
        self.status = int(status)
        super().__init__("%s failed: %s" % (where, STATUS_NAMES.get(int(status), str(status))))


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("mx", ctypes.c_int), ("my", ctypes.c_int), ("mz", ctypes.c_int),
        ("hx", ctypes.c_double), ("hy", ctypes.c_double), ("hz", ctypes.c_double),
        ("G", ctypes.c_double),
        ("precision", ctypes.c_int), ("r_near", ctypes.c_int), ("flags", ctypes.c_uint),
        ("workspace_bytes", ctypes.c_size_t), ("greens_bytes", ctypes.c_size_t),
        ("row_stride", ctypes.c_longlong),
        ("variant", ctypes.c_int * 5), ("variant_count", ctypes.c_int * 5),
        ("fused", ctypes.c_int),
    ]


# (name, restype, argtypes) for every symbol declared in include/poisson.h
_P = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double
_U = ctypes.c_uint
SIGNATURES = [
    ("poisson_plan_create", _I, [ctypes.POINTER(_P), _I, _I, _I, _D, _D, _D, _D, _I, _U, _P]),
    ("poisson_plan_create_ex", _I, [ctypes.POINTER(_P), _I, _I, _I, _D, _D, _D, _D, _I, _U, _I, _P]),
    ("poisson_solve", _I, [_P, _P, _P, _P]),
    ("poisson_solve_adjoint", _I, [_P, _P, _P, _P]),
    ("poisson_solve_batched", _I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _P]),
    ("poisson_solve_host", _I, [_P, _P, _P, _P]),
    ("poisson_plan_launch_count", _I, [_P, ctypes.POINTER(_I)]),
    ("poisson_plan_create_kernel", _I, [ctypes.POINTER(_P), _I, _I, _I, _P, ctypes.c_double, _I, ctypes.c_uint,
                                        _P]),
    ("poisson_solve_host_levels", _I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_P), ctypes.POINTER(_P), _P]),
    ("poisson_batch_get_mode", _I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_I)]),
    ("poisson_batch_set_mode", _I, [ctypes.POINTER(_P), _I, _I]),
    ("poisson_solve_pass", _I, [_P, _I, _P, _P, _P]),
    ("poisson_plan_destroy", _I, [_P]),
    ("poisson_plan_get_info", _I, [_P, ctypes.POINTER(PlanInfo)]),
    ("poisson_plan_autotune", _I, [_P, _P]),
    ("poisson_plan_set_variant", _I, [_P, _I, _I]),
    ("poisson_plan_copy_greens", _I, [_P, ctypes.POINTER(_D), ctypes.c_size_t]),
    ("poisson_plan_sync_status", _I, [_P, _P]),
    ("poisson_solve_noalloc", _I, [_I, _I, _I, _D, _D, _D, _D, _P, _P, _P]),
    ("poisson_solve_unfused", _I, [_P, _P, _P, _P]),
    ("poisson_status_string", ctypes.c_char_p, [_I]),
    ("poisson_supported_size", _I, [_I]),
]

_lock = threading.Lock()
_lib = None


def lib():
    """Load libpoisson.so (building it first if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            from . import build as _build
            path = _build.build()
            if not os.path.exists(path):
                raise ImportError("libpoisson.so is missing and could not be built")
            L = ctypes.CDLL(path)
            for name, res, args in SIGNATURES:
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _lib = L
    return _lib


def _check(status, where):
    if status != POISSON_OK:
        raise PoissonError(status, where)


def supported_size(n):
    return bool(lib().poisson_supported_size(int(n)))


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """A solve plan for an (nz, ny, nx) grid (arrays are indexed [z, y, x])."""

    def __init__(self, nx, ny=None, nz=None, h=1.0, G=1.0, precision="fp32", flags=0,
                 r_near=8, stream=None):
        ny = nx if ny is None else ny
        nz = nx if nz is None else nz
        if np.isscalar(h):
            h = (h, h, h)
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.h = tuple(float(v) for v in h)
        self.G = float(G)
        self.precision = precision
        self._handle = ctypes.c_void_p()
        st = _stream_handle(stream)
        _check(lib().poisson_plan_create_ex(ctypes.byref(self._handle), self.nx, self.ny, self.nz,
                                            self.h[0], self.h[1], self.h[2], self.G,
                                            PRECISIONS[precision], int(flags), int(r_near), st),
               "poisson_plan_create")

    @classmethod
    def from_kernel(cls, k_octant, scale=1.0, precision="fp32", flags=0, stream=None):
        """Plan for Phi = scale * sum_j k(|i - j|) rho[j] with a caller's real,
        per-axis even kernel given on the octant: k_octant[dz, dy, dx] for
        0 <= d <= n (shape (nz+1, ny+1, nx+1)); poisson_plan_create_kernel."""
        k = np.ascontiguousarray(k_octant, dtype=np.float64)
        if k.ndim != 3:
            raise ValueError("k_octant must be 3-D [dz, dy, dx]")
        nz, ny, nx = (int(v) - 1 for v in k.shape)
        self = cls.__new__(cls)
        self.nx, self.ny, self.nz = nx, ny, nz
        self.h = (1.0, 1.0, 1.0)
        self.G = 0.0
        self.precision = precision
        self._handle = ctypes.c_void_p()
        _check(lib().poisson_plan_create_kernel(ctypes.byref(self._handle), nx, ny, nz,
                                                ctypes.c_void_p(k.ctypes.data), float(scale),
                                                PRECISIONS[precision], int(flags), _stream_handle(stream)),
               "poisson_plan_create_kernel")
        return self

    # -- properties ---------------------------------------------------------
    @property
    def handle(self):
        if not self._handle:
            raise RuntimeError("plan is closed")
        return self._handle

    @property
    def shape(self):
        return (self.nz, self.ny, self.nx)

    @property
    def dtype(self):
        torch = _torch()
        return torch.float64 if self.precision == "fp64" else torch.float32

    def info(self):
        inf = PlanInfo()
        _check(lib().poisson_plan_get_info(self.handle, ctypes.byref(inf)), "poisson_plan_get_info")
        out = {f: getattr(inf, f) for f, _ in PlanInfo._fields_}
        out["variant"] = list(inf.variant)
        out["variant_count"] = list(inf.variant_count)
        return out

    def launch_count(self):
        """Kernel launches one solve makes in the current configuration."""
        n = ctypes.c_int(0)
        _check(lib().poisson_plan_launch_count(self.handle, ctypes.byref(n)), "poisson_plan_launch_count")
        return n.value

    def autotune(self, stream=None):
        _check(lib().poisson_plan_autotune(self.handle, _stream_handle(stream)), "poisson_plan_autotune")
        return self.info()["variant"]

    def set_variant(self, pass_id, variant):
        _check(lib().poisson_plan_set_variant(self.handle, int(pass_id), int(variant)),
               "poisson_plan_set_variant")

    # -- solves -------------------------------------------------------------
    def _io(self, x, out):
        torch = _torch()
        if not (isinstance(x, torch.Tensor) and x.is_cuda):
            raise TypeError("expected a CUDA tensor")
        if tuple(x.shape) != self.shape or x.dtype != self.dtype or not x.is_contiguous():
            raise ValueError("expected a contiguous %s tensor of shape %s" % (self.dtype, self.shape))
        if out is None:
            out = torch.empty_like(x)
        elif (tuple(out.shape) != self.shape or out.dtype != self.dtype or not out.is_contiguous()
              or not out.is_cuda or out.device != x.device):
            raise ValueError("bad output tensor")
        return out

    def solve(self, rho, out=None, stream=None):
        out = self._io(rho, out)
        _check(lib().poisson_solve(self.handle, ctypes.c_void_p(rho.data_ptr()),
                                   ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
               "poisson_solve")
        return out

    def adjoint(self, w, out=None, stream=None):
        out = self._io(w, out)
        _check(lib().poisson_solve_adjoint(self.handle, ctypes.c_void_p(w.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
               "poisson_solve_adjoint")
        return out

    def solve_unfused(self, rho, out=None, stream=None):
        """The plain unfused FP32 pipeline (poisson_solve_unfused): padded grid
        materialised, full per-axis FFTs, separate multiply and crop."""
        out = self._io(rho, out)
        _check(lib().poisson_solve_unfused(self.handle, ctypes.c_void_p(rho.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
               "poisson_solve_unfused")
        return out

    def solve_pass(self, pass_id, rho, phi, stream=None):
        rp = ctypes.c_void_p(rho.data_ptr()) if rho is not None else None
        pp = ctypes.c_void_p(phi.data_ptr()) if phi is not None else None
        _check(lib().poisson_solve_pass(self.handle, int(pass_id), rp, pp, _stream_handle(stream)),
               "poisson_solve_pass")

    def solve_host(self, rho_host, phi_host=None, stream=None):
        """End-to-end solve from host memory (numpy array or CPU tensor)."""
        torch = _torch()
        if isinstance(rho_host, np.ndarray):
            rho_host = torch.from_numpy(np.ascontiguousarray(rho_host))
        if phi_host is None:
            phi_host = torch.empty_like(rho_host)
        if tuple(rho_host.shape) != self.shape or rho_host.dtype != self.dtype or rho_host.is_cuda:
            raise ValueError("expected a host %s tensor of shape %s" % (self.dtype, self.shape))
        _check(lib().poisson_solve_host(self.handle, ctypes.c_void_p(rho_host.data_ptr()),
                                        ctypes.c_void_p(phi_host.data_ptr()), _stream_handle(stream)),
               "poisson_solve_host")
        return phi_host

    def greens_octant(self):
        """Transformed Green's function octant [kz, ky, kx] as float64."""
        shp = (self.nz + 1, self.ny + 1, self.nx + 1)
        out = np.empty(shp, dtype=np.float64)
        _check(lib().poisson_plan_copy_greens(self.handle, out.ctypes.data_as(ctypes.POINTER(_D)),
                                              out.size), "poisson_plan_copy_greens")
        return out

    def sync_status(self, stream=None):
        return lib().poisson_plan_sync_status(self.handle, _stream_handle(stream))

    def close(self):
        if self._handle:
            lib().poisson_plan_destroy(self._handle)
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def solve_batched(plans, rhos, phis, stream=None):
    n = len(plans)
    if len(rhos) != n or len(phis) != n:
        raise ValueError("plans, rhos and phis must have the same length")
    for p, r, o in zip(plans, rhos, phis):
        p._io(r, o)
    PA = ctypes.c_void_p * max(n, 1)
    hp = PA(*[p.handle for p in plans])
    rp = PA(*[ctypes.c_void_p(r.data_ptr()) for r in rhos])
    op = PA(*[ctypes.c_void_p(o.data_ptr()) for o in phis])
    _check(lib().poisson_solve_batched(hp, n, rp, op, _stream_handle(stream)), "poisson_solve_batched")
    return phis


def solve_host_levels(plans, rhos_host, phis_host=None, stream=None):
    """Solve independent fields from host tensors (pinned for overlap) with
    the transfers overlapped with the solves (poisson_solve_host_levels)."""
    torch = _torch()
    n = len(plans)
    if phis_host is None:
        phis_host = [torch.empty_like(r) for r in rhos_host]
    if len(rhos_host) != n or len(phis_host) != n:
        raise ValueError("plans, rhos and phis must have the same length")
    for p, r, o in zip(plans, rhos_host, phis_host):
        for t in (r, o):
            if tuple(t.shape) != p.shape or t.dtype != p.dtype or t.is_cuda or not t.is_contiguous():
                raise ValueError("expected contiguous host %s tensors of shape %s" % (p.dtype, p.shape))
    PA = ctypes.c_void_p * max(n, 1)
    hp = PA(*[p.handle for p in plans])
    rp = PA(*[ctypes.c_void_p(r.data_ptr()) for r in rhos_host])
    op = PA(*[ctypes.c_void_p(o.data_ptr()) for o in phis_host])
    _check(lib().poisson_solve_host_levels(hp, n, rp, op, _stream_handle(stream)), "poisson_solve_host_levels")
    return phis_host


def solve_noalloc(rho, h=1.0, G=1.0, out=None, stream=None):
    """Plan-free FP32 solve that allocates no device memory inside the
    library (poisson_solve_noalloc); for small grids only (16 MiB scratch).
    The library writes nx*ny*nz floats to `out`, so `out` must be a
    contiguous float32 tensor of rho's shape on rho's device; the call runs
    with rho's device current (the scratch array is looked up per device)."""
    torch = _torch()
    if not (isinstance(rho, torch.Tensor) and rho.is_cuda and rho.dtype == torch.float32
            and rho.is_contiguous() and rho.dim() == 3):
        raise ValueError("expected a contiguous 3-D float32 CUDA tensor")
    if np.isscalar(h):
        h = (h, h, h)
    nz, ny, nx = rho.shape
    if out is None:
        out = torch.empty_like(rho)
    elif not (isinstance(out, torch.Tensor) and out.is_cuda and out.device == rho.device
              and out.dtype == torch.float32 and out.is_contiguous() and tuple(out.shape) == tuple(rho.shape)):
        raise ValueError("out must be a contiguous float32 tensor of shape %s on %s"
                         % (tuple(rho.shape), rho.device))
    with torch.cuda.device(rho.device):
        _check(lib().poisson_solve_noalloc(nx, ny, nz, float(h[0]), float(h[1]), float(h[2]), float(G),
                                           ctypes.c_void_p(rho.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                           _stream_handle(stream)), "poisson_solve_noalloc")
    return out


def _plan_array(plans):
    PA = ctypes.c_void_p * max(len(plans), 1)
    return PA(*[p.handle for p in plans])


def batch_mode(plans, mode=None):
    """Get (mode=None) or set the execution mode of the batch cached for
    this plan list: 0 persistent kernel, 1 per-field launches with each
    plan's variants, 2 per-field launches with the untuned variants, -1
    undecided."""
    hp = _plan_array(plans)
    if mode is None:
        out = ctypes.c_int(-1)
        _check(lib().poisson_batch_get_mode(hp, len(plans), ctypes.byref(out)), "poisson_batch_get_mode")
        return out.value
    _check(lib().poisson_batch_set_mode(hp, len(plans), int(mode)), "poisson_batch_set_mode")
    return int(mode)


def _make_autograd():
    torch = _torch()

    def each(fn, x):
        # one field [nz, ny, nx], or a leading batch dimension solved field by
        # field on the current stream (one plan, so the solves run in order)
        x = x.contiguous()
        if x.dim() == 3:
            return fn(x)
        out = torch.empty_like(x)
        for b in range(x.shape[0]):
            fn(x[b], out=out[b])
        return out

    class PoissonSolve(torch.autograd.Function):
        """Phi = solve(rho) for rho of shape [nz, ny, nx] or [B, nz, ny, nx];
        the backward pass is the hand-written adjoint (correlation with the
        Green's function) of libpoisson."""

        @staticmethod
        def forward(ctx, rho, plan):
            ctx.plan = plan
            return each(plan.solve, rho)

        @staticmethod
        def backward(ctx, grad_phi):
            return each(ctx.plan.adjoint, grad_phi), None

    return PoissonSolve


class _LazyAutograd:
    _cls = None

    def apply(self, *args):
        if _LazyAutograd._cls is None:
            _LazyAutograd._cls = _make_autograd()
        return _LazyAutograd._cls.apply(*args)


PoissonSolve = _LazyAutograd()
