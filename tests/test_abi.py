"""The C-ABI library loads and exports what include/poisson.h declares (CPU).

No compute call is made here: only argument checks that the library rejects
before it touches the device.
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", fn)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*[A-Za-z_][\w\s\*]*?\b(poisson_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def L():
    from paper_2409_02294_gb300 import abi
    return abi.lib()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ["poisson_plan_create", "poisson_solve", "poisson_solve_batched",
                     "poisson_solve_adjoint", "poisson_plan_destroy", "poisson_status_string"]:
        assert required in names


def test_every_declared_symbol_is_exported(L):
    for name in _declared_functions():
        assert hasattr(L, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2409_02294_gb300 import abi
    bound = {n for n, _, _ in abi.SIGNATURES}
    assert _declared_functions() <= bound


def test_status_strings(L):
    for code in range(7):
        s = L.poisson_status_string(code)
        assert isinstance(s, bytes) and len(s) > 0
    assert L.poisson_status_string(99) == b"unknown status"


def test_supported_sizes(L):
    for n in [16, 32, 48, 64, 96, 128, 192, 256, 384, 512]:
        assert L.poisson_supported_size(n) == 1
    for n in [0, 1, 17, 100, 1024, -32]:
        assert L.poisson_supported_size(n) == 0


def test_argument_errors_before_any_device_work(L):
    from paper_2409_02294_gb300 import abi
    h = ctypes.c_void_p()
    create = L.poisson_plan_create
    # null out pointer
    assert L.poisson_plan_create(None, 32, 32, 32, 1.0, 1.0, 1.0, 1.0, 1, 0, None) == 1
    # bad spacing / G / flags / r_near
    assert create(ctypes.byref(h), 32, 32, 32, 0.0, 1.0, 1.0, 1.0, 1, 0, None) == 1
    assert create(ctypes.byref(h), 32, 32, 32, 1.0, -1.0, 1.0, 1.0, 1, 0, None) == 1
    assert create(ctypes.byref(h), 32, 32, 32, 1.0, 1.0, 1.0, float("nan"), 1, 0, None) == 1
    assert create(ctypes.byref(h), 32, 32, 32, 1.0, 1.0, 1.0, 1.0, 1, 0x80, None) == 1
    assert L.poisson_plan_create_ex(ctypes.byref(h), 32, 32, 32, 1.0, 1.0, 1.0, 1.0, 1, 0, -1, None) == 1
    # sizes
    assert create(ctypes.byref(h), 0, 32, 32, 1.0, 1.0, 1.0, 1.0, 1, 0, None) == 1
    assert create(ctypes.byref(h), 33, 32, 32, 1.0, 1.0, 1.0, 1.0, 1, 0, None) == 4
    assert create(ctypes.byref(h), 32, 32, 1024, 1.0, 1.0, 1.0, 1.0, 1, 0, None) == 4
    assert h.value is None
    # null plans
    x = ctypes.c_void_p(16)
    assert L.poisson_solve(None, x, x, None) == 1
    assert L.poisson_solve_adjoint(None, x, x, None) == 1
    assert L.poisson_solve_host(None, x, x, None) == 1
    assert L.poisson_solve_pass(None, 0, x, x, None) == 1
    assert L.poisson_solve_unfused(None, x, x, None) == 1
    assert L.poisson_plan_destroy(None) == 1
    assert L.poisson_plan_get_info(None, None) == 1
    assert L.poisson_plan_copy_greens(None, None, 0) == 1
    assert L.poisson_plan_sync_status(None, None) == 1
    assert L.poisson_solve_batched(None, -1, None, None, None) == 1
    assert L.poisson_solve_batched(None, 0, None, None, None) == 0
    assert abi.STATUS_NAMES[4] == "POISSON_ERR_UNSUPPORTED"
