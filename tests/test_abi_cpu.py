"""The C-ABI library loads and exports every declared entry point (CPU only, no GPU calls
that compute).  Host-side argument validation runs before any device work, so it is
checked here too."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names |= set(re.findall(r"\b(sgm_\w+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def libsgm():
    from paper_1708_03188_gb300 import build, sgm
    build.build()
    return sgm.lib()


def test_every_declared_symbol_is_exported(libsgm):
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(libsgm, n), n


def test_binding_covers_the_header(libsgm):
    from paper_1708_03188_gb300 import sgm
    assert set(_declared()) <= set(sgm._SIGNATURES)


def test_status_strings(libsgm):
    for code in range(0, -9, -1):
        s = libsgm.sgm_status_string(code).decode()
        assert s and s != "unknown status"
    assert libsgm.sgm_status_string(-99).decode() == "unknown status"


@pytest.mark.parametrize("ndim,kinds,sizes,code", [
    (0, [1], [8], -2),                 # ndim out of range
    (2, [1, 1], [8, 8], -2),           # two polynomial axes (any one axis may be polynomial)
    (2, [4, 4], [8, 8], -2),           # two R2C axes (the R2C axis may be any one axis)
    (1, [1], [3], -2),                 # Dirichlet needs N >= 4
    (1, [2], [5], -2),                 # biharmonic needs N >= 6
    (1, [2], [2049], -2),              # biharmonic needs N <= 2048 (shared-memory tables)
    (1, [9], [8], -3),                 # unknown kind
    (1, [3], [5000], -2),              # size limit
])
def test_create_rejects_bad_arguments_before_device_work(libsgm, ndim, kinds, sizes, code):
    h = ctypes.c_void_p()
    k = (ctypes.c_int * max(1, len(kinds)))(*kinds)
    n = (ctypes.c_int64 * max(1, len(sizes)))(*sizes)
    assert libsgm.sgm_space_create(ctypes.byref(h), ndim, k, n, None, 1) == code
    assert h.value is None
    assert libsgm.sgm_last_error().decode()


def test_null_arguments(libsgm):
    assert libsgm.sgm_space_create(None, 1, None, None, None, 1) == -1
    assert libsgm.sgm_space_destroy(None) == 0
    assert libsgm.sgm_scalar_product(None, None, None, None) == -1
    assert libsgm.sgm_helmholtz_solve(None, 1.0, 0.0, None, None, None) == -1
    assert libsgm.sgm_project_dx(None, 0, 1, None, None, None) == -1
