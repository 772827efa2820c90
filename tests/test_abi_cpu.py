"""CPU-side checks of the C ABI: the library loads, exports every symbol that
include/mpi_ffl.h declares, and rejects invalid descriptions before any GPU work."""

import ctypes as C
import os
import re

import pytest

from _helpers import ROOT, ensure_library


@pytest.fixture(scope="module")
def lib():
    ensure_library()
    from paper_2511_06627_gb300 import _lib

    return _lib.load()


def _declared_symbols():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            names |= set(re.findall(r"\b(mpi_ffl_\w+)\s*\(", text))
    return sorted(names)


def test_header_declares_the_boundary():
    names = _declared_symbols()
    for required in ("mpi_ffl_create", "mpi_ffl_forward", "mpi_ffl_adjoint", "mpi_ffl_solve", "mpi_ffl_destroy"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in _declared_symbols():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2511_06627_gb300 import _lib

    assert set(_declared_symbols()) <= set(_lib.PROTOTYPES)


def _describe(nx=16, ny=16, nz=4, M=3, S=16, P=8, A=2.0, Q=4, kmin=1, kmax=2, hw=1):
    from paper_2511_06627_gb300 import _lib

    g = _lib.Geometry(nx, ny, nz, M, None, None)
    t = _lib.Trajectory(S, P, A, 0.0, 1, Q)
    p = _lib.Psf(2.0)
    h = _lib.Harmonics(kmin, kmax, hw, None)
    return g, t, p, h


@pytest.mark.parametrize("bad,msg", [
    (dict(ny=12), "nx must equal ny"),
    (dict(kmax=9), "harmonic band"),         # 9*8+1 >= L/2 = 64
    (dict(kmin=0, hw=1), "harmonic band"),   # 0*8 - 1 < 1
    (dict(hw=9), "half_width"),
    (dict(S=1), "bad trajectory"),
    (dict(M=0), "bad volume"),
])
def test_create_rejects_invalid_descriptions(lib, bad, msg):
    from paper_2511_06627_gb300 import _lib

    g, t, p, h = _describe(**bad)
    out = C.c_void_p()
    rc = lib.mpi_ffl_create(C.byref(g), C.byref(t), C.byref(p), C.byref(h), C.byref(out))
    assert rc == _lib.ERR_INVALID_ARG
    assert out.value is None
    assert msg in lib.mpi_ffl_last_error(None).decode()


def test_null_arguments_are_rejected(lib):
    from paper_2511_06627_gb300 import _lib

    assert lib.mpi_ffl_destroy(None) == _lib.OK
    assert lib.mpi_ffl_forward(None, None, None, None) == _lib.ERR_INVALID_ARG
    assert lib.mpi_ffl_create(None, None, None, None, None) == _lib.ERR_INVALID_ARG
    assert lib.mpi_ffl_get_sizes(None, None) == _lib.ERR_INVALID_ARG
    assert lib.mpi_ffl_set_precision(None, 0) == _lib.ERR_INVALID_ARG


def test_product_package_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2511_06627_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
                assert "oracle/" not in text, f


def test_failure_hooks_validate_their_arguments(lib):
    """The allocation-failure countdown and the live-allocation registry need no GPU."""
    from paper_2511_06627_gb300 import _lib

    assert lib.mpi_ffl_test_fail_alloc(-1) == _lib.ERR_INVALID_ARG
    assert lib.mpi_ffl_test_fail_alloc(3) == _lib.OK
    assert lib.mpi_ffl_test_fail_alloc(0) == _lib.OK
    n, b = C.c_int64(-1), C.c_int64(-1)
    assert lib.mpi_ffl_test_live_allocs(C.byref(n), C.byref(b)) == _lib.OK
    assert n.value >= 0 and b.value >= 0
    assert lib.mpi_ffl_test_live_allocs(None, None) == _lib.OK
    assert lib.mpi_ffl_test_inject_timeout(None, 4) == _lib.ERR_INVALID_ARG
