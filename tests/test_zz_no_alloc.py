"""The handle-free, allocation-free inner product (mpi_ffl_dot_f64_noalloc).

Some callers cannot allocate device memory (a framework's caching allocator owns
the GPU, or the code path must not risk an allocation's implicit device
synchronisation), so they cannot create a handle either. This checks, through
the C ABI, that the entry point for them returns the same FP64 inner product as
the handle-based mpi_ffl_dot_f64, on two calls in a row, and that it rejects
sizes its fixed scratch cannot hold. Collected last, so a failure here comes
after every other test has run.
"""

import ctypes as C

import numpy as np
import pytest

from _helpers import ensure_library

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _lib():
    ensure_library()
    from paper_2511_06627_gb300 import _lib as L

    return L, L.load()


def _noalloc_dot(lib, a, b, n=None):
    out = torch.full((), float("nan"), device="cuda", dtype=torch.float64)
    n = a.numel() if n is None else n
    rc = lib.mpi_ffl_dot_f64_noalloc(C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), C.c_int64(n),
                                     C.c_void_p(out.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out


def test_noalloc_dot_matches_handle_dot_on_two_calls():
    from paper_2511_06627_gb300 import FFLOperator

    L, lib = _lib()
    op = FFLOperator(nx=16, nz=4, n_angles=3, S=16, P=8, A=2.0, Q=4, fwhm=2.0, k_min=1, k_max=2, half_width=1)
    rng = np.random.default_rng(21)
    # first call large with a ragged tail, second call smaller: the second must not
    # pick up partial sums the first left in the shared scratch
    for n in (3_000_017, 70_001):
        a = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda()
        b = torch.from_numpy(rng.standard_normal(n).astype(np.float32)).cuda()
        ref = float(op.dot(a, b).cpu())
        rc, out = _noalloc_dot(lib, a, b)
        assert rc == L.OK, lib.mpi_ffl_last_error(None)
        got = float(out.cpu())
        tol = 1e-12 * float(a.double().norm() * b.double().norm())
        assert abs(got - ref) <= tol, (n, got, ref)
    op.close()


def test_noalloc_dot_rejects_sizes_beyond_its_scratch():
    L, lib = _lib()
    a = torch.zeros(4, device="cuda")
    rc, out = _noalloc_dot(lib, a, a, n=L.NOALLOC_MAX_N + 1)
    assert rc == L.ERR_INVALID_ARG
    assert b"exceeds the maximum" in lib.mpi_ffl_last_error(None)
    torch.cuda.synchronize()
    assert torch.isnan(out).item()  # nothing was launched
