"""Failure detection on the GPU, in forms that fault and hang nothing.

Timeouts: every mbarrier wait of the tensor-core and projector kernels is bounded;
a kernel that gives up records a timeout, frees its TMEM and returns, and
mpi_ffl_sync_check turns the record into MPI_FFL_ERR_TIMEOUT. The test hook
mpi_ffl_test_inject_timeout makes the projector and line-GEMM blocks of the next
calls wait on a barrier that nothing arrives at (before any copy or MMA is issued),
so the bounded waits run out for real; afterwards the handle must give the same
bits as before.

Allocation failures: mpi_ffl_test_fail_alloc makes the n-th device allocation from
now fail as on a full device. Every failing call must return MPI_FFL_ERR_OOM, leave
no device allocation behind (the library's own registry of live allocations), and
leave the handle, or the next create, working.
"""

import ctypes as C

import numpy as np
import pytest

from _helpers import OP_TOL, ensure_library, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Setup, operator  # noqa: E402
from oracle.data import to_interleaved  # noqa: E402
from phantoms import config, phantom_for  # noqa: E402


@pytest.fixture(scope="module")
def env():
    ensure_library()
    from paper_2511_06627_gb300 import _lib as L

    lib = L.load()
    cfg = config("tiny")
    x = phantom_for(cfg)
    st = Setup.from_config(cfg)
    b_ref = to_interleaved(operator.forward(x, st))
    yield dict(L=L, lib=lib, cfg=cfg, x=torch.from_numpy(x).cuda(), b_ref=b_ref)
    lib.mpi_ffl_test_fail_alloc(0)


def _live(lib):
    n, b = C.c_int64(), C.c_int64()
    assert lib.mpi_ffl_test_live_allocs(C.byref(n), C.byref(b)) == 0
    return n.value, b.value


def _op(cfg, path):
    from paper_2511_06627_gb300 import FFLOperator

    op = FFLOperator.from_config(cfg)
    op.set_path(path)
    return op


@pytest.mark.parametrize("path", ["full_gemm", "line_gemm"])
def test_injected_timeout_is_reported_and_the_handle_recovers(env, path):
    from paper_2511_06627_gb300 import MpiFflError

    L, lib = env["L"], env["lib"]
    op = _op(env["cfg"], path)
    b1 = op.forward(env["x"]).clone()
    x1 = op.adjoint(b1).clone()
    op.sync_check()
    assert rel_l2(b1.cpu().numpy(), env["b_ref"]) < OP_TOL
    for direction in ("forward", "adjoint"):
        assert lib.mpi_ffl_test_inject_timeout(op._h, 256) == L.OK
        if direction == "forward":
            op.forward(env["x"])  # the projector and the GEMM both give up
        else:
            op.adjoint(b1)  # the GEMM gives up
        with pytest.raises(MpiFflError) as ei:
            op.sync_check()
        assert ei.value.code == L.ERR_TIMEOUT
        op.sync_check()  # the flag is cleared and the hook disarmed
        assert torch.equal(op.forward(env["x"]), b1)
        assert torch.equal(op.adjoint(b1), x1)
        op.sync_check()
    assert lib.mpi_ffl_test_inject_timeout(op._h, (1 << 24) + 1) == L.ERR_INVALID_ARG
    op.close()


def test_failed_creates_leak_nothing_and_the_next_create_works(env):
    from paper_2511_06627_gb300 import MpiFflError

    L, lib = env["L"], env["lib"]
    warm = _op(env["cfg"], "staged")
    ref = warm.forward(env["x"]).clone()
    warm.close()
    torch.cuda.synchronize()
    base = _live(lib)
    failures = 0
    for n in range(1, 200):
        assert lib.mpi_ffl_test_fail_alloc(n) == L.OK
        try:
            op = _op(env["cfg"], "staged")
        except MpiFflError as e:
            assert e.code == L.ERR_OOM, e
            assert _live(lib) == base, n
            failures += 1
            continue
        op.close()  # n is past the allocations of create: the countdown is still armed
        assert lib.mpi_ffl_test_fail_alloc(0) == L.OK
        assert _live(lib) == base
        break
    assert failures >= 20
    op = _op(env["cfg"], "staged")
    assert torch.equal(op.forward(env["x"]), ref)
    op.close()
    assert _live(lib) == base


def test_failed_first_use_allocations_roll_back(env):
    """Allocations made on first use: the staged path's time signal, the collapsed
    operator built by set_path, the staging of host buffers."""
    from paper_2511_06627_gb300 import MpiFflError

    L, lib = env["L"], env["lib"]
    refs = {}
    for p in ("staged", "full_gemm"):
        o = _op(env["cfg"], p)
        refs[p] = o.forward(env["x"]).clone()
        o.close()
    torch.cuda.synchronize()
    base = _live(lib)
    from paper_2511_06627_gb300 import FFLOperator

    op = FFLOperator.from_config(env["cfg"])  # staged; its time signal is not yet allocated
    after_create = _live(lib)
    assert lib.mpi_ffl_test_fail_alloc(1) == L.OK
    with pytest.raises(MpiFflError) as ei:
        op.forward(env["x"])
    assert ei.value.code == L.ERR_OOM
    assert _live(lib) == after_create
    assert torch.equal(op.forward(env["x"]), refs["staged"])
    # set_path builds the collapsed operator: every allocation of that build may fail
    n_fail = 0
    for n in range(1, 100):
        assert lib.mpi_ffl_test_fail_alloc(n) == L.OK
        before = _live(lib)
        try:
            op.set_path("full_gemm")
        except MpiFflError as e:
            assert e.code == L.ERR_OOM, e
            assert _live(lib) == before, n
            assert torch.equal(op.forward(env["x"]), refs["staged"])  # still on its old path
            n_fail += 1
            continue
        assert lib.mpi_ffl_test_fail_alloc(0) == L.OK
        break
    assert n_fail >= 5
    assert torch.equal(op.forward(env["x"]), refs["full_gemm"])
    # host buffers: the device staging is allocated on the first host call
    xh = env["x"].cpu().pin_memory()
    assert lib.mpi_ffl_test_fail_alloc(2) == L.OK
    with pytest.raises(MpiFflError) as ei:
        op.forward(xh)
    assert ei.value.code == L.ERR_OOM
    assert lib.mpi_ffl_test_fail_alloc(0) == L.OK
    assert torch.equal(op.forward(xh), refs["full_gemm"])
    op.close()
    torch.cuda.synchronize()
    assert _live(lib) == base
