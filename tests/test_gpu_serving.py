"""Continuous batching: jobs of different sizes advanced together give the same
reconstruction as alone, within the solver tolerance (rel-L2 1e-3, in fact
bit-identical), and the server admits requests by HBM budget while others run."""

import ctypes as C

import numpy as np
import pytest

from _helpers import RECON_TOL, ensure_library, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Setup, operator, solver  # noqa: E402
from oracle.data import make_data, to_interleaved  # noqa: E402
from phantoms import config, phantom_ellipsoids, phantom_tiny  # noqa: E402

GEOMS = [
    {k: config("tiny")[k] for k in ("nx", "nz", "n_angles", "S", "P", "A", "phi0", "zigzag", "Q", "fwhm",
                                     "k_min", "k_max", "half_width")},
    dict(nx=24, nz=6, n_angles=5, S=64, P=64, A=5.0, phi0=0.1, zigzag=1, Q=8, fwhm=2.5, k_min=1, k_max=6, half_width=2),
    dict(nx=40, nz=8, n_angles=12, S=128, P=80, A=6.0, phi0=0.0, zigzag=0, Q=8, fwhm=3.0, k_min=2, k_max=8,
         half_width=3),
]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


def _data(geom, seed):
    st = Setup(**geom)
    x = phantom_ellipsoids(geom["nx"], geom["nz"], seed=seed, n_ellipsoids=4, n_points=2)
    b, _ = make_data(st, x, noise=0.01, seed=seed)
    return st, x, b


def _job_api():
    from paper_2511_06627_gb300 import _lib as L
    from paper_2511_06627_gb300.serving import JobStatus, _declare

    lib = L.load()
    _declare(lib)
    return L, lib, JobStatus


def _make_job(lib, L, op, b_dev, iters, tau, lam, stop_rel=0.0):
    p = L.SolveParams(iters, lam, tau, 20, C.c_uint64(1234), 1, stop_rel, 0.0)
    h = C.c_void_p()
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.mpi_ffl_job_create(op._h, C.c_void_p(b_dev.data_ptr()), None, C.byref(p), C.byref(h), s) == 0
    return h


def _run(lib, jobs, iters):
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    arr = (C.c_void_p * len(jobs))(*jobs)
    for _ in range(iters):
        assert lib.mpi_ffl_job_step(arr, len(jobs), s) == 0


def _result(lib, op, h):
    x = op.new_volume()
    assert lib.mpi_ffl_job_result(h, C.c_void_p(x.data_ptr()), C.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()
    return x.cpu().numpy()


@pytest.mark.parametrize("path", ["full_gemm", "line_gemm", "full_gemm_tf32"])
def test_jobs_alone_and_in_the_mix_agree(path):
    from paper_2511_06627_gb300 import PREC_TF32, FFLOperator

    L, lib, _ = _job_api()
    iters = 30
    problems = []
    for i, g in enumerate(GEOMS):
        st, x, b = _data(g, seed=60 + i)
        op = FFLOperator(**g)
        op.set_path(path.replace("_tf32", ""))
        if path.endswith("_tf32"):
            op.set_precision(PREC_TF32)
        ata = op.power_norm(40, 1234)
        lam = 1e-3 * ata / 10.0
        tau = 1.0 / (ata + lam * 12.0)
        problems.append((g, st, op, torch.from_numpy(to_interleaved(b).astype(np.float32)).cuda(), tau, lam))
    alone = []
    for g, st, op, bd, tau, lam in problems:
        h = _make_job(lib, L, op, bd, iters, tau, lam)
        _run(lib, [h.value], iters)
        alone.append(_result(lib, op, h))
        lib.mpi_ffl_job_destroy(h)
        # the same solve through mpi_ffl_solve
        xs, _ = op.solve(bd, iters=iters, lam=lam, tau=tau)
        assert rel_l2(alone[-1], xs.cpu().numpy()) < 1e-6
    hs = [_make_job(lib, L, op, bd, iters, tau, lam) for g, st, op, bd, tau, lam in problems]
    _run(lib, [h.value for h in hs], iters)
    for (g, st, op, bd, tau, lam), h, xa in zip(problems, hs, alone):
        xm = _result(lib, op, h)
        assert rel_l2(xm, xa) < RECON_TOL
        assert np.array_equal(xm, xa)  # same kernels, same summation order per job
        lib.mpi_ffl_job_destroy(h)


def test_batched_job_matches_oracle_solve():
    from paper_2511_06627_gb300 import FFLOperator

    L, lib, _ = _job_api()
    g = GEOMS[0]
    st = Setup(**g)
    x_true = phantom_tiny(g["nx"], g["nz"], seed=0)
    b, _ = make_data(st, x_true, noise=0.01, seed=0)
    shape = (st.nz, st.nx, st.nx)
    ata = solver.power_norm(lambda v: operator.adjoint(operator.forward(v, st), st), shape, n_iter=50)
    lam = solver.default_lambda(ata, shape)
    tau = solver.step_size(ata, lam, shape)
    x_ref, _ = solver.solve(lambda v: operator.forward(v, st), lambda r: operator.adjoint(r, st), b, shape, tau, lam, 50)
    op = FFLOperator(**g)
    op.set_path("full_gemm")
    other = FFLOperator(**GEOMS[2])
    other.set_path("full_gemm")
    _, _, b2 = _data(GEOMS[2], seed=7)
    h = _make_job(lib, L, op, torch.from_numpy(to_interleaved(b).astype(np.float32)).cuda(), 50, tau, lam)
    h2 = _make_job(lib, L, other, torch.from_numpy(to_interleaved(b2).astype(np.float32)).cuda(), 50, tau, lam)
    _run(lib, [h.value, h2.value], 50)
    assert rel_l2(_result(lib, op, h), x_ref) < RECON_TOL
    lib.mpi_ffl_job_destroy(h)
    lib.mpi_ffl_job_destroy(h2)


def test_early_stop_in_the_mix_matches_alone():
    from paper_2511_06627_gb300 import FFLOperator

    L, lib, JobStatus = _job_api()
    g0, g1 = GEOMS[0], GEOMS[1]
    ops, bds = [], []
    for i, g in enumerate((g0, g1)):
        _, _, b = _data(g, seed=70 + i)
        op = FFLOperator(**g)
        op.set_path("full_gemm")
        ops.append(op)
        bds.append(torch.from_numpy(to_interleaved(b).astype(np.float32)).cuda())
    taus = [1.0 / (1.05 * op.power_norm(40, 1234)) for op in ops]
    xs, rep = ops[0].solve(bds[0], iters=300, lam=0.0, tau=taus[0], stop_rel=2e-3)
    h0 = _make_job(lib, L, ops[0], bds[0], 300, taus[0], 0.0, stop_rel=2e-3)
    h1 = _make_job(lib, L, ops[1], bds[1], 300, taus[1], 0.0, stop_rel=0.0)
    _run(lib, [h0.value, h1.value], 300)
    st = JobStatus()
    assert lib.mpi_ffl_job_status(h0, C.byref(st), C.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    assert st.stopped == 1 and st.iters_done == rep["iters_done"]
    assert rel_l2(_result(lib, ops[0], h0), xs.cpu().numpy()) < 1e-6
    assert lib.mpi_ffl_job_status(h1, C.byref(st), C.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    assert st.iters_done == 300
    lib.mpi_ffl_job_destroy(h0)
    lib.mpi_ffl_job_destroy(h1)


def test_server_admits_by_budget_and_overlaps_requests():
    from paper_2511_06627_gb300.serving import ReconServer, Request, estimate_request_bytes, run_sequential

    reqs = []
    for i in range(8):
        g = GEOMS[i % 3]
        _, _, b = _data(g, seed=80 + i)
        reqs.append(Request(geometry=g, data=torch.from_numpy(to_interleaved(b).astype(np.float32)),
                            iters=40, arrival=0.01 * i, name=f"r{i}"))
    budget = int(2.5 * max(estimate_request_bytes(g) for g in GEOMS))
    server = ReconServer(hbm_budget_bytes=budget, path="full_gemm", max_active=8)
    out = server.run(reqs)
    assert len(out) == 8 and all(r.finished is not None for r in out)
    assert server.peak_bytes <= budget
    # some request started while another was still running
    spans = sorted((r.admitted, r.finished) for r in out)
    assert any(spans[i + 1][0] < spans[i][1] for i in range(len(spans) - 1))
    # each result equals the same solve run alone
    import copy

    solo = run_sequential([copy.copy(r) for r in reqs], path="full_gemm")
    by_name = {r.name: r for r in solo}
    for r in out:
        assert rel_l2(r.result.cpu().numpy(), by_name[r.name].result.cpu().numpy()) < RECON_TOL
