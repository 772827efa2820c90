"""Parity of the GPU solve (Eq. (26)) and power iteration with the FP64 oracle.

Reconstructed volumes must match the oracle within rel-L2 1e-3."""

import numpy as np
import pytest

from _helpers import RECON_TOL, ensure_library, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Setup, operator, solver  # noqa: E402
from oracle.data import make_data, to_interleaved  # noqa: E402
from phantoms import config, phantom_for  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


@pytest.fixture(scope="module")
def tiny():
    from paper_2511_06627_gb300 import FFLOperator

    cfg = config("tiny")
    st = Setup.from_config(cfg)
    x_true = phantom_for(cfg)
    b, info = make_data(st, x_true, noise=cfg["noise"], seed=cfg["seed"])
    shape = (st.nz, st.nx, st.nx)
    ata = solver.power_norm(lambda v: operator.adjoint(operator.forward(v, st), st), shape, n_iter=50, seed=1234)
    lam = solver.default_lambda(ata, shape)
    tau = solver.step_size(ata, lam, shape)
    op = FFLOperator.from_config(cfg)
    return dict(cfg=cfg, st=st, x_true=x_true, b=b, ata=ata, lam=lam, tau=tau, op=op, shape=shape)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def test_power_norm_matches_oracle(tiny):
    got = tiny["op"].power_norm(50, 1234)
    assert abs(got - tiny["ata"]) <= 1e-4 * tiny["ata"]


def test_solve_matches_oracle(tiny):
    st, b = tiny["st"], tiny["b"]
    iters = tiny["cfg"]["iters"]
    x_ref, hist = solver.solve(lambda v: operator.forward(v, st), lambda r: operator.adjoint(r, st),
                               b, tiny["shape"], tiny["tau"], tiny["lam"], iters)
    x, rep = tiny["op"].solve(_t(to_interleaved(b)), iters=iters, lam=tiny["lam"], tau=tiny["tau"])
    xg = x.cpu().numpy()
    assert rel_l2(xg, x_ref) < RECON_TOL
    assert xg.min() >= 0.0
    assert rep["iters_done"] == iters
    assert abs(rep["residual_first"] - hist[0]) <= 1e-4 * hist[0]
    assert abs(rep["residual_last"] - hist[-1]) <= RECON_TOL * hist[-1]


def test_solve_with_power_iteration_and_default_lambda(tiny):
    b = _t(to_interleaved(tiny["b"]))
    x, rep = tiny["op"].solve(b, iters=5, lam=-1.0, tau=0.0, n_power=50, seed=1234)
    assert abs(rep["ata_norm"] - tiny["ata"]) <= 1e-4 * tiny["ata"]
    assert abs(rep["lam"] - tiny["lam"]) <= 1e-4 * tiny["lam"]
    assert abs(rep["tau"] - tiny["tau"]) <= 1e-4 * tiny["tau"]


def test_early_stop_matches_oracle(tiny):
    st, b = tiny["st"], tiny["b"]
    x_ref, hist = solver.solve(lambda v: operator.forward(v, st), lambda r: operator.adjoint(r, st),
                               b, tiny["shape"], tiny["tau"], tiny["lam"], 200, stop_rel=1e-3)
    x, rep = tiny["op"].solve(_t(to_interleaved(b)), iters=200, lam=tiny["lam"], tau=tiny["tau"], stop_rel=1e-3)
    assert abs(rep["iters_done"] - len(hist)) <= 1
    assert rep["iters_done"] < 200


def test_unconstrained_solve_matches_oracle(tiny):
    st, b = tiny["st"], tiny["b"]
    x_ref, _ = solver.solve(lambda v: operator.forward(v, st), lambda r: operator.adjoint(r, st),
                            b, tiny["shape"], tiny["tau"], tiny["lam"], 20, nonneg=False)
    x, _ = tiny["op"].solve(_t(to_interleaved(b)), iters=20, lam=tiny["lam"], tau=tiny["tau"], nonneg=False)
    assert rel_l2(x.cpu().numpy(), x_ref) < RECON_TOL


@pytest.mark.parametrize("path", ["staged", "full_gemm"])
def test_non_finite_data_stop_the_solve(tiny, path):
    """A NaN in the data makes the FP64 residual non-finite: the solve stops and returns
    MPI_FFL_ERR_NONFINITE instead of iterating on garbage."""
    from paper_2511_06627_gb300 import FFLOperator, MpiFflError
    from paper_2511_06627_gb300._lib import ERR_NONFINITE

    op = FFLOperator.from_config(tiny["cfg"])
    op.set_path(path)
    b = to_interleaved(tiny["b"]).astype(np.float32)
    b.flat[17] = np.nan
    with pytest.raises(MpiFflError) as ei:
        op.solve(_t(b), iters=20, lam=tiny["lam"], tau=tiny["tau"])
    assert ei.value.code == ERR_NONFINITE
    # the handle stays usable: a clean solve afterwards matches a fresh handle
    x1, _ = op.solve(_t(to_interleaved(tiny["b"])), iters=10, lam=tiny["lam"], tau=tiny["tau"])
    fresh = FFLOperator.from_config(tiny["cfg"])
    fresh.set_path(path)
    x2, _ = fresh.solve(_t(to_interleaved(tiny["b"])), iters=10, lam=tiny["lam"], tau=tiny["tau"])
    assert np.array_equal(x1.cpu().numpy(), x2.cpu().numpy())
