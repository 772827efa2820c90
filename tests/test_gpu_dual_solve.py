"""Reconstruction from both scans of the dual-drive acquisition (Sec. 3.1): the solve
(Eq. (26)) and power iteration on the stacked operator [A; A_z] and on A_z alone,
against the FP64 oracle's Eq. (26) on the same stacked operator (rel-L2 1e-3)."""

import numpy as np
import pytest

from _helpers import RECON_TOL, ensure_library, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Setup, operator, solver, zdrive  # noqa: E402
from oracle.data import to_interleaved  # noqa: E402
from phantoms import config, phantom_for  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


@pytest.fixture(scope="module")
def tiny():
    cfg = config("tiny")
    st = Setup.from_config(cfg)
    x_true = phantom_for(cfg).astype(np.float64)
    rng = np.random.default_rng(51)
    M = st.n_angles
    b = np.concatenate([operator.forward(x_true, st), zdrive.forward_z(x_true, st)])
    sigma = 0.01 * np.abs(b).max()
    b = b + sigma / np.sqrt(2) * (rng.standard_normal(b.shape) + 1j * rng.standard_normal(b.shape))
    ops = {
        "xz": (lambda v: np.concatenate([operator.forward(v, st), zdrive.forward_z(v, st)]),
               lambda r: operator.adjoint(r[:M], st) + zdrive.adjoint_z(r[M:], st), b),
        "z": (lambda v: zdrive.forward_z(v, st), lambda r: zdrive.adjoint_z(r, st), b[M:]),
    }
    return dict(cfg=cfg, st=st, ops=ops, shape=(st.nz, st.nx, st.nx))


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("scans", ["xz", "z"])
def test_solve_on_the_selected_scans(tiny, scans):
    from paper_2511_06627_gb300 import FFLOperator

    apply_a, apply_at, b = tiny["ops"][scans]
    shape = tiny["shape"]
    ata = solver.power_norm(lambda v: apply_at(apply_a(v)), shape, n_iter=50, seed=1234)
    lam = solver.default_lambda(ata, shape)
    tau = solver.step_size(ata, lam, shape)
    iters = 30
    x_ref, hist = solver.solve(apply_a, apply_at, b, shape, tau, lam, iters)
    op = FFLOperator.from_config(tiny["cfg"])
    op.set_path("full_gemm")
    op.set_scans(scans)
    assert op.solve_data_shape[0] == (2 if scans == "xz" else 1) * tiny["st"].n_angles
    got_ata = op.power_norm(50, 1234)
    assert abs(got_ata - ata) <= 1e-4 * ata
    x, rep = op.solve(_t(to_interleaved(b)), iters=iters, lam=lam, tau=tau)
    op.sync_check()
    assert rel_l2(x.cpu().numpy(), x_ref) < RECON_TOL
    assert abs(rep["residual_first"] - hist[0]) <= 1e-4 * hist[0]
    assert abs(rep["b_norm"] - np.linalg.norm(b)) <= 1e-5 * np.linalg.norm(b)


def test_scan_selection_is_checked(tiny):
    from paper_2511_06627_gb300 import FFLOperator, MpiFflError

    op = FFLOperator.from_config(tiny["cfg"])
    with pytest.raises(MpiFflError):
        op.set_scans(4)
    op.set_scans("xz")
    assert op.scans == 3
    with pytest.raises(ValueError):  # x-drive data alone no longer fit the solve
        op.solve(torch.zeros(op.data_shape, device="cuda"), iters=1)
    with pytest.raises(MpiFflError):  # gradients use the x-drive scan only
        op.param_grad(torch.zeros(op.vol_shape, device="cuda"), torch.zeros(op.data_shape, device="cuda"))
    op.set_scans("x")
    assert op.solve_data_shape == op.data_shape
