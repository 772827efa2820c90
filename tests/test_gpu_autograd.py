"""Autograd wrapper and calibration gradients (per-angle gain, PSF width) against
central finite differences of the FP64 oracle (h = 1e-3, rel 1e-4)."""

import numpy as np
import pytest

from _helpers import OP_TOL, ensure_library, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Setup, operator  # noqa: E402
from oracle.data import to_interleaved  # noqa: E402
from phantoms import phantom_ellipsoids, random_volume  # noqa: E402

# the phantom-scale scan (24 angles, 64 samples/period, harmonics 1..12 at +-3 bins, FWHM 3)
# on a smaller volume and line so that finite differences of the oracle stay quick
GEOM = dict(nx=32, nz=6, n_angles=24, S=64, P=64, A=6.0, phi0=0.0, zigzag=1, Q=8, fwhm=3.0,
            k_min=1, k_max=12, half_width=3)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _oracle_loss(x, gb, gains, fwhm):
    st = Setup(**{**GEOM, "fwhm": fwhm}, gains=np.asarray(gains, dtype=np.float64))
    return float(np.sum((operator.forward(x, st) * np.conj(gb)).real))


@pytest.mark.parametrize("path", ["staged", "fused", "line_gemm", "full_gemm"])
def test_calibration_gradients_match_oracle_finite_differences(path):
    from paper_2511_06627_gb300 import FFLOperator

    rng = np.random.default_rng(51)
    gains = rng.uniform(0.95, 1.05, GEOM["n_angles"]).astype(np.float32).astype(np.float64)
    x = phantom_ellipsoids(GEOM["nx"], GEOM["nz"], seed=5, n_ellipsoids=4, n_points=2).astype(np.float64)
    shape = (GEOM["n_angles"], GEOM["nz"], (12) * 7)
    gb = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64).astype(np.complex128)
    from paper_2511_06627_gb300 import MpiFflError

    op = FFLOperator(**GEOM, gains=gains)
    try:
        op.set_path(path)
    except MpiFflError:
        pytest.skip(f"path {path} does not take this shape")
    gg, gw = op.param_grad(_t(x), _t(to_interleaved(gb)))
    gg = gg.cpu().numpy().astype(np.float64)
    gw = float(gw.cpu().numpy()[0])
    # loss(g, w) = <gb, A(g, w) x> is linear in each gain: central differences are exact up to rounding
    h = 1e-3
    fd_g = np.empty(GEOM["n_angles"])
    for m in range(GEOM["n_angles"]):
        gp, gm_ = gains.copy(), gains.copy()
        gp[m] += h
        gm_[m] -= h
        fd_g[m] = (_oracle_loss(x, gb, gp, 3.0) - _oracle_loss(x, gb, gm_, 3.0)) / (2 * h)
    fd_w = (_oracle_loss(x, gb, gains, 3.0 + h) - _oracle_loss(x, gb, gains, 3.0 - h)) / (2 * h)
    assert rel_l2(gg, fd_g) < 1e-4
    assert abs(gw - fd_w) <= 1e-4 * abs(fd_w)


def test_autograd_function_matches_library_products():
    from paper_2511_06627_gb300 import FFLOperator
    from paper_2511_06627_gb300.autograd import apply_a

    op = FFLOperator(**GEOM)
    op.set_path("line_gemm")
    st = Setup(**GEOM)
    xn = random_volume(GEOM["nz"], GEOM["nx"], seed=52).astype(np.float32)
    x = _t(xn).requires_grad_(True)
    g = torch.ones(GEOM["n_angles"], device="cuda", requires_grad=True)
    w = torch.tensor([3.0], device="cuda", requires_grad=True)
    b = apply_a(op, x, g, w)
    assert rel_l2(b.detach().cpu().numpy(), to_interleaved(operator.forward(xn, st))) < OP_TOL
    gb = torch.randn_like(b)
    (b * gb).sum().backward()
    ref_x = operator.adjoint(gb.cpu().numpy()[..., 0] + 1j * gb.cpu().numpy()[..., 1], st)
    assert rel_l2(x.grad.cpu().numpy(), ref_x) < OP_TOL
    gg, gw = op.param_grad(x.detach(), gb)
    np.testing.assert_allclose(g.grad.cpu().numpy(), gg.cpu().numpy(), rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(w.grad.cpu().numpy(), gw.cpu().numpy(), rtol=1e-5, atol=1e-6)


def test_calibration_fit_recovers_gains_and_psf_width():
    """Known phantom, unknown per-angle gains and PSF width: the fit moves both to the truth."""
    from paper_2511_06627_gb300 import FFLOperator
    from paper_2511_06627_gb300.autograd import calibrate

    geom = dict(GEOM, n_angles=8)
    rng = np.random.default_rng(53)
    g_true = rng.uniform(0.95, 1.05, 8)
    w_true = 3.3
    x = phantom_ellipsoids(geom["nx"], geom["nz"], seed=6, n_ellipsoids=5, n_points=3)
    st = Setup(**{**geom, "fwhm": w_true}, gains=g_true)
    b = _t(to_interleaved(operator.forward(x.astype(np.float64), st)))
    op = FFLOperator(**geom)
    op.set_path("line_gemm")
    # x fixed at the phantom: a calibration scan
    xt = _t(x)
    from paper_2511_06627_gb300.autograd import apply_a

    g = torch.ones(8, device="cuda", requires_grad=True)
    w = torch.tensor([3.0], device="cuda", requires_grad=True)
    # 9 calibration parameters: quasi-Newton handles the gain/width coupling
    optim = torch.optim.LBFGS([g, w], lr=1.0, max_iter=200, line_search_fn="strong_wolfe",
                              tolerance_grad=1e-12, tolerance_change=1e-16, history_size=20)
    losses = []

    def closure():
        optim.zero_grad()
        loss = 0.5 * ((apply_a(op, xt, g, w) - b) ** 2).sum()
        loss.backward()
        losses.append(float(loss.detach()))
        return loss

    optim.step(closure)
    gf, wf = g.detach().cpu().numpy(), float(w.detach())
    assert losses[-1] < 1e-4 * losses[0], (losses[0], losses[-1], wf, gf - g_true)
    assert abs(wf - w_true) < 0.01, wf
    assert np.max(np.abs(gf - g_true)) < 2e-3, gf - g_true
    # joint volume + calibration fit: the data misfit falls
    xj, gj, wj, hist = calibrate(op, b, iters=50, gains0=[1.0] * 8, fwhm0=3.0)
    assert hist[-1] < 0.2 * hist[0]
    assert float(xj.min()) >= 0.0


# ---------------------------------------------------------------------------------
# The calibration workload at its own geometry: the phantom-scale scan (128^2 x 64,
# 24 angles, 64 lines x 256 periods x 64 samples, harmonics 1..12 at +-3 bins, FWHM 3)
# with unknown per-angle gains and PSF width.

from phantoms import config, phantom_for  # noqa: E402

PH = {k: config("phantom")[k] for k in ("nx", "nz", "n_angles", "S", "P", "A", "phi0", "zigzag", "Q", "fwhm",
                                         "k_min", "k_max", "half_width")}


@pytest.fixture(scope="module")
def phantom_fd():
    """Central differences (h = 1e-3) of loss(g, w) = <gb, A(g, w) x> by the FP64 oracle.
    loss is a sum over angles and angle m alone depends on g_m, so the difference for
    g_m needs only angle m's data at g_m +- h; the width moves every angle."""
    rng = np.random.default_rng(61)
    M = PH["n_angles"]
    gains = rng.uniform(0.95, 1.05, M).astype(np.float32).astype(np.float64)
    x = phantom_for(config("phantom")).astype(np.float64)
    nb = (PH["k_max"] - PH["k_min"] + 1) * (2 * PH["half_width"] + 1)
    shape = (M, PH["nz"], nb)
    gb = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64).astype(np.complex128)
    h = 1e-3

    def angle_loss(m, g_m, w):
        st = Setup(**{**PH, "fwhm": w}, gains=np.full(M, g_m))
        d = operator.forward_stages(x, st, angles=np.array([m]))["data"][0]
        return float(np.sum((d * np.conj(gb[m])).real))

    fd_g = np.array([(angle_loss(m, gains[m] + h, 3.0) - angle_loss(m, gains[m] - h, 3.0)) / (2 * h)
                     for m in range(M)])

    b_plus = operator.forward(x, Setup(**{**PH, "fwhm": 3.0 + h}, gains=gains))
    b_minus = operator.forward(x, Setup(**{**PH, "fwhm": 3.0 - h}, gains=gains))
    fd_w = (float(np.sum((b_plus * np.conj(gb)).real)) - float(np.sum((b_minus * np.conj(gb)).real))) / (2 * h)
    # |<gb, (dA/dw) x>| is a sum of terms of random sign; an error of relative size e in
    # the vector (dA/dw) x moves it by at most e ||gb|| ||(dA/dw) x|| (Cauchy-Schwarz)
    scale_w = float(np.linalg.norm(gb) * np.linalg.norm((b_plus - b_minus) / (2 * h)))
    return dict(x=x, gb=gb, gains=gains, fd_g=fd_g, fd_w=fd_w, scale_w=scale_w)


@pytest.mark.parametrize("path", ["staged", "fused", "line_gemm", "full_gemm"])
def test_calibration_gradients_at_the_phantom_geometry(phantom_fd, path):
    from paper_2511_06627_gb300 import FFLOperator

    op = FFLOperator(**PH, gains=phantom_fd["gains"])
    op.set_path(path)  # P = 256: every path takes this shape, the fused one included
    gg, gw = op.param_grad(_t(phantom_fd["x"]), _t(to_interleaved(phantom_fd["gb"])))
    gg = gg.cpu().numpy().astype(np.float64)
    gw = float(gw.cpu().numpy()[0])
    assert rel_l2(gg, phantom_fd["fd_g"]) < 1e-4
    # the width gradient within 1e-4 of the difference, or, where its terms cancel,
    # within what the operator tolerance on (dA/dw) x allows (Cauchy-Schwarz)
    bound = max(1e-4 * abs(phantom_fd["fd_w"]), OP_TOL * phantom_fd["scale_w"])
    assert abs(gw - phantom_fd["fd_w"]) <= bound, (gw, phantom_fd["fd_w"], bound)
    op.close()


def test_joint_fit_at_the_phantom_geometry():
    """200 iterations of the joint volume + calibration fit (x >= 0 by projected
    gradient, gains and width by Adam) on data from unknown gains U(0.95, 1.05) and a
    PSF width of 3.3 voxels, started at unit gains and width 3. The volume and the gains
    share one scale (A(c g) x / c = A(g) x), so the gains are compared after dividing by
    their mean."""
    from paper_2511_06627_gb300 import FFLOperator
    from paper_2511_06627_gb300.autograd import calibrate

    rng = np.random.default_rng(62)
    M = PH["n_angles"]
    g_true = rng.uniform(0.95, 1.05, M)
    w_true = 3.3
    x_true = phantom_for(config("phantom")).astype(np.float64)
    st = Setup(**{**PH, "fwhm": w_true}, gains=g_true)
    b = _t(to_interleaved(operator.forward(x_true, st)))
    op = FFLOperator(**PH)
    op.set_path("line_gemm")  # W holds no PSF: a new width only replaces the PSF taps
    xj, gj, wj, hist = calibrate(op, b, iters=200, gains0=[1.0] * M, fwhm0=3.0)
    gj = gj.cpu().numpy().astype(np.float64)
    wj = float(wj.cpu().numpy()[0])
    assert len(hist) == 200 and hist[-1] < 0.05 * hist[0], (hist[0], hist[-1])
    assert float(xj.min()) >= 0.0
    err0 = np.max(np.abs(1.0 - g_true / g_true.mean()))
    err = np.max(np.abs(gj / gj.mean() - g_true / g_true.mean()))
    assert err < 0.5 * err0, (err, err0)
    assert abs(wj - w_true) < 0.5 * abs(3.0 - w_true), wj
    op.close()


def test_width_change_off_the_full_gemm_path_rebuilds_w_h_on_return():
    """A new PSF width set while another path is selected leaves W H stale; selecting
    the full-GEMM path again rebuilds it for the new width."""
    from paper_2511_06627_gb300 import FFLOperator

    x = _t(phantom_ellipsoids(GEOM["nx"], GEOM["nz"], seed=7, n_ellipsoids=4, n_points=2))
    op = FFLOperator(**GEOM)
    op.set_path("full_gemm")
    op.forward(x)
    op.set_path("line_gemm")
    op.set_fwhm(3.4)
    b_line = op.forward(x).clone()
    op.set_path("full_gemm")
    b_full = op.forward(x).clone()
    fresh = FFLOperator(**{**GEOM, "fwhm": 3.4})
    fresh.set_path("full_gemm")
    assert torch.equal(b_full, fresh.forward(x))
    st = Setup(**{**GEOM, "fwhm": 3.4})
    ref = to_interleaved(operator.forward(x.cpu().numpy().astype(np.float64), st))
    assert rel_l2(b_full.cpu().numpy(), ref) < OP_TOL
    assert rel_l2(b_line.cpu().numpy(), ref) < OP_TOL
