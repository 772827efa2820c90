"""Pins for the oracle's PSF (Appendix B, Eq. (31)) and trajectory (Eqs. (3)-(4), (7))."""

import math

import numpy as np
import pytest

from oracle import Setup, operator, psf, trajectory


def test_langevin_derivative_matches_numerical_derivative():
    """L'(x) against a central difference of L(x) = coth x - 1/x (Appendix B)."""
    x = np.concatenate([np.linspace(-8, -0.06, 50), np.linspace(0.051, 8, 50), [0.049, -0.03, 0.2]])
    h = 1e-5
    num = (psf.langevin(x + h) - psf.langevin(x - h)) / (2 * h)
    np.testing.assert_allclose(psf.langevin_deriv(x), num, rtol=2e-8, atol=1e-10)


def test_langevin_derivative_series_branch_is_continuous():
    x = np.array([0.05 - 1e-12, 0.05 + 1e-12])
    v = psf.langevin_deriv(x)
    assert abs(v[0] - v[1]) < 1e-12
    assert abs(float(psf.langevin_deriv(np.array([0.0]))[0]) - 1.0 / 3.0) < 1e-15


@pytest.mark.parametrize("fwhm", [2.0, 3.0, 4.5])
def test_psf_peak_and_half_width(fwhm):
    u = np.array([0.0, fwhm / 2, -fwhm / 2])
    v = psf.h(u, fwhm)
    np.testing.assert_allclose(v, [1.0, 0.5, 0.5], atol=1e-12)
    uu = np.linspace(0.01, 40, 400)
    np.testing.assert_allclose(psf.h(uu, fwhm), psf.h(-uu, fwhm), rtol=1e-14)
    assert (np.diff(psf.h(uu, fwhm)) < 0).all()


def test_psf_tail_is_inverse_square():
    # L'(x) -> 1/x^2, so h(u) -> 3 a^2 / u^2 far out: no truncation anywhere
    a = psf.width_scale(3.0)
    u = np.array([100.0, 300.0])
    np.testing.assert_allclose(psf.h(u, 3.0), 3 * a * a / u**2, rtol=1e-12)


def test_dh_dfwhm_matches_finite_difference():
    u = np.linspace(-30, 30, 241)
    for fwhm in (2.0, 3.0):
        e = 1e-6
        num = (psf.h(u, fwhm + e) - psf.h(u, fwhm - e)) / (2 * e)
        np.testing.assert_allclose(psf.dh_dfwhm(u, fwhm), num, rtol=1e-6, atol=1e-9)


def _small_setup(**kw):
    base = dict(nx=24, nz=2, n_angles=1, S=32, P=16, A=5.0, Q=8, fwhm=2.0, k_min=1, k_max=4, half_width=2)
    base.update(kw)
    return Setup(**base)


def test_velocity_is_derivative_of_position():
    st = _small_setup()
    for line in (0, 1):
        xi, v = trajectory.line_positions(st, line)
        cd = (xi[2:] - xi[:-2]) / 2.0
        # central difference error <= A (2 pi / S)^3 / 6
        bound = st.A * (2 * math.pi / st.S) ** 3 / 6 + 1e-12
        assert np.abs(cd - v[1:-1]).max() <= bound


def test_zigzag_reverses_slow_sweep():
    st = _small_setup()
    xi0, _ = trajectory.line_positions(st, 0)
    xi1, _ = trajectory.line_positions(st, 1)
    j = np.arange(st.L)
    drive = st.A * np.sin(2 * math.pi * j / st.S)
    np.testing.assert_allclose(xi0 + xi1 - 2 * drive, st.nx - 1, atol=1e-12)
    assert abs(xi0[0] - 0.0) < 1e-12 and abs(xi0[-1] - drive[-1] - (st.nx - 1)) < 1e-12


def test_fine_index_stays_on_grid():
    st = _small_setup(A=6.0)
    for line in (0, 1):
        xi, _ = trajectory.line_positions(st, line)
        n, f = trajectory.fine_index(st, xi)
        assert n.min() >= 0 and n.max() <= st.n_fine - 2
        assert f.min() >= 0 and f.max() <= 1.0 + 1e-12
        np.testing.assert_allclose(n + f, st.Q * xi + st.D, atol=1e-9)


@pytest.mark.parametrize("Q", [8, 16])
def test_point_source_reproduces_psf(Q):
    """A delta at bin i0 gives s_j / (g v_j) = h(xi_j - i0) within max|h''| / (8 Q^2)."""
    st = _small_setup(Q=Q, fwhm=2.0)
    i0 = 9
    vol = np.zeros((st.nz, st.nx, st.nx))
    vol[:, 4, i0] = 1.0  # theta = 0 projects column x = i0 onto bin i0
    stages = operator.forward_stages(vol, st)
    np.testing.assert_allclose(stages["proj"][0, :, i0], 1.0, atol=1e-14)
    for line in range(st.nz):
        xi, v = trajectory.line_positions(st, line)
        ratio = stages["sig"][0, line] / v
        ok = np.abs(v) > 1e-3
        uu = np.linspace(-5, 5, 20001)
        a = psf.width_scale(2.0)
        hpp = np.abs(np.gradient(np.gradient(psf.h(uu, 2.0), uu), uu)).max()
        err = np.abs(ratio[ok] - psf.h(xi[ok] - i0, 2.0))
        assert err.max() <= hpp / (8 * Q * Q) * 1.01
        assert a > 0
    # exact where Q xi is an integer: the fine grid holds h itself
    fine = stages["fine"][0, 0]
    e = np.arange(st.n_fine)
    np.testing.assert_allclose(fine, psf.h((e - st.D) / st.Q - i0, 2.0), rtol=1e-14, atol=1e-15)
