"""Pins of the tensor-PSF and coil-map oracle (Appendix B Eq. (31), operator B of
Eq. (13)), each against something other than the oracle itself: closed forms of the
Langevin function computed here with `math`, far-field asymptotes, the 1D model on
the drive axis, a point source, and adjoint identities."""

import math

import numpy as np
import pytest

from oracle import Setup, operator, psf, tensor_psf, trajectory

SMALL = dict(nx=16, nz=10, n_angles=3, S=32, P=16, A=3.0, phi0=0.3, zigzag=1, Q=8, fwhm=2.0,
             k_min=1, k_max=4, half_width=2)


def _setup(**over):
    kw = dict(SMALL)
    kw.update(over)
    return Setup(**kw)


def _coth(x):
    return math.cosh(x) / math.sinh(x)


def _ld(x):  # L'(x) = 1/x^2 - 1/sinh(x)^2, from its definition
    return 1.0 / x**2 - 1.0 / math.sinh(x) ** 2


def _l(x):  # L(x) = coth(x) - 1/x
    return _coth(x) - 1.0 / x


def test_peak_is_one():
    assert tensor_psf.h_uu(0.0, 0.0, 2.5) == 1.0


@pytest.mark.parametrize("fwhm", [1.5, 3.0])
def test_drive_axis_is_the_1d_psf(fwhm):
    u = np.linspace(-40, 40, 801)
    assert np.allclose(tensor_psf.h_uu(u, 0.0, fwhm), psf.h(u, fwhm), rtol=1e-14, atol=0)


@pytest.mark.parametrize("k", [0.5, 1.0, 2.0, 7.0])
def test_transverse_axis_closed_form(k):
    """u = 0: only the transverse eigenvalue, 3 L(xi)/xi, at z = k a."""
    fwhm = 2.0
    a = psf.width_scale(fwhm)
    assert math.isclose(float(tensor_psf.h_uu(0.0, k * a, fwhm)), 3.0 * _l(k) / k, rel_tol=1e-13)
    if k == 1.0:  # 3 (coth 1 - 1), with coth 1 = (e^2 + 1)/(e^2 - 1)
        e2 = math.e**2
        assert math.isclose(float(tensor_psf.h_uu(0.0, a, fwhm)), 3.0 * ((e2 + 1) / (e2 - 1) - 1), rel_tol=1e-13)


def test_far_field_asymptotes():
    """L -> 1 gives 3a/|z| across the drive axis; L' ~ 1/xi^2 gives 3a^2/u^2 along it."""
    fwhm = 2.0
    a = psf.width_scale(fwhm)
    for r in (1e3, 1e4):
        assert math.isclose(float(tensor_psf.h_uu(0.0, r, fwhm)) * r / (3 * a), 1.0, rel_tol=2 * a / r)
        assert math.isclose(float(tensor_psf.h_uu(r, 0.0, fwhm)) * r * r / (3 * a * a), 1.0, rel_tol=1e-9)


@pytest.mark.parametrize("r", [0.7, 2.0, 5.5])
def test_diagonal_is_the_mean_of_the_axes(r):
    """At 45 degrees u^2/rho^2 = z^2/rho^2 = 1/2."""
    fwhm = 2.0
    a = psf.width_scale(fwhm)
    x = r / a
    want = 1.5 * (_ld(x) + _l(x) / x)
    assert math.isclose(float(tensor_psf.h_uu(r / math.sqrt(2), r / math.sqrt(2), fwhm)), want, rel_tol=1e-12)


def test_tensor_eigenpairs_and_rotation_invariance():
    fwhm = 2.0
    a = psf.width_scale(fwhm)
    rng = np.random.default_rng(3)
    for _ in range(20):
        u, z = rng.uniform(-6, 6, 2)
        uu, uz, zz = (float(t) for t in tensor_psf.tensor_inplane(u, z, fwhm))
        rho = math.hypot(u, z)
        w, V = np.linalg.eigh(np.array([[uu, uz], [uz, zz]]))
        want = sorted([3 * _ld(rho / a), 3 * _l(rho / a) / (rho / a)])
        assert np.allclose(w, want, rtol=1e-12)
        ev_col = V[:, int(np.argmin(np.abs(w - 3 * _ld(rho / a))))]
        assert math.isclose(abs(ev_col @ np.array([u, z])) / rho, 1.0, rel_tol=1e-9)
        th = rng.uniform(0, 2 * math.pi)  # the trace depends on rho only
        ur, zr = u * math.cos(th) - z * math.sin(th), u * math.sin(th) + z * math.cos(th)
        uu2, _, zz2 = (float(t) for t in tensor_psf.tensor_inplane(ur, zr, fwhm))
        assert math.isclose(uu + zz, uu2 + zz2, rel_tol=1e-12)


def test_series_branch_meets_the_closed_form():
    for x in (0.0499999, 0.0500001, 0.03):
        direct = (_coth(x) - 1 / x) / x
        assert math.isclose(float(tensor_psf.langevin_over_x(x)), direct, rel_tol=1e-9)


def test_single_slice_gives_the_1d_line_signal():
    """A projection on slice z0 only: line z0 sees h_uu(., 0), the 1D PSF."""
    st = _setup()
    rng = np.random.default_rng(4)
    proj = np.zeros((2, st.nz, st.nx))
    proj[:, 4] = rng.random((2, st.nx))
    ang = np.array([0, 1])
    s2 = operator.resample_fwd(tensor_psf.psf_fwd_2d(proj, st), st, ang)
    s1 = operator.resample_fwd(operator.psf_fwd(proj, st), st, ang)
    assert np.allclose(s2[:, 4], s1[:, 4], rtol=1e-12, atol=1e-15)
    assert np.abs(s2[:, 6]).max() > 0.05 * np.abs(s2[:, 4]).max()  # other lines see it too


def _uu_second_derivative_bound(d, fwhm):
    u = np.linspace(-40, 40, 160001)
    hh = tensor_psf.h_uu(u, float(d), fwhm)
    return np.abs(np.gradient(np.gradient(hh, u), u)).max()


@pytest.mark.parametrize("line", [2, 5, 6, 9])
def test_point_source_signal_is_the_shifted_tensor_psf(line):
    """Unit projection at (z0, u0): line l's signal is g v_j h_uu(xi_j - u0, l - z0),
    within max|d^2 h/du^2| / (8 Q^2) of the fine-grid interpolation."""
    st = _setup(gains=np.array([1.3, 1.0, 1.0]))
    z0, u0 = 5, 7
    proj = np.zeros((1, st.nz, st.nx))
    proj[0, z0, u0] = 1.0
    sig = operator.resample_fwd(tensor_psf.psf_fwd_2d(proj, st), st, np.array([0]))[0, line]
    xi, v = trajectory.line_positions(st, line)
    ref = 1.3 * v * tensor_psf.h_uu(xi - u0, line - z0, st.fwhm)
    bound = 1.3 * np.abs(v) * _uu_second_derivative_bound(line - z0, st.fwhm) / (8 * st.Q**2) + 1e-13
    assert np.all(np.abs(sig - ref) <= bound)


def test_coil_map_weights_the_source_slice():
    """b multiplies the source (z', i), not the line being read: a point source seen
    through b = 2 at its own position doubles on every line, and b = 0 there removes it."""
    st = _setup()
    x = np.zeros((st.nz, st.nx, st.nx))
    x[5, 7, 8] = 1.0
    base = tensor_psf.forward_stages(x, st, None, angles=np.array([0]))
    proj = base["proj"][0]
    src = proj != 0
    b2 = np.where(src, 2.0, 5.0)
    doubled = tensor_psf.forward_stages(x, st, b2, angles=np.array([0]))["data"]
    assert np.allclose(doubled, 2.0 * base["data"], rtol=1e-12, atol=1e-14)
    b0 = np.where(src, 0.0, 1.0)
    assert np.abs(tensor_psf.forward_stages(x, st, b0, angles=np.array([0]))["data"]).max() < 1e-14
    assert np.abs(base["data"]).max() > 1e-3


def test_reflection_in_z_reflects_the_lines():
    """h_uu is even in z: without zig-zag, reversing the slices reverses c's lines."""
    st = _setup(zigzag=0)
    rng = np.random.default_rng(5)
    p = rng.standard_normal((2, st.nz, st.nx))
    c = tensor_psf.psf_fwd_2d(p, st)
    cr = tensor_psf.psf_fwd_2d(p[:, ::-1], st)
    assert np.allclose(cr, c[:, ::-1], rtol=1e-12, atol=1e-13)


def test_stage_and_operator_adjoints():
    st = _setup(gains=np.array([0.9, 1.1, 1.0]))
    rng = np.random.default_rng(6)
    p = rng.standard_normal((2, st.nz, st.nx))
    c = rng.standard_normal((2, st.nz, st.n_fine))
    assert math.isclose(np.vdot(tensor_psf.psf_fwd_2d(p, st), c), np.vdot(p, tensor_psf.psf_adj_2d(c, st)),
                        rel_tol=1e-12)
    coil = rng.uniform(0.5, 1.5, (st.nz, st.nx))
    x = rng.random((st.nz, st.nx, st.nx))
    y = rng.standard_normal(st.data_shape) + 1j * rng.standard_normal(st.data_shape)
    lhs = np.sum(np.real(tensor_psf.forward(x, st, coil) * np.conj(y)))
    rhs = np.sum(x * tensor_psf.adjoint(y, st, coil))
    assert math.isclose(lhs, rhs, rel_tol=1e-12)
