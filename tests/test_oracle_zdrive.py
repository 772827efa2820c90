"""Pins of the z-drive scan in the oracle (Sec. 3.1, dual drive axes), each against
something other than the oracle itself: a closed-form point-source signal within the
fine-grid interpolation bound, exact translation along z, and adjoint identities of
every stage (literal transposes built independently by scatter)."""

import numpy as np
import pytest

from oracle import Setup, psf, zdrive

SMALL = dict(nx=16, nz=12, n_angles=3, S=32, P=16, A=3.0, phi0=0.3, zigzag=1, Q=8, fwhm=2.0,
             k_min=1, k_max=4, half_width=2)


def _setup(**over):
    kw = dict(SMALL)
    kw.update(over)
    return Setup(**kw)


def _h2_bound(fwhm, Q):
    # max |h''| on a fine grid, times 1/(8 Q^2): the linear-interpolation error bound
    x = np.linspace(-40, 40, 200001)
    d2 = np.gradient(np.gradient(psf.h(x, fwhm), x), x)
    return np.abs(d2).max() / (8.0 * Q * Q)


@pytest.mark.parametrize("line", [3, 5, 6])
def test_point_source_signal_is_the_shifted_psf(line):
    """A unit projection value at (z0, u0): the z-drive signal of a line is
    v_j (1 - |c_j - u0|)_+ h(l + zeta_j - z0), within max|h''| / (8 Q^2)."""
    st = _setup()
    z0, u0 = 5, 7
    proj = np.zeros((1, st.nz, st.nx))
    proj[0, z0, u0] = 1.0
    sig = zdrive.resample_fwd_z(zdrive.psf_fwd_z(proj, st), st, angles=np.array([0]))[0, line]
    c = zdrive.slow_positions(st, line)
    zeta, v = zdrive.drive_positions(st)
    ref = v * np.maximum(0.0, 1.0 - np.abs(c - u0)) * psf.h(line + zeta - z0, st.fwhm)
    wu = np.maximum(0.0, 1.0 - np.abs(c - u0))
    bound = _h2_bound(st.fwhm, st.Q) * np.abs(v) * wu + 1e-12
    assert np.all(np.abs(sig - ref) <= bound)
    assert np.abs(sig).max() > 0.1  # the line passes near the source


def test_shift_by_two_slices_shifts_the_signal_by_two_lines():
    """Translating the projection by two slices along z (one zig-zag period of the
    raster) moves the signal by two lines, exactly, where the grid edge does not cut."""
    st = _setup(nz=16)
    rng = np.random.default_rng(1)
    p = np.zeros((1, st.nz, st.nx))
    p[0, 4:9] = rng.random((5, st.nx))
    q = np.roll(p, 2, axis=1)
    s_p = zdrive.resample_fwd_z(zdrive.psf_fwd_z(p, st), st, angles=np.array([0]))[0]
    s_q = zdrive.resample_fwd_z(zdrive.psf_fwd_z(q, st), st, angles=np.array([0]))[0]
    for line in range(2, 12):
        assert np.allclose(s_q[line], s_p[line - 2], rtol=1e-12, atol=1e-14)


def test_stage_adjoints():
    st = _setup()
    rng = np.random.default_rng(2)
    p = rng.standard_normal((2, st.nz, st.nx))
    c = rng.standard_normal((2, st.nx, zdrive.n_fine_z(st)))
    assert np.isclose(np.vdot(zdrive.psf_fwd_z(p, st), c), np.vdot(p, zdrive.psf_adj_z(c, st)), rtol=1e-12)
    s = rng.standard_normal((2, st.nz, st.L))
    ang = np.array([0, 1])
    lhs = np.vdot(zdrive.resample_fwd_z(c, st, ang), s)
    rhs = np.vdot(c, zdrive.resample_adj_z(s, st, ang))
    assert np.isclose(lhs, rhs, rtol=1e-12)


def test_operator_adjoint_identity():
    st = _setup(gains=np.array([0.9, 1.1, 1.0]))
    rng = np.random.default_rng(3)
    x = rng.random((st.nz, st.nx, st.nx))
    y = rng.standard_normal(st.data_shape) + 1j * rng.standard_normal(st.data_shape)
    lhs = np.sum(np.real(zdrive.forward_z(x, st) * np.conj(y)))
    rhs = np.sum(x * zdrive.adjoint_z(y, st))
    assert np.isclose(lhs, rhs, rtol=1e-12)


def test_columns_outside_the_detector_read_zero():
    """The u read stays on the detector: a projection that is zero except in the last
    column gives no signal where the slow position is below N - 2."""
    st = _setup()
    p = np.zeros((1, st.nz, st.nx))
    p[0, :, st.nx - 1] = 1.0
    sig = zdrive.resample_fwd_z(zdrive.psf_fwd_z(p, st), st, angles=np.array([0]))[0, 0]
    c = zdrive.slow_positions(st, 0)
    assert np.all(sig[c < st.nx - 2] == 0.0)
