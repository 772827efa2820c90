"""Pins for the oracle's harmonic-band compression (Sec. 2.1, Appendix A)."""

import cmath
import math

import numpy as np

from oracle import Setup, operator


def _setup(**kw):
    base = dict(nx=8, nz=2, n_angles=2, S=8, P=8, A=2.0, Q=4, fwhm=2.0, k_min=1, k_max=3, half_width=1)
    base.update(kw)
    return Setup(**base)


def test_kept_bins_are_harmonic_bands():
    st = _setup()
    # harmonic k of the drive lies on bin k*P of a P-period line
    assert list(st.bins) == [7, 8, 9, 15, 16, 17, 23, 24, 25]


def test_compression_matches_direct_sum():
    """Eq. (27) evaluated term by term in complex arithmetic (brute force)."""
    st = _setup()
    rng = np.random.default_rng(0)
    sig = rng.standard_normal((1, 1, st.L))
    dg = rng.standard_normal(st.n_bins) + 1j * rng.standard_normal(st.n_bins)
    st.d_gamma = dg
    got = operator.compress_fwd(sig, st)[0, 0]
    L = st.L
    for q, w in enumerate(st.bins):
        acc = 0j
        for j in range(L):
            acc += sig[0, 0, j] * cmath.exp(2j * math.pi * w * j / L)
        assert abs(got[q] - dg[q] * acc / math.sqrt(L)) < 1e-12


def test_parseval_when_all_bins_are_kept():
    """Eq. (28): with every bin kept, ||F s|| = ||s|| and residuals agree."""
    st = _setup(bins=np.arange(64))
    rng = np.random.default_rng(1)
    s1 = rng.standard_normal((2, 2, 64))
    s2 = rng.standard_normal((2, 2, 64))
    b1, b2 = operator.compress_fwd(s1, st), operator.compress_fwd(s2, st)
    assert abs(np.linalg.norm(b1) - np.linalg.norm(s1)) < 1e-12 * np.linalg.norm(s1)
    assert abs(np.linalg.norm(b1 - b2) - np.linalg.norm(s1 - s2)) < 1e-12 * np.linalg.norm(s1 - s2)
    # and the adjoint is the inverse
    np.testing.assert_allclose(operator.compress_adj(b1, st), s1, atol=1e-12)


def test_information_retained_is_bounded_and_monotone():
    """Eq. (30): I(s, S) <= 1, grows with the kept set, equals 1 for all bins."""
    rng = np.random.default_rng(2)
    s = rng.standard_normal(128)
    sets = [np.array([3]), np.array([3, 4, 5]), np.arange(1, 64), np.arange(128)]
    vals = [operator.information_retained(s, b) for b in sets]
    assert all(v <= 1 + 1e-12 for v in vals)
    assert all(vals[i] <= vals[i + 1] + 1e-15 for i in range(3))
    assert abs(vals[-1] - 1.0) < 1e-12


def test_compression_adjoint_dot():
    st = _setup()
    st.d_gamma = np.exp(1j * np.linspace(0, 2, st.n_bins)) * np.linspace(0.5, 1.5, st.n_bins)
    rng = np.random.default_rng(3)
    s = rng.standard_normal((2, 2, st.L))
    y = rng.standard_normal((2, 2, st.n_bins)) + 1j * rng.standard_normal((2, 2, st.n_bins))
    lhs = np.sum((operator.compress_fwd(s, st) * np.conj(y)).real)
    rhs = np.sum(s * operator.compress_adj(y, st))
    assert abs(lhs - rhs) < 1e-12 * np.linalg.norm(s) * np.linalg.norm(y)


def test_pure_harmonic_lands_on_its_bin():
    """A cosine at harmonic k of the drive puts sqrt(L)/2 on bin k*P only."""
    st = _setup()
    L, k = st.L, 2
    j = np.arange(L)
    s = np.cos(2 * math.pi * k * j / st.S)[None, None, :]
    b = operator.compress_fwd(s, st)[0, 0]
    expect = np.zeros(st.n_bins, complex)
    expect[list(st.bins).index(k * st.P)] = math.sqrt(L) / 2
    np.testing.assert_allclose(b, expect, atol=1e-12)


def test_information_retained_closed_forms():
    """Eq. (30) on signals whose spectra are known in closed form.

    A cosine on bin w0 (0 < w0 < L/2) splits its energy equally between bins w0 and
    L - w0, so keeping w0 alone retains exactly 1/sqrt(2) and keeping both retains 1.
    A constant sits on bin 0 alone. For a cos(w1) + c cos(w2), keeping the pair of w1
    retains |a| / sqrt(a^2 + c^2): a ratio of norms, not of energies, which a dropped
    square root would turn into a^2 / (a^2 + c^2)."""
    L, P, k = 96, 8, 3
    j = np.arange(L)
    w0 = k * P
    s = np.cos(2 * math.pi * w0 * j / L + 0.4)
    assert abs(operator.information_retained(s, np.array([w0])) - 1 / math.sqrt(2)) < 1e-12
    assert abs(operator.information_retained(s, np.array([w0, L - w0])) - 1.0) < 1e-12
    assert operator.information_retained(s, np.array([w0 + 1, L - w0 - 1])) < 1e-12
    assert abs(operator.information_retained(np.full(L, 2.5), np.array([0])) - 1.0) < 1e-12
    a, c, w1, w2 = 3.0, 4.0, 2 * P, 5 * P
    s2 = a * np.cos(2 * math.pi * w1 * j / L) + c * np.cos(2 * math.pi * w2 * j / L - 1.1)
    assert abs(operator.information_retained(s2, np.array([w1, L - w1])) - 0.6) < 1e-12
    assert abs(operator.information_retained(s2, np.array([w2, L - w2])) - 0.8) < 1e-12
    assert abs(operator.information_retained(s2, np.array([w1])) - 0.6 / math.sqrt(2)) < 1e-12
