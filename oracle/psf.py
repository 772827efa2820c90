"""Langevin-derivative PSF along the drive axis (oracle, float64).

Appendix B gives the Langevin function L(x) = coth(x) - 1/x and the tensor
PSF, Eq. (31), whose collinear (drive/receive along the same axis) term is
L'(|Gx|/H_sat). Reading used here for a 1D drive along u: h(u) = 3 L'(u/a),
normalised to h(0) = 1 (L'(0) = 1/3), with a chosen so that the full width
at half maximum is `fwhm` voxels. The absolute scale (m, beta, G in Eq. (7))
is absorbed into the per-angle gain.

L'(x) = 1/x^2 - 1/sinh(x)^2; for |x| < 0.05 the Taylor series
1/3 - x^2/15 + 2x^4/189 - x^6/675 avoids the cancellation.
The PSF is never truncated: L' decays like 1/x^2.
"""

import numpy as np
from scipy.optimize import brentq


def langevin(x):
    """L(x) = coth(x) - 1/x (Appendix B), with its series near 0."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = np.abs(x) < 1e-3
    xs = x[small]
    out[small] = xs / 3.0 - xs**3 / 45.0
    xl = x[~small]
    out[~small] = 1.0 / np.tanh(xl) - 1.0 / xl
    return out


def langevin_deriv(x):
    """L'(x) = 1/x^2 - 1/sinh(x)^2."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    ax = np.abs(x)
    small = ax < 0.05
    x2 = x[small] ** 2
    out[small] = 1.0 / 3.0 - x2 / 15.0 + 2.0 * x2**2 / 189.0 - x2**3 / 675.0
    xl = ax[~small]
    with np.errstate(over="ignore"):
        sh = np.sinh(xl)
        out[~small] = 1.0 / (xl * xl) - 1.0 / (sh * sh)
    return out


def half_max_point():
    """x_h > 0 with L'(x_h) = L'(0)/2 = 1/6."""
    return brentq(lambda x: float(langevin_deriv(np.array([x]))[0]) - 1.0 / 6.0, 0.5, 5.0, xtol=1e-15)


def width_scale(fwhm):
    """a such that h(u) = 3 L'(u/a) has full width at half maximum fwhm."""
    return fwhm / (2.0 * half_max_point())


def h(u, fwhm):
    """PSF value at offset u (voxels)."""
    return 3.0 * langevin_deriv(np.asarray(u, dtype=np.float64) / width_scale(fwhm))


def dh_dfwhm(u, fwhm, eps=None):
    """d h(u) / d fwhm, analytically: h = 3 L'(u/a), a = fwhm/(2 x_h).

    dh/dfwhm = 3 L''(u/a) * (-u/a^2) * da/dfwhm = -3 L''(u/a) (u/a) / fwhm,
    with L''(x) = -2/x^3 + 2 cosh(x)/sinh(x)^3 (series -2x/15 + 8x^3/189 - 6x^5/675 near 0).
    """
    a = width_scale(fwhm)
    x = np.asarray(u, dtype=np.float64) / a
    out = np.empty_like(x)
    small = np.abs(x) < 0.05
    xs = x[small]
    out[small] = -2.0 * xs / 15.0 + 8.0 * xs**3 / 189.0 - 6.0 * xs**5 / 675.0
    xl = x[~small]
    with np.errstate(over="ignore", invalid="ignore"):
        sh = np.sinh(xl)
        val = -2.0 / xl**3 + 2.0 * np.cosh(xl) / sh**3
    val = np.where(np.abs(xl) > 350, -2.0 / xl**3, val)
    out[~small] = val
    return -3.0 * out * x / fwhm
