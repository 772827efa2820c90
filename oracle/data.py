"""Noisy compressed data for the synthetic workloads (oracle side).

Noise: white Gaussian in time with sigma = `noise` x max|s_j| of the
noiseless signal. Because F is unitary (Appendix A, Eq. (28)), on the kept
bins (0 < omega < L/2) this is complex Gaussian with variance sigma^2/2 per
real component, independent across bins, so it is drawn there directly.

Nonidealities of the phantom-scale workload (Sec. 1, amplifier drift and
coil gain): per-angle gains U(1 - s, 1 + s) and a slow linear baseline
a_m + b_m (line*L + j)/(N_z L) in time, with a_m, b_m ~ U(-d, d) x peak.
They enter the data only; the plain solve does not model them.
"""

import numpy as np

from . import operator
from .setup import Setup


def make_data(setup, x_true, noise, seed=0, gain_spread=0.0, drift=0.0):
    """Return (b, info) with b complex [M][N_z][n_bins]."""
    rng = np.random.default_rng(seed + 7919)
    true = Setup(**{k: getattr(setup, k) for k in (
        "nx", "nz", "n_angles", "S", "P", "A", "phi0", "zigzag", "Q", "fwhm",
        "k_min", "k_max", "half_width")}, angles=setup.angles, bins=setup.bins,
        d_gamma=setup.d_gamma)
    if gain_spread > 0.0:
        true.gains = rng.uniform(1.0 - gain_spread, 1.0 + gain_spread, size=setup.n_angles)
    else:
        true.gains = setup.gains.copy()
    b = operator.forward(x_true, true)
    peak = operator.max_abs_signal(x_true, true)
    if drift > 0.0:
        L = setup.L
        for m in range(setup.n_angles):
            a_m, b_m = rng.uniform(-drift, drift, size=2) * peak
            j = np.arange(L, dtype=np.float64)
            lines = np.arange(setup.nz, dtype=np.float64)[:, None]
            sig = a_m + b_m * (lines * L + j[None, :]) / (setup.nz * L)
            b[m] += operator.compress_fwd(sig, setup)
    sigma = noise * peak
    if sigma > 0.0:
        b = b + (rng.standard_normal(b.shape) + 1j * rng.standard_normal(b.shape)) * (sigma / np.sqrt(2.0))
    return b, dict(peak=peak, sigma=sigma, gains=true.gains)


def to_interleaved(b):
    """complex [..., q] -> float [..., q, 2] (re, im)."""
    b = np.asarray(b)
    return np.stack([b.real, b.imag], axis=-1)


def from_interleaved(a):
    a = np.asarray(a, dtype=np.float64)
    return a[..., 0] + 1j * a[..., 1]
