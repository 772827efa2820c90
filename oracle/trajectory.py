"""FFL trajectory along the drive axis (oracle, float64).

Sec. 1.2, Eqs. (3)-(4): a sinusoidal drive moves the field-free line,
xi(t) = slow(t) + A sin(2 pi f0 t + phi0); Eq. (7) weights the signal by the
velocity v = xi'. Sec. 3.1: a slow raster moves back and forth along the
drive axis (zig-zag) and steps slowly in z.

Reading used here: one raster line per z slice, sampled at j = 0..L-1 with
S samples per drive period. The slow part sweeps the detector from bin 0 to
bin N-1, c_j = (N-1) j / (L-1), reversed on odd lines when zig-zag is on; the
step between lines is instantaneous and not sampled. Positions are in
detector-bin units; velocity is in bins per sample.
"""

import numpy as np


def line_positions(setup, line):
    """(xi_j, v_j) for j = 0..L-1 on raster line `line`."""
    L, n = setup.L, setup.nx
    j = np.arange(L, dtype=np.float64)
    slope = (n - 1) / (L - 1)
    if setup.zigzag and line % 2 == 1:
        slow = (n - 1) - slope * j
        dslow = -slope
    else:
        slow = slope * j
        dslow = slope
    phase = 2.0 * np.pi * j / setup.S + setup.phi0
    xi = slow + setup.A * np.sin(phase)
    v = dslow + setup.A * (2.0 * np.pi / setup.S) * np.cos(phase)
    return xi, v


def fine_index(setup, xi):
    """Fine-grid interpolation cell n and fraction f for positions xi.

    t = (xi - u_lo) Q = Q xi + D; n = min(floor(t), N_e - 2), f = t - n, so the
    right end of the grid is reached with f = 1.
    """
    t = setup.Q * xi + setup.D
    n = np.minimum(np.floor(t), setup.n_fine - 2).astype(np.int64)
    if (n < 0).any() or (t > setup.n_fine - 1 + 1e-9).any():
        raise ValueError("trajectory leaves the fine grid")
    return n, t - n
