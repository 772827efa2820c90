"""Finite-difference regulariser T (oracle, float64).

Sec. 3.3, Eq. (25) names T a finite-difference operator without fixing its
form. Reading used here: first-order forward differences along x, y and z,
(T_d x)[v] = x[v + e_d] - x[v] for every v whose neighbour lies inside the
volume (no wrap-around, i.e. Neumann boundary). T^T T is then the 7-point
negative Laplacian with a reduced diagonal on the faces.
"""

import math

import numpy as np


def apply_t(x):
    """T x as a list of three difference arrays (axis 0 = z, 1 = y, 2 = x)."""
    x = np.asarray(x, dtype=np.float64)
    return [np.diff(x, axis=a) for a in range(3)]


def apply_tt(d_list, shape):
    """T^T applied to the three difference arrays."""
    out = np.zeros(shape)
    for a, d in enumerate(d_list):
        pad_lo = [(0, 0)] * 3
        pad_hi = [(0, 0)] * 3
        pad_lo[a] = (1, 0)
        pad_hi[a] = (0, 1)
        # (T^T d)[i] = d[i-1] - d[i], with d[-1] = d[n-1] = 0
        out += np.pad(d, pad_lo) - np.pad(d, pad_hi)
    return out


def ttt(x):
    """T^T T x."""
    x = np.asarray(x, dtype=np.float64)
    return apply_tt(apply_t(x), x.shape)


def ttt_norm(shape):
    """||T^T T||_2 = sum_d 4 sin^2(pi (n_d - 1) / (2 n_d)) (Kronecker sum of 1D Neumann Laplacians)."""
    return sum(4.0 * math.sin(math.pi * (n - 1) / (2.0 * n)) ** 2 for n in shape)
