"""Parallel-beam projection P_theta and its transpose (oracle, float64).

Sec. 2.2, Eqs. (16)-(17): rho_theta(x, z) = integral of rho((x, y) Q_theta^T, z) dy
with Q_theta = [[cos, sin], [-sin, cos]]. For object-plane coordinates
(X, Y) measured from the volume centre c = (N-1)/2, the point (x, y)Q_theta^T
is (x cos + y sin, -x sin + y cos): the ray through detector position u runs
along d = (sin, cos) and u = X cos - Y sin.

Eq. (19) only says that P_theta is a sparse Riemann-sum operator. Reading
used here (Joseph's method): if |cos| >= |sin| (within 1e-9, ties go this
way) the ray is marched row by row; in row y_r the x position is
f = u/cos + (y_r - c) tan + c and the voxel row is sampled by linear
interpolation, the sum scaled by 1/|cos|. Otherwise it is marched column by
column with f = -u/sin + (x_c - c) cot + c and scale 1/|sin|. Interpolation
uses hat weights max(0, 1 - |f - k|) over k = 0..N-1 (zero outside the grid).
Detector bins i = 0..N-1 sit at u_i = i - c.
"""

import numpy as np


def row_major(theta):
    """True when the ray is marched along rows (|cos| >= |sin| up to 1e-9)."""
    return abs(np.cos(theta)) >= abs(np.sin(theta)) - 1e-9


def _hat(f, n):
    """Indices and weights of hat interpolation at positions f on 0..n-1.

    Returns (k0, w0, k1, w1) with invalid neighbours given weight 0 and a
    clamped index, so that value = w0*a[k0] + w1*a[k1].
    """
    k = np.floor(f)
    t = f - k
    k = k.astype(np.int64)
    k0, k1 = k, k + 1
    w0 = np.where((k0 >= 0) & (k0 < n), 1.0 - t, 0.0)
    w1 = np.where((k1 >= 0) & (k1 < n), t, 0.0)
    return np.clip(k0, 0, n - 1), w0, np.clip(k1, 0, n - 1), w1


def _rays(theta, n):
    """Per march step s: interpolation positions f[s, i] along the step's voxel line.

    Returns (row_major, f, scale).
    """
    c = (n - 1) / 2.0
    u = np.arange(n) - c
    cs, sn = np.cos(theta), np.sin(theta)
    steps = np.arange(n, dtype=np.float64)[:, None] - c
    if row_major(theta):
        f = u[None, :] / cs + steps * (sn / cs) + c
        return True, f, 1.0 / abs(cs)
    f = -u[None, :] / sn + steps * (cs / sn) + c
    return False, f, 1.0 / abs(sn)


def project(vol, thetas):
    """P: vol[z][y][x] -> proj[m][z][i] (Sec. 2.2, Eq. (19))."""
    vol = np.asarray(vol, dtype=np.float64)
    nz, n, n2 = vol.shape
    assert n == n2
    out = np.zeros((len(thetas), nz, n))
    for m, th in enumerate(thetas):
        rm, f, scale = _rays(th, n)
        acc = np.zeros((nz, n))
        for s in range(n):
            k0, w0, k1, w1 = _hat(f[s], n)
            line = vol[:, s, :] if rm else vol[:, :, s]  # row y=s, or column x=s
            acc += w0 * line[:, k0] + w1 * line[:, k1]
        out[m] = acc * scale
    return out


def backproject(proj, thetas, n):
    """P^T: proj[m][z][i] -> vol[z][y][x], the literal transpose (scatter form)."""
    proj = np.asarray(proj, dtype=np.float64)
    nz = proj.shape[1]
    vol = np.zeros((nz, n, n))
    for m, th in enumerate(thetas):
        rm, f, scale = _rays(th, n)
        pm = proj[m] * scale
        for s in range(n):
            k0, w0, k1, w1 = _hat(f[s], n)
            line = np.zeros((nz, n))
            np.add.at(line, (slice(None), k0), pm * w0)
            np.add.at(line, (slice(None), k1), pm * w1)
            if rm:
                vol[:, s, :] += line
            else:
                vol[:, :, s] += line
    return vol


def matrix(thetas, n):
    """Dense P for one z slice, shape [M*n, n*n] (tiny grids only)."""
    cols = []
    for v in range(n * n):
        e = np.zeros((1, n, n))
        e.reshape(-1)[v] = 1.0
        cols.append(project(e, thetas).reshape(-1))
    return np.stack(cols, axis=1)
