"""The z-drive scan of the dual-drive acquisition (oracle, float64).

Sec. 3.1: at every projection angle the scanner acquires two scans, one with the
drive field along x and one along z. The x-drive scan is A of operator.py; this
module adds the z-drive scan A_z. The dual-drive operator is [A; A_z] (data
stacked) with transpose A^T y + A_z^T y_z.

Readings (the paper gives the scanner's raster and the two drive axes, not the
z-drive signal model):
  - Same raster as the x-drive scan: line l is the z slice l, the slow position
    c_j sweeps the detector from bin 0 to N-1 (reversed on odd lines with
    zig-zag), with the same S, P, A and phase.
  - The drive moves the FFL along z: sample j of line l sits at
    (u, z) = (c_j, l + A sin(2 pi j / S + phi0)), and the velocity along the drive
    axis is v_j = A (2 pi / S) cos(2 pi j / S + phi0) (the slow raster moves along
    u only; the step between lines is instantaneous).
  - The PSF is the same Langevin derivative h (Appendix B, collinear drive and
    receive), now along z, with full support over the z slices of the projection.
  - As for the x drive, the PSF-convolved projection is evaluated on a grid Q
    times finer than the slices, z_lo + e/Q with z_lo = -D/Q, e = 0..N_ez-1,
    N_ez = (N_z - 1) Q + 2 D + 1, and read by linear interpolation: along z at
    t = Q z + D (cell n = min(floor t, N_ez - 2), fraction t - n), along u between
    the detector bins floor(c_j) and floor(c_j) + 1 (zero outside the detector).
  - The z-drive data are compressed exactly like the x-drive data (same kept bins,
    D_Gamma and gains).
"""

import numpy as np

from . import operator, psf


def n_fine_z(setup):
    return (setup.nz - 1) * setup.Q + 2 * setup.D + 1


def slow_positions(setup, line):
    """c_j: the slow raster position along u on raster line `line`."""
    L, n = setup.L, setup.nx
    j = np.arange(L, dtype=np.float64)
    slope = (n - 1) / (L - 1)
    if setup.zigzag and line % 2 == 1:
        return (n - 1) - slope * j
    return slope * j


def drive_positions(setup):
    """(zeta_j, v_j): offset of the FFL along z from its line, and its velocity."""
    j = np.arange(setup.L, dtype=np.float64)
    phase = 2.0 * np.pi * j / setup.S + setup.phi0
    return setup.A * np.sin(phase), setup.A * (2.0 * np.pi / setup.S) * np.cos(phase)


# ----------------------------------------------------------------------------- H_z

def psf_matrix_z(setup, fwhm=None):
    """H_z as a dense [N_ez, N_z] matrix: H_z[e, z'] = h(z_lo + e/Q - z')."""
    fwhm = setup.fwhm if fwhm is None else fwhm
    e = np.arange(n_fine_z(setup), dtype=np.float64)
    zs = np.arange(setup.nz, dtype=np.float64)
    return psf.h((e[:, None] - setup.D) / setup.Q - zs[None, :], fwhm)


def psf_fwd_z(proj, setup):
    """cz[m, u, e] = sum_z' proj[m, z', u] h(z_lo + e/Q - z')."""
    proj = np.asarray(proj, dtype=np.float64)
    return np.einsum("mzu,ez->mue", proj, psf_matrix_z(setup), optimize=True)


def psf_adj_z(cz, setup):
    cz = np.asarray(cz, dtype=np.float64)
    return np.einsum("mue,ez->mzu", cz, psf_matrix_z(setup), optimize=True)


# ----------------------------------------------------------------------------- E_z V_z B

def _line_tables(setup, line):
    """Bilinear read of line `line`: u cell and weight, z cell and weight, velocity."""
    c = slow_positions(setup, line)
    u0 = np.floor(c).astype(np.int64)
    a = c - u0
    zeta, v = drive_positions(setup)
    t = setup.Q * (line + zeta) + setup.D
    n = np.minimum(np.floor(t), n_fine_z(setup) - 2).astype(np.int64)
    if (n < 0).any() or (t > n_fine_z(setup) - 1 + 1e-9).any():
        raise ValueError("z trajectory leaves the fine grid")
    return u0, a, n, t - n, v


def resample_fwd_z(cz, setup, angles=None):
    """s[m, l, j] = g_m v_j bilinear(cz[m], (c_j, t_j)); columns outside [0, N) read 0."""
    cz = np.asarray(cz, dtype=np.float64)
    M = cz.shape[0]
    N = setup.nx
    gains = setup.gains if angles is None else setup.gains[angles]
    pad = np.zeros((M, N + 1, cz.shape[2]))
    pad[:, :N] = cz
    out = np.empty((M, setup.nz, setup.L))
    for line in range(setup.nz):
        u0, a, n, f, v = _line_tables(setup, line)
        col0 = (1.0 - f) * pad[:, u0, n] + f * pad[:, u0, n + 1]
        col1 = (1.0 - f) * pad[:, u0 + 1, n] + f * pad[:, u0 + 1, n + 1]
        out[:, line] = gains[:, None] * v[None, :] * ((1.0 - a) * col0 + a * col1)
    return out


def resample_adj_z(sig, setup, angles=None):
    """The literal transpose of resample_fwd_z: every sample scattered back onto the
    four grid points it read, with the same weights (bincount sums the scatter)."""
    sig = np.asarray(sig, dtype=np.float64)
    M = sig.shape[0]
    N = setup.nx
    nez = n_fine_z(setup)
    gains = setup.gains if angles is None else setup.gains[angles]
    out = np.zeros((M, (N + 1) * nez))
    for line in range(setup.nz):
        u0, a, n, f, v = _line_tables(setup, line)
        idx = np.concatenate([u0 * nez + n, u0 * nez + n + 1, (u0 + 1) * nez + n, (u0 + 1) * nez + n + 1])
        wts = np.concatenate([(1.0 - a) * (1.0 - f), (1.0 - a) * f, a * (1.0 - f), a * f])
        for m in range(M):
            w = gains[m] * v * sig[m, line]
            out[m] += np.bincount(idx, weights=wts * np.tile(w, 4), minlength=(N + 1) * nez)
    return out.reshape(M, N + 1, nez)[:, :N]


# ----------------------------------------------------------------------------- A_z

def forward_stages_z(x, setup, angles=None):
    """All intermediates of A_z x: dict(proj, fine_z, sig, data)."""
    th = setup.angles if angles is None else setup.angles[angles]
    from . import projection

    proj = projection.project(x, th)
    cz = psf_fwd_z(proj, setup)
    sig = resample_fwd_z(cz, setup, angles)
    return dict(proj=proj, fine_z=cz, sig=sig, data=operator.compress_fwd(sig, setup))


def adjoint_stages_z(y, setup, angles=None):
    """All intermediates of A_z^T y: dict(sig, fine_z, proj, vol)."""
    th = setup.angles if angles is None else setup.angles[angles]
    from . import projection

    sig = operator.compress_adj(y, setup)
    cz = resample_adj_z(sig, setup, angles)
    proj = psf_adj_z(cz, setup)
    return dict(sig=sig, fine_z=cz, proj=proj, vol=projection.backproject(proj, th, setup.nx))


def forward_z(x, setup):
    """b_z = A_z x, complex [M][N_z][n_bins]; one angle at a time."""
    out = np.empty(setup.data_shape, dtype=np.complex128)
    for m in range(setup.n_angles):
        out[m] = forward_stages_z(x, setup, angles=np.array([m]))["data"][0]
    return out


def adjoint_z(y, setup):
    """x = A_z^T y = Re(A_z^H y), real [N_z][N][N]; one angle at a time."""
    y = np.asarray(y, dtype=np.complex128)
    out = np.zeros((setup.nz, setup.nx, setup.nx))
    for m in range(setup.n_angles):
        out += adjoint_stages_z(y[m:m + 1], setup, angles=np.array([m]))["vol"]
    return out
