"""The full tensor PSF and the receive-coil map in the FFL plane (oracle, float64).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this module; the product path never does.

Sec. 1.2, Eq. (7) and Appendix B, Eq. (31): the signal is
    s0(t) = m sum_ij int rho(x) v_j(t) b_i(x) h_ij(xi(t) - x) dx,
with the 3x3 tensor PSF
    h(x) = [ L'(|Gx|/Hs) (Gx)(Gx)^T / (|Gx| Hs) + L(|Gx|/Hs) (I - (Gx)(Gx)^T/|Gx|^2) ] G / |Gx|.
In the projection plane of an FFL along y (Sec. 2.2, Eq. (19)) the position is
x' = (u, z), u along the scanner's x axis (the detector axis of P_theta) and z
along the slices.

Readings (the paper gives the tensor and the coil field, not their use in the
projection model):
  - G = diag(-G0, 0, G0) (Eq. (2)), so |Gx'| = G0 rho, rho = sqrt(u^2 + z^2): the
    tensor has the eigenvalue L'(xi)/Hs along n = Gx'/|Gx'| and L(xi)/(Hs xi)
    across it, xi = rho / a with a = Hs/G0 in voxels.
  - Drive along x with the receive coil along x (collinear), so the signal takes
    the (x, x) component. Normalised by the constant of the 1D reading (psf.py):
        h_uu(u, z) = 3 [ L'(xi) u^2/rho^2 + (L(xi)/xi) z^2/rho^2 ],  h_uu(0, 0) = 1.
    On z = 0 this is the 1D PSF 3 L'(u/a), and a comes from the FWHM along the
    drive axis exactly as there. The transverse term decays like 1/rho: no
    truncation in either direction.
  - The coil sensitivity (operator B) is the x component b(z, u) of the coil
    field on the projection plane, in scanner coordinates: the object rotates,
    the scanner does not (Eq. (19)), so the same map applies at every angle. B
    multiplies the projection before H, together with the per-angle gain.
  - H then couples the slices: the PSF-convolved projection on line l (slice l)
    at fine point e is
        c[m, l, e] = sum_{z', i} b[z', i] proj[m, z', i] h_uu(u_lo + e/Q - i, l - z'),
    on the fine grid of operator.py (u_lo = -D/Q). E, V, the gains and S D F
    are those of operator.py.
"""

import numpy as np

from . import operator, projection, psf


def langevin_over_x(x):
    """L(x)/x, with the series 1/3 - x^2/45 + 2x^4/945 - x^6/4725 for |x| < 0.05."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    ax = np.abs(x)
    small = ax < 0.05
    x2 = x[small] ** 2
    out[small] = 1.0 / 3.0 - x2 / 45.0 + 2.0 * x2**2 / 945.0 - x2**3 / 4725.0
    xl = ax[~small]
    out[~small] = (1.0 / np.tanh(xl) - 1.0 / xl) / xl
    return out


def tensor_inplane(u, z, fwhm):
    """The normalised in-plane tensor 3 [L'(xi) n n^T + (L(xi)/xi)(I - n n^T)] at offset
    (u, z), n = (u, z)/rho: returns its (uu, uz, zz) components."""
    u = np.asarray(u, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    u, z = np.broadcast_arrays(u, z)
    a = psf.width_scale(fwhm)
    rho2 = u * u + z * z
    xi = np.sqrt(rho2) / a
    col = 3.0 * psf.langevin_deriv(xi)
    tra = 3.0 * langevin_over_x(xi)
    at0 = rho2 == 0.0
    safe = np.where(at0, 1.0, rho2)
    cu, cz, cuz = np.where(at0, 1.0, u * u / safe), np.where(at0, 0.0, z * z / safe), np.where(at0, 0.0, u * z / safe)
    # at the origin both eigenvalues are 1: any direction gives the identity
    return col * cu + tra * cz, (col - tra) * cuz, col * cz + tra * cu


def h_uu(u, z, fwhm):
    """Collinear (x drive, x receive) component of the PSF at in-plane offset (u, z)."""
    return tensor_inplane(u, z, fwhm)[0]


# ----------------------------------------------------------------------------- B and H

def coil_apply(proj, coil):
    """B: proj[m, z, i] * b[z, i] (coil None: a uniform coil, b = 1)."""
    proj = np.asarray(proj, dtype=np.float64)
    if coil is None:
        return proj
    return proj * np.asarray(coil, dtype=np.float64)[None]


def psf_matrix_offset(setup, d, fwhm=None):
    """H_d as a dense [N_e, N] matrix: H_d[e, i] = h_uu(u_lo + e/Q - i, d)."""
    fwhm = setup.fwhm if fwhm is None else fwhm
    e = np.arange(setup.n_fine, dtype=np.float64)
    i = np.arange(setup.nx, dtype=np.float64)
    u = (e[:, None] - setup.D) / setup.Q - i[None, :]
    return h_uu(u, float(d), fwhm)


def psf_fwd_2d(proj, setup):
    """c[m, l, :] = sum_{z'} H_{l - z'} proj[m, z', :], over every slice offset."""
    proj = np.asarray(proj, dtype=np.float64)
    M, nz, _ = proj.shape
    out = np.zeros((M, nz, setup.n_fine))
    for d in range(-(nz - 1), nz):
        Hd = psf_matrix_offset(setup, d)
        lo, hi = max(0, d), min(nz, nz + d)  # lines l with 0 <= l - d < nz
        out[:, lo:hi] += proj[:, lo - d:hi - d] @ Hd.T
    return out


def psf_adj_2d(fine, setup):
    """proj[m, z', :] = sum_l H_{l - z'}^T c[m, l, :]."""
    fine = np.asarray(fine, dtype=np.float64)
    M, nz, _ = fine.shape
    out = np.zeros((M, nz, setup.nx))
    for d in range(-(nz - 1), nz):
        Hd = psf_matrix_offset(setup, d)
        lo, hi = max(0, d), min(nz, nz + d)
        out[:, lo - d:hi - d] += fine[:, lo:hi] @ Hd
    return out


# ----------------------------------------------------------------------------- A, A^T

def forward_stages(x, setup, coil=None, angles=None):
    """All intermediates of A x with the tensor PSF: dict(proj, coil, fine, sig, data)."""
    th = setup.angles if angles is None else setup.angles[angles]
    proj = projection.project(x, th)
    pb = coil_apply(proj, coil)
    fine = psf_fwd_2d(pb, setup)
    sig = operator.resample_fwd(fine, setup, angles)
    return dict(proj=proj, coil=pb, fine=fine, sig=sig, data=operator.compress_fwd(sig, setup))


def adjoint_stages(y, setup, coil=None, angles=None):
    """All intermediates of A^T y with the tensor PSF: dict(sig, fine, coil, proj, vol)."""
    th = setup.angles if angles is None else setup.angles[angles]
    sig = operator.compress_adj(y, setup)
    fine = operator.resample_adj(sig, setup, angles)
    pb = psf_adj_2d(fine, setup)
    proj = coil_apply(pb, coil)
    return dict(sig=sig, fine=fine, coil=pb, proj=proj, vol=projection.backproject(proj, th, setup.nx))


def forward(x, setup, coil=None):
    """b = A x with the tensor PSF and coil map, complex [M][N_z][n_bins]."""
    out = np.empty(setup.data_shape, dtype=np.complex128)
    for m in range(setup.n_angles):
        out[m] = forward_stages(x, setup, coil, angles=np.array([m]))["data"][0]
    return out


def adjoint(y, setup, coil=None):
    """x = A^T y = Re(A^H y) with the tensor PSF and coil map, real [N_z][N][N]."""
    y = np.asarray(y, dtype=np.complex128)
    vol = np.zeros((setup.nz, setup.nx, setup.nx))
    for m in range(setup.n_angles):
        vol += adjoint_stages(y[m:m + 1], setup, coil, angles=np.array([m]))["vol"]
    return vol
