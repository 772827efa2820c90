"""The compressed 3D FFL-MPI operator A and its adjoint (oracle, float64).

Sec. 2.2, Eq. (23) and Sec. 3.3, Eq. (24):
    A = blockdiag_m(A_DC) [P_theta_1; ...; P_theta_M],
Sec. 2.1, Eq. (13):  A_DC = S D_Gamma F V E H B.

Stages, applied per angle m and raster line l (= z slice):
  P   proj[m,l,i]  = (P_theta_m x)[l, i]                     projection.py
  H   c[m,l,e]     = sum_i proj[m,l,i] h(u_lo + e/Q - i)      (full support)
  E,V,B  s[m,l,j]  = g_m v_j ((1-f_j) c[m,l,n_j] + f_j c[m,l,n_j+1])
  S D F  b[m,l,q]  = D_q L^{-1/2} sum_j s[m,l,j] exp(+2 pi i omega_q j / L)

The paper factors the PSF (H) and the FFL selection (E) but gives no rule
for evaluating the convolved image between detector bins; the reading used
here evaluates it on a grid Q times finer than the bins and interpolates
linearly at the FFL position (t = Q xi + D, cell n, fraction f). F uses the
unitary +i convention of Appendix A, Eq. (27). B is one scalar gain per angle
(a spatially uniform receive coil).

The adjoint is taken under the real inner product <b, y> = sum Re(b conj y)
(the update of Eq. (26) keeps only real values): A^T y = Re(A^H y).
"""

import numpy as np
import scipy.fft

from . import projection, psf, trajectory


def _workers():
    import os

    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


# ----------------------------------------------------------------------------- H

def psf_matrix(setup, fwhm=None):
    """H as a dense [N_e, N] matrix: H[e, i] = h(u_lo + e/Q - i)."""
    fwhm = setup.fwhm if fwhm is None else fwhm
    e = np.arange(setup.n_fine, dtype=np.float64)
    i = np.arange(setup.nx, dtype=np.float64)
    u = (e[:, None] - setup.D) / setup.Q - i[None, :]
    return psf.h(u, fwhm)


def psf_fwd(proj, setup, fwhm=None):
    return np.asarray(proj, dtype=np.float64) @ psf_matrix(setup, fwhm).T


def psf_adj(fine, setup, fwhm=None):
    return np.asarray(fine, dtype=np.float64) @ psf_matrix(setup, fwhm)


# ----------------------------------------------------------------------------- E V B

def _line_tables(setup, line):
    xi, v = trajectory.line_positions(setup, line)
    n, f = trajectory.fine_index(setup, xi)
    return n, f, v


def resample_fwd(fine, setup, angles=None):
    """s[m,l,j] = g_m v_j lerp(fine[m,l,:], t_j); `angles` selects gains for a subset."""
    fine = np.asarray(fine, dtype=np.float64)
    M, nz, _ = fine.shape
    gains = setup.gains if angles is None else setup.gains[angles]
    out = np.empty((M, nz, setup.L))
    for line in range(nz):
        n, f, v = _line_tables(setup, line)
        row = fine[:, line, :]
        out[:, line, :] = gains[:, None] * v[None, :] * ((1.0 - f) * row[:, n] + f * row[:, n + 1])
    return out


def resample_adj(sig, setup, angles=None):
    sig = np.asarray(sig, dtype=np.float64)
    M, nz, _ = sig.shape
    gains = setup.gains if angles is None else setup.gains[angles]
    out = np.zeros((M, nz, setup.n_fine))
    for line in range(nz):
        n, f, v = _line_tables(setup, line)
        for m in range(M):
            w = gains[m] * v * sig[m, line]
            out[m, line] += np.bincount(n, weights=(1.0 - f) * w, minlength=setup.n_fine)
            out[m, line] += np.bincount(n + 1, weights=f * w, minlength=setup.n_fine)
    return out


# ----------------------------------------------------------------------------- S D F

def compress_fwd(sig, setup):
    """b_q = D_q L^{-1/2} sum_j s_j exp(+2 pi i omega_q j / L) for the kept bins."""
    sig = np.asarray(sig, dtype=np.float64)
    L = setup.L
    spec = scipy.fft.ifft(sig, axis=-1, workers=_workers()) * np.sqrt(L)
    return spec[..., setup.bins] * setup.d_gamma


def compress_adj(data, setup):
    """s_j = L^{-1/2} Re sum_q conj(D_q) y_q exp(-2 pi i omega_q j / L)."""
    data = np.asarray(data, dtype=np.complex128)
    L = setup.L
    full = np.zeros(data.shape[:-1] + (L,), dtype=np.complex128)
    full[..., setup.bins] = np.conj(setup.d_gamma) * data
    return np.real(scipy.fft.fft(full, axis=-1, workers=_workers())) / np.sqrt(L)


# ----------------------------------------------------------------------------- A, A^T

def forward_stages(x, setup, angles=None):
    """All intermediates of A x: dict(proj, fine, sig, data)."""
    th = setup.angles if angles is None else setup.angles[angles]
    proj = projection.project(x, th)
    fine = psf_fwd(proj, setup)
    sig = resample_fwd(fine, setup, angles)
    data = compress_fwd(sig, setup)
    return dict(proj=proj, fine=fine, sig=sig, data=data)


def adjoint_stages(y, setup, angles=None):
    """All intermediates of A^T y: dict(sig, fine, proj, vol)."""
    th = setup.angles if angles is None else setup.angles[angles]
    sig = compress_adj(y, setup)
    fine = resample_adj(sig, setup, angles)
    proj = psf_adj(fine, setup)
    vol = projection.backproject(proj, th, setup.nx)
    return dict(sig=sig, fine=fine, proj=proj, vol=vol)


def forward(x, setup):
    """b = A x, complex [M][N_z][n_bins]; evaluated one angle at a time."""
    out = np.empty(setup.data_shape, dtype=np.complex128)
    for m in range(setup.n_angles):
        out[m] = forward_stages(x, setup, angles=np.array([m]))["data"][0]
    return out


def adjoint(y, setup):
    """x = A^T y = Re(A^H y), real [N_z][N][N]; evaluated one angle at a time."""
    y = np.asarray(y, dtype=np.complex128)
    vol = np.zeros((setup.nz, setup.nx, setup.nx))
    for m in range(setup.n_angles):
        vol += adjoint_stages(y[m:m + 1], setup, angles=np.array([m]))["vol"]
    return vol


def max_abs_signal(x, setup):
    """max_j |s_j| of the noiseless time signal of A x (sets the noise level)."""
    mx = 0.0
    for m in range(setup.n_angles):
        sig = forward_stages(x, setup, angles=np.array([m]))["sig"]
        mx = max(mx, float(np.abs(sig).max()))
    return mx


def information_retained(sig, bins):
    """I(s, S) = sqrt(sum_{w in S} |s_hat_w|^2) / ||s|| (Appendix A, Eq. (30))."""
    sig = np.asarray(sig, dtype=np.float64)
    L = sig.shape[-1]
    spec = scipy.fft.ifft(sig, axis=-1) * np.sqrt(L)
    return np.sqrt((np.abs(spec[..., bins]) ** 2).sum()) / np.linalg.norm(sig)
