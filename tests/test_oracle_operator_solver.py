"""Pins for the oracle's full operator A (Eq. (23)), regulariser T and solver (Eqs. (25)-(26))."""

import math

import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

from oracle import Setup, operator, regularizer, solver
from oracle.data import from_interleaved, make_data, to_interleaved


def _tiny(**kw):
    base = dict(nx=6, nz=4, n_angles=3, S=8, P=4, A=1.5, Q=4, fwhm=2.0, k_min=1, k_max=2, half_width=1)
    base.update(kw)
    return Setup(**base)


def _dot(a, b):
    return float(np.sum((np.asarray(a) * np.conj(np.asarray(b))).real))


@pytest.mark.parametrize("kw", [dict(), dict(zigzag=0), dict(n_angles=5, nx=10, nz=3, S=16, P=8, A=2.5, k_max=3)])
def test_adjoint_dot_product_per_stage_and_end_to_end(kw):
    st = _tiny(**kw)
    st.gains = np.linspace(0.9, 1.1, st.n_angles)
    st.d_gamma = np.exp(0.3j * np.arange(st.n_bins))
    rng = np.random.default_rng(0)
    x = rng.standard_normal((st.nz, st.nx, st.nx))
    y = rng.standard_normal(st.data_shape) + 1j * rng.standard_normal(st.data_shape)
    fs = operator.forward_stages(x, st)
    # stage by stage: <H p, c> = <p, H^T c>, <EV c, s> = <c, (EV)^T s>
    c = rng.standard_normal(fs["fine"].shape)
    assert abs(_dot(operator.psf_fwd(fs["proj"], st), c) - _dot(fs["proj"], operator.psf_adj(c, st))) < 1e-12 * np.linalg.norm(c) * np.linalg.norm(fs["fine"])
    s = rng.standard_normal(fs["sig"].shape)
    assert abs(_dot(operator.resample_fwd(fs["fine"], st), s) - _dot(fs["fine"], operator.resample_adj(s, st))) < 1e-12 * np.linalg.norm(s) * np.linalg.norm(fs["sig"]) * 10
    Ax = operator.forward(x, st)
    ATy = operator.adjoint(y, st)
    lhs, rhs = _dot(Ax, y), _dot(x, ATy)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Ax) * np.linalg.norm(y)


def test_operator_is_block_diagonal_over_angles_and_linear_in_gain():
    st = _tiny()
    rng = np.random.default_rng(1)
    x = rng.standard_normal((st.nz, st.nx, st.nx))
    full = operator.forward(x, st)
    one = operator.forward_stages(x, st, angles=np.array([1]))["data"][0]
    np.testing.assert_allclose(full[1], one, atol=1e-13)
    st.gains = np.array([1.0, 2.5, 1.0])
    scaled = operator.forward(x, st)
    np.testing.assert_allclose(scaled[1], 2.5 * full[1], atol=1e-12)
    np.testing.assert_allclose(scaled[0], full[0], atol=1e-13)


def test_interleaved_round_trip():
    b = np.array([[1 + 2j, -3.5 + 0.25j]])
    np.testing.assert_array_equal(from_interleaved(to_interleaved(b)), b)


# ----------------------------------------------------------------------------- T


def _dense_difference_matrix(shape):
    """T built entry by entry: one row per (axis, voxel with an inside neighbour)."""
    nz, ny, nx = shape
    idx = np.arange(nz * ny * nx).reshape(shape)
    rows = []
    for axis, (dz, dy, dx) in enumerate(((1, 0, 0), (0, 1, 0), (0, 0, 1))):
        for z in range(nz):
            for y in range(ny):
                for x in range(nx):
                    if z + dz < nz and y + dy < ny and x + dx < nx:
                        r = np.zeros(idx.size)
                        r[idx[z + dz, y + dy, x + dx]] = 1.0
                        r[idx[z, y, x]] = -1.0
                        rows.append(r)
    return np.array(rows)


def test_ttt_matches_dense_difference_operator():
    shape = (3, 4, 5)
    T = _dense_difference_matrix(shape)
    rng = np.random.default_rng(2)
    x = rng.standard_normal(shape)
    np.testing.assert_allclose(regularizer.ttt(x).reshape(-1), T.T @ T @ x.reshape(-1), atol=1e-12)
    # constants are in the null space (Neumann boundary)
    np.testing.assert_allclose(regularizer.ttt(np.ones(shape)), 0.0, atol=1e-14)


@pytest.mark.parametrize("shape", [(3, 4, 5), (2, 6, 6), (1, 5, 7)])
def test_ttt_norm_closed_form(shape):
    T = _dense_difference_matrix(shape)
    ev = np.linalg.eigvalsh(T.T @ T)
    assert abs(ev.max() - regularizer.ttt_norm(shape)) < 1e-10


# ----------------------------------------------------------------------------- solver


def test_splitmix64_published_outputs():
    """SplitMix64 from state 0: the first two published outputs are
    0xE220A8397B1DCDAF and 0x6E789E6AA1B965F4."""
    u = solver.splitmix64_uniform(0, 2)
    expect = np.array([0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4], dtype=np.uint64)
    np.testing.assert_array_equal(u, (expect >> np.uint64(11)).astype(np.float64) * 2.0**-52 - 1.0)
    v = solver.splitmix64_uniform(1234, 100000)
    assert v.min() >= -1.0 and v.max() < 1.0 and abs(v.mean()) < 0.01


def _dense_a(st):
    n = st.nz * st.nx * st.nx
    cols = []
    for i in range(n):
        e = np.zeros(n)
        e[i] = 1.0
        cols.append(operator.forward(e.reshape(st.nz, st.nx, st.nx), st).reshape(-1))
    Ac = np.stack(cols, axis=1)
    return np.concatenate([Ac.real, Ac.imag], axis=0)  # real-stacked [2*rows, n]


def test_power_iteration_matches_eigvalsh():
    st = _tiny()
    Ar = _dense_a(st)
    top = np.linalg.eigvalsh(Ar.T @ Ar).max()
    shape = (st.nz, st.nx, st.nx)
    est = solver.power_norm(lambda v: operator.adjoint(operator.forward(v, st), st), shape, n_iter=200)
    assert abs(est - top) < 1e-6 * top


def _tiny_problem():
    st = _tiny()
    shape = (st.nz, st.nx, st.nx)
    Ar = _dense_a(st)
    rng = np.random.default_rng(3)
    xt = np.abs(rng.standard_normal(shape)) * (rng.uniform(size=shape) < 0.3)
    b = operator.forward(xt, st) + 0.05 * (rng.standard_normal(st.data_shape) + 1j * rng.standard_normal(st.data_shape))
    ata = np.linalg.eigvalsh(Ar.T @ Ar).max()
    lam = 0.05 * ata / regularizer.ttt_norm(shape)
    tau = solver.step_size(ata, lam, shape)
    return st, shape, Ar, b, lam, tau


def test_unconstrained_solve_reaches_normal_equations():
    """Without the projection, Eq. (26) converges to (A^T A + lam T^T T) x = A^T b."""
    st, shape, Ar, b, lam, tau = _tiny_problem()
    br = np.concatenate([b.real.reshape(-1), b.imag.reshape(-1)])
    T = _dense_difference_matrix(shape)
    x_chol = scipy.linalg.cho_solve(scipy.linalg.cho_factor(Ar.T @ Ar + lam * T.T @ T), Ar.T @ br)
    x, hist = solver.solve(lambda v: operator.forward(v, st), lambda r: operator.adjoint(r, st), b, shape,
                           tau, lam, iters=1500, nonneg=False)
    assert np.linalg.norm(x.reshape(-1) - x_chol) < 1e-6 * np.linalg.norm(x_chol)


def test_projected_solve_reaches_nnls():
    """With the projection, the fixed point is the NNLS solution of [A; sqrt(lam) T]."""
    st, shape, Ar, b, lam, tau = _tiny_problem()
    br = np.concatenate([b.real.reshape(-1), b.imag.reshape(-1)])
    T = _dense_difference_matrix(shape)
    K = np.concatenate([Ar, math.sqrt(lam) * T], axis=0)
    rhs = np.concatenate([br, np.zeros(T.shape[0])])
    x_nnls, _ = scipy.optimize.nnls(K, rhs, maxiter=5000)
    x, hist = solver.solve(lambda v: operator.forward(v, st), lambda r: operator.adjoint(r, st), b, shape,
                           tau, lam, iters=3000, nonneg=True)
    assert np.linalg.norm(x.reshape(-1) - x_nnls) < 1e-5 * np.linalg.norm(x_nnls)
    assert x.min() >= 0.0
    assert hist[-1] <= hist[0]


def test_make_data_noise_level():
    st = _tiny(n_angles=2)
    x = np.zeros((st.nz, st.nx, st.nx))
    x[1, 2, 3] = 1.0
    b0, info0 = make_data(st, x, noise=0.0)
    b1, info1 = make_data(st, x, noise=0.5, seed=4)
    assert info0["sigma"] == 0.0 and info1["sigma"] == pytest.approx(0.5 * info1["peak"])
    r = (b1 - b0).reshape(-1)
    # complex Gaussian with E|n|^2 = sigma^2
    assert 0.5 < np.mean(np.abs(r) ** 2) / info1["sigma"] ** 2 < 1.6
