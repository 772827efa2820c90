"""Pins for the oracle's parallel-beam projector (Sec. 2.2, Eqs. (16)-(19))."""

import math

import numpy as np
import pytest

from oracle import projection
from phantoms.generators import add_gaussian, phantom_tiny


def test_theta_zero_is_sum_over_y():
    rng = np.random.default_rng(1)
    vol = rng.standard_normal((3, 12, 12))
    p = projection.project(vol, np.array([0.0]))[0]
    np.testing.assert_allclose(p, vol.sum(axis=1), rtol=0, atol=1e-12)


def test_theta_ninety_is_sum_over_x_reversed():
    # u = X cos - Y sin = -Y at 90 deg: detector bin i sees row y = N-1-i
    rng = np.random.default_rng(2)
    vol = rng.standard_normal((3, 12, 12))
    p = projection.project(vol, np.array([math.pi / 2]))[0]
    np.testing.assert_allclose(p, vol.sum(axis=2)[:, ::-1], rtol=0, atol=1e-12)


def test_theta_180_mirrors_theta_zero():
    rng = np.random.default_rng(3)
    vol = rng.standard_normal((2, 10, 10))
    p0 = projection.project(vol, np.array([0.0]))[0]
    p180 = projection.project(vol, np.array([math.pi]))[0]
    np.testing.assert_allclose(p180, p0[:, ::-1], atol=1e-12)


def _disc(n, r, sub=4):
    """Uniform disc of radius r about the slice centre, sub x sub supersampled."""
    c = (n - 1) / 2.0
    offs = (np.arange(sub) + 0.5) / sub - 0.5
    yy, xx = np.meshgrid(np.arange(n) - c, np.arange(n) - c, indexing="ij")
    acc = np.zeros((n, n))
    for oy in offs:
        for ox in offs:
            acc += ((yy + oy) ** 2 + (xx + ox) ** 2) <= r * r
    return (acc / sub**2)[None]


@pytest.mark.parametrize("n,r", [(32, 5.0), (64, 20.0)])
def test_uniform_ball_chords(n, r):
    """A uniform disc projects to chord lengths 2 sqrt(r^2 - d^2) at every angle."""
    vol = _disc(n, r)
    c = (n - 1) / 2.0
    thetas = np.arange(7) * math.pi / 7 + 0.1
    p = projection.project(vol, thetas)[:, 0, :]
    u = np.arange(n) - c
    inner = np.abs(u) <= r - 2.0  # the outermost chords cross only partly filled edge voxels
    exact = 2.0 * np.sqrt(np.maximum(r * r - u * u, 0.0))
    err = np.abs(p[:, inner] - exact[None, inner]) / exact[None, inner]
    assert err.max() < 0.03


def test_mass_is_preserved_for_smooth_objects():
    """Each ray sum is a Riemann sum (spacing 1/|cos| or 1/|sin|) of the
    interpolated slice, so sum_u p(u) equals the slice mass for objects that
    are smooth on the voxel scale."""
    n, nz = 48, 3
    vol = np.zeros((nz, n, n))
    rng = np.random.default_rng(4)
    for _ in range(6):
        cen = (rng.uniform(0, nz - 1), *(rng.uniform(-10, 10, size=2) + (n - 1) / 2))
        add_gaussian(vol, cen, rng.uniform(2.0, 3.0), rng.uniform(0.1, 1.0))
    thetas = np.arange(9) * math.pi / 9 + 0.05
    p = projection.project(vol, thetas)
    mass = p.sum(axis=2)  # [m][z]
    ref = vol.sum(axis=(1, 2))[None, :]
    assert (np.abs(mass - ref) / ref).max() < 5e-3


def test_backprojection_is_matrix_transpose():
    thetas = np.array([0.0, 0.3, math.pi / 4, 1.2, math.pi / 2, 2.5])
    n = 7
    P = projection.matrix(thetas, n)  # built column by column from project()
    rng = np.random.default_rng(5)
    proj = rng.standard_normal((len(thetas), 1, n))
    bp = projection.backproject(proj, thetas, n)
    np.testing.assert_allclose(bp.reshape(-1), P.T @ proj.reshape(-1), atol=1e-12)


def test_projection_adjoint_dot():
    thetas = np.arange(5) * math.pi / 5
    rng = np.random.default_rng(6)
    x = rng.standard_normal((3, 16, 16))
    y = rng.standard_normal((5, 3, 16))
    lhs = np.sum(projection.project(x, thetas) * y)
    rhs = np.sum(x * projection.backproject(y, thetas, 16))
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(y) * 16


def test_ray_sums_of_linear_field_match_closed_form():
    """For f = a + bx*x + by*y, row interpolation is exact and the integrand is
    linear along the ray, so the row sum equals the exact line integral:
    n * f(ray midpoint) / |cos| (midpoint rule is exact for linear functions)."""
    n = 16
    c = (n - 1) / 2.0
    a, bx, by = 0.7, -0.3, 0.45
    yy, xx = np.meshgrid(np.arange(n, dtype=float), np.arange(n, dtype=float), indexing="ij")
    vol = (a + bx * xx + by * yy)[None]
    for th in (0.1, 0.35, -0.5, math.pi - 0.3):
        p = projection.project(vol, np.array([th]))[0, 0]
        for i in range(n):
            u = i - c
            if abs(u / math.cos(th)) + c * abs(math.tan(th)) > c:
                continue  # ray leaves the grid inside the volume's rows
            exact = n * (a + bx * (u / math.cos(th) + c) + by * c) / abs(math.cos(th))
            assert abs(p[i] - exact) < 1e-11 * n


def test_tie_goes_to_rows():
    assert projection.row_major(math.pi / 4)
    assert projection.row_major(3 * math.pi / 4)
    assert not projection.row_major(math.pi / 4 + 1e-3)
    vol = phantom_tiny(16, 4, seed=0).astype(np.float64)
    p = projection.project(vol, np.array([math.pi / 4]))
    assert np.isfinite(p).all()
