"""Seeded phantom volumes (x[z][y][x], voxel centres at integer indices).

The shapes stand in for the paper's phantom and in-vivo scans (Sec. 4.2-4.3):
point-like sources, uniform balls, random ellipsoids spanning a 1000:1
dynamic range, and a mouse-like layout (bright liver, tumour, faint foci,
weak background). Every support stays inside the inscribed cylinder
r < N/2 - 2 about the z axis, so no angle's projection leaves the detector.
All randomness comes from numpy.random.default_rng(seed).
"""

import numpy as np


def _grid(nz, n):
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    y = np.arange(n, dtype=np.float64)[None, :, None]
    x = np.arange(n, dtype=np.float64)[None, None, :]
    return z, y, x


def _rotation(rng):
    """Uniformly random 3x3 rotation (QR of a Gaussian matrix)."""
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def add_gaussian(vol, center, sigma, amplitude):
    """Add amplitude * exp(-|r-c|^2 / (2 sigma^2)), evaluated in a 5-sigma box."""
    nz, n, _ = vol.shape
    rad = int(np.ceil(5 * sigma)) + 1
    lo = [max(0, int(np.floor(c)) - rad) for c in center]
    hi = [min(s, int(np.floor(c)) + rad + 1) for c, s in zip(center, (nz, n, n))]
    z = np.arange(lo[0], hi[0])[:, None, None]
    y = np.arange(lo[1], hi[1])[None, :, None]
    x = np.arange(lo[2], hi[2])[None, None, :]
    d2 = (z - center[0]) ** 2 + (y - center[1]) ** 2 + (x - center[2]) ** 2
    vol[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] += amplitude * np.exp(-d2 / (2 * sigma**2))


def add_ellipsoid(vol, center, semi_axes, rot, amplitude, supersample=1):
    """Add a uniform ellipsoid (voxel-averaged over supersample^3 sub-points)."""
    nz, n, _ = vol.shape
    rmax = max(semi_axes) + 1
    lo = [max(0, int(np.floor(c - rmax))) for c in center]
    hi = [min(s, int(np.ceil(c + rmax)) + 1) for c, s in zip(center, (nz, n, n))]
    acc = np.zeros((hi[0] - lo[0], hi[1] - lo[1], hi[2] - lo[2]))
    offs = (np.arange(supersample) + 0.5) / supersample - 0.5
    inv = rot.T / np.asarray(semi_axes)[:, None]  # maps (dz,dy,dx) -> unit-sphere coords
    z0 = np.arange(lo[0], hi[0])[:, None, None] - center[0]
    y0 = np.arange(lo[1], hi[1])[None, :, None] - center[1]
    x0 = np.arange(lo[2], hi[2])[None, None, :] - center[2]
    for oz in offs:
        for oy in offs:
            for ox in offs:
                dz, dy, dx = z0 + oz, y0 + oy, x0 + ox
                q = 0.0
                for a in range(3):
                    t = inv[a, 0] * dz + inv[a, 1] * dy + inv[a, 2] * dx
                    q = q + t * t
                acc += q <= 1.0
    vol[lo[0]:hi[0], lo[1]:hi[1], lo[2]:hi[2]] += amplitude * acc / supersample**3


def _center_in_cylinder(rng, n, nz, margin_xy, margin_z):
    """A random centre whose margin-ball stays inside r < n/2 - 2 and inside z."""
    c = (n - 1) / 2.0
    rmax = n / 2.0 - 2.0 - margin_xy
    if rmax <= 0:
        raise ValueError("object too large for the volume")
    while True:
        px, py = rng.uniform(-rmax, rmax, size=2)
        if px * px + py * py <= rmax * rmax:
            break
    margin_z = min(margin_z, (nz - 1) / 2.0)
    pz = rng.uniform(margin_z, nz - 1 - margin_z)
    return (pz, c + py, c + px)


def phantom_tiny(nx=32, nz=16, seed=0):
    """3 Gaussian sources (sigma 0.5 vox) plus a uniform ball r=5 (4^3 supersampled).

    Amplitudes log-uniform over 1e-2..1.
    """
    rng = np.random.default_rng(seed)
    vol = np.zeros((nz, nx, nx))
    for _ in range(3):
        cen = _center_in_cylinder(rng, nx, nz, 2.5, 2.5)
        add_gaussian(vol, cen, 0.5, 10 ** rng.uniform(-2, 0))
    r = min(5.0, nx / 2.0 - 4.0, (nz - 3) / 2.0)
    cen = _center_in_cylinder(rng, nx, nz, r + 1.0, min(r + 1.0, (nz - 1) / 2.0))
    add_ellipsoid(vol, cen, (r, r, r), np.eye(3), 10 ** rng.uniform(-2, 0), supersample=4)
    return vol.astype(np.float32)


def phantom_ellipsoids(nx=128, nz=64, seed=0, n_ellipsoids=20, n_points=4):
    """Random additive ellipsoids (semi-axes U(3,20), random rotation,
    concentrations log-U(1e-3..1)) plus point sources."""
    rng = np.random.default_rng(seed)
    vol = np.zeros((nz, nx, nx))
    amax = min(20.0, nx / 2.0 - 4.0, (nz - 3) / 2.0)
    amin = min(3.0, amax)
    for _ in range(n_ellipsoids):
        axes = rng.uniform(amin, amax, size=3)
        rot = _rotation(rng)
        m = float(axes.max())
        cen = _center_in_cylinder(rng, nx, nz, m + 1.0, min(m + 1.0, (nz - 1) / 2.0))
        add_ellipsoid(vol, cen, axes, rot, 10 ** rng.uniform(-3, 0), supersample=2 if nx <= 64 else 1)
    for _ in range(n_points):
        cen = _center_in_cylinder(rng, nx, nz, 2.5, 2.5)
        add_gaussian(vol, cen, 0.5, 10 ** rng.uniform(-3, 0))
    return vol.astype(np.float32)


def phantom_invivo(nx=256, nz=128, seed=0, n_foci=200):
    """Mouse-like layout: body ellipsoid with a 1e-4 background, a bright
    'liver' ellipsoid (about 60x45x30 vox at 256^2x128) at 1.0, a 'tumour'
    sphere (r about 12) at 0.3 and faint Gaussian foci log-U(1e-3..1e-2)."""
    rng = np.random.default_rng(seed)
    s = nx / 256.0
    sz = nz / 128.0
    vol = np.zeros((nz, nx, nx))
    c = (nx - 1) / 2.0
    cz = (nz - 1) / 2.0
    body = (0.42 * nz, 0.30 * nx, 0.42 * nx)  # (z, y, x) semi-axes
    body = (min(body[0], cz - 1), min(body[1], nx / 2.0 - 3), min(body[2], nx / 2.0 - 3))
    add_ellipsoid(vol, (cz, c, c), body, np.eye(3), 1e-4)
    liver = (15.0 * sz, 22.5 * s, 30.0 * s)
    add_ellipsoid(vol, (cz + 0.15 * nz, c - 0.05 * nx, c - 0.08 * nx), liver, np.eye(3), 1.0)
    r_t = 12.0 * s
    add_ellipsoid(vol, (cz - 0.2 * nz, c + 0.1 * nx, c + 0.2 * nx), (r_t, r_t, r_t), np.eye(3), 0.3)
    for _ in range(n_foci):
        # foci inside the body ellipsoid
        while True:
            p = rng.uniform(-1, 1, size=3)
            if (p * p).sum() <= 0.8:
                break
        cen = (cz + p[0] * body[0], c + p[1] * body[1], c + p[2] * body[2])
        add_gaussian(vol, cen, 0.7, 10 ** rng.uniform(-3, -2))
    return vol.astype(np.float32)


def phantom_for(cfg, seed=None):
    """The phantom a recipe names, at the recipe's size."""
    seed = cfg.get("seed", 0) if seed is None else seed
    kind = cfg.get("phantom", "ellipsoids")
    if kind == "tiny":
        return phantom_tiny(cfg["nx"], cfg["nz"], seed)
    if kind == "invivo":
        return phantom_invivo(cfg["nx"], cfg["nz"], seed)
    return phantom_ellipsoids(cfg["nx"], cfg["nz"], seed)


def random_volume(nz, n, seed, dtype=np.float64):
    """Standard-normal volume x[z][y][x] (for adjoint and parity tests)."""
    return np.random.default_rng(seed).standard_normal((nz, n, n)).astype(dtype)


def random_data(shape, seed, dtype=np.float64):
    """Standard-normal real array of the given shape (e.g. interleaved complex data)."""
    return np.random.default_rng(seed).standard_normal(shape).astype(dtype)


def sensitivity_series(nx, nz, amounts, seed=0, sigma=1.2):
    """A stand-in for the paper's sensitivity phantom (Sec. 4.2, Figs. 4-5): point-like
    samples of known iron amounts on one slice, plus void regions for the background.

    Each sample is a Gaussian blob whose integral equals its amount. Samples sit on the
    middle slice, evenly spaced on a circle about the rotation axis (radius 0.45 N/2),
    so that the rotating acquisition treats them alike.
    Returns (volume float32 [nz][nx][nx], sample_boxes, void_boxes). Boxes are
    (z0, z1, y0, y1, x0, x1), half-open. Each sample box is a cube of half-width
    3 sigma + 1 around its sample. The five void boxes lie on slices a quarter of the
    height away from the samples.
    """
    rng = np.random.default_rng(seed)
    vol = np.zeros((nz, nx, nx), dtype=np.float64)
    zc = nz // 2
    yc = (nx - 1) / 2.0
    k = len(amounts)
    rad = 0.45 * (nx / 2.0)
    h = max(1, int(np.ceil(3 * sigma)) + 1)
    sample_boxes = []
    for s_, amt in enumerate(amounts):
        phi = 2 * np.pi * s_ / k + 0.3
        c = (zc + rng.uniform(-0.3, 0.3), yc + rad * np.sin(phi) + rng.uniform(-0.3, 0.3),
             (nx - 1) / 2.0 + rad * np.cos(phi))
        add_gaussian(vol, c, sigma, float(amt) / (2.0 * np.pi * sigma * sigma) ** 1.5)
        iz, iy, ix = (int(round(v)) for v in c)
        sample_boxes.append((iz - h, iz + h + 1, iy - h, iy + h + 1, ix - h, ix + h + 1))
    w = max(2, nx // 16)
    void_boxes = []
    for j, zq in enumerate((nz // 4, nz // 4, 3 * nz // 4, 3 * nz // 4, nz // 4)):
        ang = 2 * np.pi * j / 5
        cy = int(round(yc + 0.3 * nx * np.sin(ang)))
        cx = int(round((nx - 1) / 2.0 + 0.3 * nx * np.cos(ang)))
        dz = max(1, nz // 16)
        void_boxes.append((zq - dz, zq + dz, cy - w, cy + w, cx - w, cx + w))
    return vol.astype(np.float32), sample_boxes, void_boxes
