"""Workload recipes for the five synthetic configurations.

Each recipe is a plain dict of numbers: volume size, FFL angle count, scan
trajectory (samples per drive period S, periods per raster line P, drive
amplitude A in voxels, fine-grid factor Q), PSF width, harmonic band and
solver settings. The scan follows the paper's acquisition description
(Sec. 3.1: FFL rotated about z over 180 deg, sinusoidal drive plus zig-zag
slow raster); sizes follow the paper's 128^3-class meshes and 21-36 angles
(Sec. 4.1, Tables 2-3) re-shaped as listed below.
"""

import copy

CONFIGS = {
    # Plain method, tiny: 32x32x16, 8 angles, 16 lines x 128 periods x 64 samples.
    "tiny": dict(
        name="tiny", nx=32, nz=16, n_angles=8,
        S=64, P=128, A=6.0, phi0=0.0, zigzag=1, Q=8,
        fwhm=2.0, k_min=1, k_max=8, half_width=2,
        noise=0.01, iters=50, seed=0, phantom="tiny",
    ),
    # Plain method, phantom scale: 128x128x64, 24 angles, 25M samples.
    "phantom": dict(
        name="phantom", nx=128, nz=64, n_angles=24,
        S=64, P=256, A=6.0, phi0=0.0, zigzag=1, Q=8,
        fwhm=3.0, k_min=1, k_max=12, half_width=3,
        noise=0.005, iters=100, seed=0, phantom="ellipsoids",
        gain_spread=0.05, drift=0.01,
    ),
    # Precision, in-vivo scale: 256x256x128, 36 angles, ~302M samples.
    "invivo": dict(
        name="invivo", nx=256, nz=128, n_angles=36,
        S=128, P=512, A=6.0, phi0=0.0, zigzag=1, Q=8,
        fwhm=3.0, k_min=1, k_max=16, half_width=4,
        noise=0.005, iters=100, seed=0, phantom="invivo",
    ),
}


def config(name):
    """Return a deep copy of a named recipe."""
    return copy.deepcopy(CONFIGS[name])


def scaled_config(name, nx=None, nz=None, n_angles=None, P=None, S=None):
    """A recipe with some sizes overridden (used for small parity cases)."""
    c = config(name)
    for key, val in (("nx", nx), ("nz", nz), ("n_angles", n_angles), ("P", P), ("S", S)):
        if val is not None:
            c[key] = val
    return c


def serving_mix(seed=0, n_requests=64):
    """Request recipes for the serving workload: a Poisson stream of mixed jobs.

    Sizes {64^3, 128^2x64, 192^2x96, 256^2x128}, 8-36 angles, harmonics
    1..K with K in 8..16 and half-width K/4, S=64 for N<=192 else 128, P=2N.
    Returns a list of dicts (arrival times are filled in by the caller from
    its measured rate).
    """
    import numpy as np

    rng = np.random.default_rng(seed)
    sizes = [(64, 64), (128, 64), (192, 96), (256, 128)]
    out = []
    for r in range(n_requests):
        nx, nz = sizes[int(rng.integers(0, len(sizes)))]
        K = int(rng.integers(8, 17))
        out.append(dict(
            name=f"req{r}", nx=nx, nz=nz, n_angles=int(rng.integers(8, 37)),
            S=64 if nx <= 192 else 128, P=2 * nx, A=6.0, phi0=0.0, zigzag=1, Q=8,
            fwhm=3.0, k_min=1, k_max=K, half_width=max(1, K // 4),
            noise=0.005, iters=100, seed=int(rng.integers(0, 2**31 - 1)),
            phantom="ellipsoids" if nx < 256 else "invivo",
        ))
    return out
