"""Problem description for the oracle (geometry, trajectory, PSF, harmonics).

The derived quantities follow the readings stated below:

* Angles (Sec. 3.1, equally spaced over the full 180 deg): theta_m = m*pi/M,
  m = 0..M-1 (180 deg itself would repeat 0 deg).
* Lines: one raster line per z slice; segment = one line of one angle.
* Samples: L = S*P per line (S samples per drive period, P periods).
* Fine grid: D = ceil(A*Q), u_lo = -D/Q, N_e = (N-1)*Q + 2*D + 1 points at
  detector positions u_lo + e/Q (detector bin i sits at position i).
* Kept bins (Sec. 2.1, Eq. (11)): omega = k*P + delta for k = k_min..k_max,
  delta = -w..w (harmonic k of the drive falls on bin k*P of a line).
"""

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Setup:
    nx: int
    nz: int
    n_angles: int
    S: int
    P: int
    A: float = 6.0
    phi0: float = 0.0
    zigzag: int = 1
    Q: int = 8
    fwhm: float = 2.0
    k_min: int = 1
    k_max: int = 8
    half_width: int = 2
    angles: np.ndarray = None
    gains: np.ndarray = None
    d_gamma: np.ndarray = None  # complex per kept bin, None = identity
    bins: np.ndarray = field(default=None)  # explicit kept-bin list (overrides harmonics)

    def __post_init__(self):
        if self.angles is None:
            self.angles = np.arange(self.n_angles, dtype=np.float64) * math.pi / self.n_angles
        self.angles = np.asarray(self.angles, dtype=np.float64)
        if self.gains is None:
            self.gains = np.ones(self.n_angles)
        self.gains = np.asarray(self.gains, dtype=np.float64)
        L = self.S * self.P
        if self.bins is None:
            if self.k_min * self.P - self.half_width < 1 or self.k_max * self.P + self.half_width >= L // 2:
                raise ValueError("harmonic band leaves 1 <= omega < L/2")
            k = np.arange(self.k_min, self.k_max + 1)
            d = np.arange(-self.half_width, self.half_width + 1)
            self.bins = (k[:, None] * self.P + d[None, :]).reshape(-1)
        self.bins = np.asarray(self.bins, dtype=np.int64)
        if self.d_gamma is None:
            self.d_gamma = np.ones(len(self.bins), dtype=np.complex128)
        self.d_gamma = np.asarray(self.d_gamma, dtype=np.complex128)

    @classmethod
    def from_config(cls, cfg, **over):
        keys = ("nx", "nz", "n_angles", "S", "P", "A", "phi0", "zigzag", "Q", "fwhm",
                "k_min", "k_max", "half_width")
        kw = {k: cfg[k] for k in keys if k in cfg}
        kw.update(over)
        return cls(**kw)

    @property
    def L(self):
        return self.S * self.P

    @property
    def D(self):
        return int(math.ceil(self.A * self.Q - 1e-9))

    @property
    def n_fine(self):
        return (self.nx - 1) * self.Q + 2 * self.D + 1

    @property
    def n_bins(self):
        return len(self.bins)

    @property
    def data_shape(self):
        """Complex data layout [M][N_z][n_bins] (bins ordered k-major, delta ascending)."""
        return (self.n_angles, self.nz, self.n_bins)
