"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This package holds workload recipes (sizes, scan parameters) and phantom
volumes only. It contains none of the reconstruction method's arithmetic
(no projection, PSF, resampling, DFT or solver step), so that the oracle and
the CUDA path can both draw their inputs from it without sharing method code.
"""

from .configs import CONFIGS, config, scaled_config  # noqa: F401
from .generators import (  # noqa: F401
    phantom_for,
    phantom_tiny,
    phantom_ellipsoids,
    phantom_invivo,
    random_volume,
    random_data,
)
