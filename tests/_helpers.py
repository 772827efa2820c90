"""Shared helpers for the tests (no method arithmetic here)."""

import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# Tolerances stated for the hot path: FP32 operator applications must match the
# FP64 oracle within rel-L2 1e-5; reconstructed volumes within rel-L2 1e-3.
OP_TOL = 1e-5
RECON_TOL = 1e-3


def rel_l2(a, b):
    """||a - b|| / ||b|| in FP64, complex inputs compared as complex."""
    cplx = np.iscomplexobj(a) or np.iscomplexobj(b)
    a = np.asarray(a, dtype=np.complex128 if cplx else np.float64)
    b = np.asarray(b, dtype=np.complex128 if cplx else np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def ensure_library():
    """Build libmpiffl.so in-tree if it is missing; return its path."""
    from paper_2511_06627_gb300 import _lib

    if not os.path.exists(_lib.LIB_PATH):
        from paper_2511_06627_gb300 import build

        build.build()
    return _lib.LIB_PATH


def oracle_setup_kwargs(cfg):
    keys = ("nx", "nz", "n_angles", "S", "P", "A", "phi0", "zigzag", "Q", "fwhm", "k_min", "k_max", "half_width")
    return {k: cfg[k] for k in keys if k in cfg}
