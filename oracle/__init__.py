"""FP64 CPU oracle for the compressed 3D FFL-MPI operator and its solve.

TEST INFRASTRUCTURE ONLY. This package is imported by tests/, by
__graft_entry__.smoke() (to check one small GPU call) and by bench.py's CPU
baseline leg. The product package never imports, links or runs it, and it
shares no code, tables or constants with the CUDA path; both sides draw only
their seeded inputs from the separate `phantoms` package.

It follows the paper (arXiv 2511.06627) step by step, in float64:

  projection   Sec. 2.2, Eqs. (16)-(17), (19): parallel-beam line integrals
               about z, discretised by Joseph interpolation
  psf          Sec. 1.2, Eq. (7) and Appendix B, Eq. (31): Langevin-derivative
               PSF along the drive axis
  trajectory   Sec. 1.2, Eqs. (3)-(4), (7) and Sec. 3.1: FFL position and
               velocity of a sinusoidal drive plus a zig-zag slow raster
  operator     Sec. 1.3 Eq. (9), Sec. 2.1 Eqs. (11), (13), Sec. 2.2 Eq. (23),
               Appendix A Eq. (27): A = blockdiag(S D_Gamma F V E H B) [P_theta]
  zdrive       Sec. 3.1: the z-drive scan of the dual-drive acquisition, A_z
  regularizer  Sec. 3.3, Eq. (25): finite-difference operator T
  solver       Sec. 3.3, Eqs. (25)-(26): accelerated projected gradient descent
  data         noisy compressed data for the synthetic workloads

Where the paper leaves a choice open, the oracle takes one reading; each is
named in the docstring of the function that makes it. Every function here is
pinned by a test in tests/test_oracle_*.py against something other than
itself (closed forms, special cases, brute force, library routines).
"""

from .setup import Setup  # noqa: F401
from . import projection, psf, trajectory, operator, regularizer, solver, data, zdrive  # noqa: F401
