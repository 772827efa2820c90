"""Writes recon_phantom.npz: the FP64 oracle's reconstruction of the phantom-scale
workload, the expected value of the phantom-scale reconstruction parity tests.

Workload: 128 x 128 x 64 volume of 20 seeded ellipsoids and 4 point sources, 24 FFL
angles, 64 lines x 256 drive periods x 64 samples per angle, PSF FWHM 3 voxels,
harmonics 1..12 kept at +-3 bins. Data b = A x with per-angle gains U(0.95, 1.05) and
a linear baseline drift (both unmodelled by the solve), plus complex Gaussian noise at
0.5 % of the peak signal, all seeded (seed 0). The solve is Eq. (26) of Sec. 3.3, 100
iterations from zero with the non-negativity projection, tau from 50 power
iterations on A^T A (SplitMix64 start vector, seed 1234) and the default lambda. The
data are stored too (float32, as the GPU path takes them, and as the oracle's solve
took them), so that the expected volume does not depend on how another machine's
libm rounds the phantom's ellipsoid boundaries.

Only the oracle and the phantom generators run here. Command (from the repository
root; about 10 minutes on 8 cores):

    python tests/golden/make_recon_phantom.py
"""

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import Setup, operator, solver  # noqa: E402
from oracle.data import make_data  # noqa: E402
from phantoms import config, phantom_for  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "recon_phantom.npz")
POWER_ITERS = 50
POWER_SEED = 1234


def main():
    t0 = time.time()
    cfg = config("phantom")
    st = Setup.from_config(cfg)
    x_true = phantom_for(cfg)
    b, info = make_data(st, x_true, noise=cfg["noise"], seed=cfg["seed"], gain_spread=cfg["gain_spread"],
                        drift=cfg["drift"])
    shape = (st.nz, st.nx, st.nx)
    ata = solver.power_norm(lambda v: operator.adjoint(operator.forward(v, st), st), shape, n_iter=POWER_ITERS,
                            seed=POWER_SEED)
    lam = solver.default_lambda(ata, shape)
    tau = solver.step_size(ata, lam, shape)
    # the solve takes the data as the GPU path receives them: complex, rounded to float32
    b = b.real.astype(np.float32).astype(np.float64) + 1j * b.imag.astype(np.float32).astype(np.float64)
    x, hist = solver.solve(lambda v: operator.forward(v, st), lambda r: operator.adjoint(r, st), b, shape, tau, lam,
                           cfg["iters"])
    np.savez_compressed(OUT, x=x.astype(np.float32), b=np.stack([b.real, b.imag], -1).astype(np.float32),
                        ata=ata, lam=lam, tau=tau, hist=np.asarray(hist),
                        iters=cfg["iters"], seed=cfg["seed"], power_iters=POWER_ITERS, power_seed=POWER_SEED,
                        gains=info["gains"], b_norm=float(np.linalg.norm(b)), x_norm=float(np.linalg.norm(x)))
    print(f"wrote {OUT}: ||A^T A|| = {ata:.6e}, lambda = {lam:.6e}, tau = {tau:.6e}, "
          f"residual {hist[0]:.4e} -> {hist[-1]:.4e}, {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
