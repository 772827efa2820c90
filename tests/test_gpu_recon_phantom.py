"""Reconstruction parity at the phantom scale (Sec. 3.3, Eq. (26)).

The phantom-scale workload: 128 x 128 x 64 volume of seeded ellipsoids and point
sources, 24 FFL angles, 64 lines x 256 drive periods x 64 samples per angle, PSF FWHM
3 voxels, harmonics 1..12 at +-3 bins, data with unmodelled per-angle gains, baseline
drift and 0.5 % noise. 100 iterations of Eq. (26) on every evaluation path, and as a
batched job beside another job, must match the FP64 oracle's reconstruction within
rel-L2 1e-3. The oracle's volume is stored in tests/golden/recon_phantom.npz (written
by tests/golden/make_recon_phantom.py from the oracle alone, about 10 minutes on
8 cores), together with the data it was solved from.
"""

import ctypes as C
import os

import numpy as np
import pytest

from _helpers import RECON_TOL, ensure_library, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from phantoms import config, phantom_for  # noqa: E402

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "recon_phantom.npz")


@pytest.fixture(scope="module")
def phantom():
    ensure_library()
    g = np.load(GOLDEN)
    cfg = config("phantom")
    assert int(g["iters"]) == cfg["iters"] and int(g["seed"]) == cfg["seed"]
    b = np.ascontiguousarray(g["b"], dtype=np.float32)
    assert b.shape == (cfg["n_angles"], cfg["nz"], (cfg["k_max"] - cfg["k_min"] + 1) * (2 * cfg["half_width"] + 1), 2)
    return dict(cfg=cfg, b=torch.from_numpy(b).cuda(), x=g["x"].astype(np.float64), ata=float(g["ata"]),
                lam=float(g["lam"]), tau=float(g["tau"]), hist=g["hist"], power_iters=int(g["power_iters"]),
                power_seed=int(g["power_seed"]))


def _op(cfg, key):
    from paper_2511_06627_gb300 import PREC_BF16X3, PREC_TF32, FFLOperator

    op = FFLOperator.from_config(cfg)
    tf32 = key.endswith("_tf32")
    path = key[: -len("_tf32")] if tf32 else key
    op.set_path(path)
    if path in ("line_gemm", "full_gemm"):
        op.set_precision(PREC_TF32 if tf32 else PREC_BF16X3)
    return op


def test_power_norm_matches_the_oracle(phantom):
    op = _op(phantom["cfg"], "full_gemm")
    got = op.power_norm(phantom["power_iters"], phantom["power_seed"])
    assert abs(got - phantom["ata"]) <= 1e-4 * phantom["ata"]
    op.close()


@pytest.mark.parametrize("key", ["staged", "fused", "line_gemm", "line_gemm_tf32", "full_gemm", "full_gemm_tf32"])
def test_reconstruction_matches_the_oracle(phantom, key):
    op = _op(phantom["cfg"], key)
    iters = phantom["cfg"]["iters"]
    x, rep = op.solve(phantom["b"], iters=iters, lam=phantom["lam"], tau=phantom["tau"])
    xg = x.cpu().numpy()
    err = rel_l2(xg, phantom["x"])
    assert err < RECON_TOL, (key, err)
    assert xg.min() >= 0.0
    assert rep["iters_done"] == iters
    hist = phantom["hist"]
    assert abs(rep["residual_first"] - hist[0]) <= 1e-5 * hist[0]
    assert abs(rep["residual_last"] - hist[-1]) <= RECON_TOL * hist[-1]
    op.close()


def test_batched_job_matches_the_oracle(phantom):
    """The phantom reconstruction advanced as a job of a continuous batch, beside a
    smaller job of another geometry, on the full-GEMM path."""
    from paper_2511_06627_gb300 import _lib as L
    from paper_2511_06627_gb300.serving import _declare

    lib = L.load()
    _declare(lib)
    cfg = phantom["cfg"]
    iters = cfg["iters"]
    op = _op(cfg, "full_gemm")
    tiny = config("tiny")
    other = _op(tiny, "full_gemm")
    b2 = other.forward(torch.from_numpy(phantom_for(tiny)).cuda())
    s = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    hs = []
    for o, bd in ((op, phantom["b"]), (other, b2)):
        p = L.SolveParams(iters, phantom["lam"], phantom["tau"], 20, C.c_uint64(1234), 1, 0.0, 0.0)
        h = C.c_void_p()
        assert lib.mpi_ffl_job_create(o._h, C.c_void_p(bd.data_ptr()), None, C.byref(p), C.byref(h), s) == 0
        hs.append(h)
    arr = (C.c_void_p * 2)(*[h.value for h in hs])
    for _ in range(iters):
        assert lib.mpi_ffl_job_step(arr, 2, s) == 0
    x = op.new_volume()
    assert lib.mpi_ffl_job_result(hs[0], C.c_void_p(x.data_ptr()), s) == 0
    torch.cuda.synchronize()
    err = rel_l2(x.cpu().numpy(), phantom["x"])
    assert err < RECON_TOL, err
    for h in hs:
        lib.mpi_ffl_job_destroy(h)
    op.close()
    other.close()
