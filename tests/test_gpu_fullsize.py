"""Parity at the benchmark's full size (256^2 x 128 volume, 36 angles, 128 x 512 x 128
time samples per angle), in the configuration the benchmark times: every evaluation
path against the FP64 oracle on sampled angles (the oracle computes one angle of A
and of A^T at a time), and the adjoint identity over all angles."""

import numpy as np
import pytest

from _helpers import OP_TOL, ensure_library, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Setup, operator  # noqa: E402
from phantoms import config, phantom_for  # noqa: E402

# theta = 0 (rows), 45 deg (the tie, rows), 100 deg (columns), 155 deg (rows)
ANGLES = [0, 9, 20, 31]
PATHS = ["full_gemm", "line_gemm", "fused", "staged"]


@pytest.fixture(scope="module")
def big():
    ensure_library()
    from paper_2511_06627_gb300 import FFLOperator

    cfg = config("invivo")
    st = Setup.from_config(cfg)
    x = phantom_for(cfg)
    op = FFLOperator.from_config(cfg)
    xo = x.astype(np.float64)
    rng = np.random.default_rng(5)
    ref_b, ys, ref_x = {}, {}, {}
    for m in ANGLES:
        ref_b[m] = operator.forward_stages(xo, st, angles=np.array([m]))["data"][0]
        y = rng.standard_normal(ref_b[m].shape) + 1j * rng.standard_normal(ref_b[m].shape)
        ys[m] = y
        ref_x[m] = operator.adjoint_stages(y[None], st, angles=np.array([m]))["vol"]
    return dict(cfg=cfg, st=st, x=x, op=op, ref_b=ref_b, ys=ys, ref_x=ref_x)


@pytest.mark.parametrize("path", PATHS)
def test_full_size_sampled_angles_match_the_oracle(big, path):
    from paper_2511_06627_gb300 import MpiFflError

    op, st = big["op"], big["st"]
    try:
        op.set_path(path)
    except MpiFflError:
        pytest.skip(f"path {path} does not take this shape")
    b = op.forward(torch.from_numpy(big["x"]).cuda()).cpu().numpy().astype(np.float64)
    for m in ANGLES:
        got = b[m, ..., 0] + 1j * b[m, ..., 1]
        assert rel_l2(got, big["ref_b"][m]) < OP_TOL, (path, m)
        y_full = np.zeros(st.data_shape, dtype=np.complex128)
        y_full[m] = big["ys"][m]
        y_dev = torch.from_numpy(np.stack([y_full.real, y_full.imag], -1).astype(np.float32)).cuda()
        xa = op.adjoint(y_dev).cpu().numpy().astype(np.float64)
        assert rel_l2(xa, big["ref_x"][m]) < OP_TOL, (path, m)
    op.sync_check()


def test_full_size_adjoint_identity(big):
    """<A x, y> = <x, A^T y> over all 36 angles, the inner products in FP64 on the device."""
    op = big["op"]
    op.set_path("full_gemm")
    x = torch.from_numpy(big["x"]).cuda()
    g = torch.Generator(device="cuda").manual_seed(3)
    y = torch.randn(op.data_shape, device="cuda", generator=g)
    ax, aty = op.forward(x), op.adjoint(y)
    lhs = float(op.dot(ax, y))
    rhs = float(op.dot(x, aty))
    # relative to the Cauchy-Schwarz bound: FP32 operator error of ~1e-6 rel-L2
    scale = max(float(op.dot(ax, ax)) * float(op.dot(y, y)), float(op.dot(x, x)) * float(op.dot(aty, aty))) ** 0.5
    assert abs(lhs - rhs) <= 1e-5 * scale
