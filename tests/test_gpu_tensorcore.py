"""Parity of the tensor-core (tcgen05) line kernels with the FP64 oracle.

With precision BF16X3 the forward fuses E V B with the band DFT and the adjoint
fuses the band synthesis with the transposed resampling; both must match the
oracle within the FP32 operator tolerance (rel-L2 1e-5)."""

import numpy as np
import pytest

from _helpers import OP_TOL, ensure_library, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Setup, operator  # noqa: E402
from oracle.data import to_interleaved  # noqa: E402
from phantoms import config, phantom_for, random_volume  # noqa: E402

CASES = {
    "tiny": {k: config("tiny")[k] for k in ("nx", "nz", "n_angles", "S", "P", "A", "phi0", "zigzag", "Q", "fwhm",
                                             "k_min", "k_max", "half_width")},
    # S = 128 (one line per MMA tile), odd line count per trajectory, k_min > 1, no zig-zag
    "s128": dict(nx=40, nz=6, n_angles=5, S=128, P=128, A=5.0, phi0=0.2, zigzag=0, Q=8, fwhm=2.5,
                 k_min=2, k_max=6, half_width=4),
    # S = 64 with zig-zag, P = 256, seven kept bins per harmonic, D_Gamma
    "s64": dict(nx=36, nz=5, n_angles=3, S=64, P=256, A=6.0, phi0=0.0, zigzag=1, Q=8, fwhm=3.0,
                k_min=1, k_max=5, half_width=3, gamma=True),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


def _make(name, precision):
    from paper_2511_06627_gb300 import FFLOperator

    kw = dict(CASES[name])
    gamma = kw.pop("gamma", False)
    nb = (kw["k_max"] - kw["k_min"] + 1) * (2 * kw["half_width"] + 1)
    dg = None
    if gamma:
        q = np.arange(nb)
        dg = ((0.6 + 0.4 * np.sin(q)) * np.exp(-0.4j * q)).astype(np.complex64)
    gains = np.linspace(1.05, 0.95, kw["n_angles"]).astype(np.float32)
    st = Setup(**kw, gains=gains.astype(np.float64), d_gamma=None if dg is None else dg.astype(np.complex128))
    op = FFLOperator(**kw, gains=gains, d_gamma=dg, precision=precision)
    return st, op


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("name", list(CASES))
def test_bf16x3_forward_matches_oracle(name):
    from paper_2511_06627_gb300 import PREC_BF16X3

    st, op = _make(name, PREC_BF16X3)
    x = random_volume(st.nz, st.nx, seed=31).astype(np.float32)
    b = op.forward(_t(x))
    op.sync_check()
    ref = to_interleaved(operator.forward(x, st))
    assert rel_l2(b.cpu().numpy(), ref) < OP_TOL


@pytest.mark.parametrize("name", list(CASES))
def test_bf16x3_adjoint_matches_oracle(name):
    from paper_2511_06627_gb300 import PREC_BF16X3

    st, op = _make(name, PREC_BF16X3)
    rng = np.random.default_rng(32)
    y = (rng.standard_normal(st.data_shape) + 1j * rng.standard_normal(st.data_shape)).astype(np.complex64)
    x = op.adjoint(_t(to_interleaved(y)))
    op.sync_check()
    ref = operator.adjoint(y, st)
    assert rel_l2(x.cpu().numpy(), ref) < OP_TOL


def test_bf16x3_phantom_forward_matches_fp32_path():
    from paper_2511_06627_gb300 import PREC_BF16X3, PREC_FP32

    cfg = config("tiny")
    st, op = _make("tiny", PREC_FP32)
    x = _t(phantom_for(cfg))
    b32 = op.forward(x).clone()
    op.set_precision(PREC_BF16X3)
    b3 = op.forward(x)
    op.sync_check()
    assert rel_l2(b3.cpu().numpy(), b32.cpu().numpy()) < OP_TOL


def test_unsupported_shape_refuses_tensor_cores():
    from paper_2511_06627_gb300 import PREC_BF16X3, FFLOperator, MpiFflError

    op = FFLOperator(nx=16, nz=3, n_angles=2, S=24, P=10, A=3.0, Q=4, fwhm=2.0, k_min=1, k_max=3, half_width=1)
    with pytest.raises(MpiFflError):
        op.set_precision(PREC_BF16X3)


def test_handles_of_different_shapes_coexist():
    """Kernel launch attributes are process-wide: a later handle with a smaller
    shared-memory carve-up must not break an earlier, larger one."""
    from paper_2511_06627_gb300 import PREC_BF16X3

    st_big, op_big = _make("s64", PREC_BF16X3)
    st_small, op_small = _make("tiny", PREC_BF16X3)
    x = random_volume(st_big.nz, st_big.nx, seed=33).astype(np.float32)
    b = op_big.forward(_t(x))
    op_big.sync_check()
    assert rel_l2(b.cpu().numpy(), to_interleaved(operator.forward(x, st_big))) < OP_TOL
