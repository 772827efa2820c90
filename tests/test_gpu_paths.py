"""Every evaluation path of A and A^T (staged FP32, fused tensor-core, line GEMM,
full GEMM) against the FP64 oracle, within the FP32 operator tolerance."""

import math

import numpy as np
import pytest

from _helpers import OP_TOL, ensure_library, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Setup, operator  # noqa: E402
from oracle.data import to_interleaved  # noqa: E402
from phantoms import config, random_volume  # noqa: E402

KEYS = ("nx", "nz", "n_angles", "S", "P", "A", "phi0", "zigzag", "Q", "fwhm", "k_min", "k_max", "half_width")
CASES = {
    "tiny": {k: config("tiny")[k] for k in KEYS},
    "ragged": dict(nx=21, nz=5, n_angles=7, S=24, P=10, A=3.5, phi0=0.3, zigzag=1, Q=4, fwhm=2.5,
                   k_min=1, k_max=3, half_width=2),
    "s128": dict(nx=40, nz=6, n_angles=5, S=128, P=128, A=5.0, phi0=0.2, zigzag=0, Q=8, fwhm=2.5,
                 k_min=2, k_max=6, half_width=4),
    "wide_band": dict(nx=48, nz=4, n_angles=4, S=64, P=128, A=6.0, phi0=0.0, zigzag=1, Q=8, fwhm=3.0,
                      k_min=1, k_max=16, half_width=4, gamma=True),
    # 64-bin detectors: the full-GEMM forward takes its A operand from the projector
    "n64_zigzag": dict(nx=64, nz=5, n_angles=3, S=24, P=10, A=3.5, phi0=0.1, zigzag=1, Q=4, fwhm=2.5,
                       k_min=1, k_max=3, half_width=2),
    "n64_plain": dict(nx=64, nz=10, n_angles=4, S=32, P=12, A=4.0, phi0=0.25, zigzag=0, Q=4, fwhm=2.0,
                      k_min=1, k_max=4, half_width=2),
    # the widest detector the library takes (512 bins): the plain projector, 512-row GEMMs
    "n512": dict(nx=512, nz=3, n_angles=3, S=32, P=16, A=4.0, phi0=0.1, zigzag=1, Q=4, fwhm=2.5,
                 k_min=1, k_max=3, half_width=2),
}
PATHS = ["staged", "fused", "line_gemm", "full_gemm"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


def _make(name):
    from paper_2511_06627_gb300 import FFLOperator

    kw = dict(CASES[name])
    gamma = kw.pop("gamma", False)
    nb = (kw["k_max"] - kw["k_min"] + 1) * (2 * kw["half_width"] + 1)
    dg = None
    if gamma:
        q = np.arange(nb)
        dg = ((0.7 + 0.3 * np.cos(0.5 * q)) * np.exp(0.3j * q)).astype(np.complex64)
    gains = np.linspace(0.97, 1.04, kw["n_angles"]).astype(np.float32)
    st = Setup(**kw, gains=gains.astype(np.float64), d_gamma=None if dg is None else dg.astype(np.complex128))
    op = FFLOperator(**kw, gains=gains, d_gamma=dg)
    return st, op


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _set(op, path):
    from paper_2511_06627_gb300 import MpiFflError

    try:
        op.set_path(path)
    except MpiFflError:
        pytest.skip(f"path {path} does not take this shape")


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("name", list(CASES))
def test_path_forward_and_adjoint(name, path):
    st, op = _make(name)
    _set(op, path)
    x = random_volume(st.nz, st.nx, seed=41).astype(np.float32)
    b = op.forward(_t(x))
    rng = np.random.default_rng(42)
    y = (rng.standard_normal(st.data_shape) + 1j * rng.standard_normal(st.data_shape)).astype(np.complex64)
    xa = op.adjoint(_t(to_interleaved(y)))
    op.sync_check()
    assert rel_l2(b.cpu().numpy(), to_interleaved(operator.forward(x, st))) < OP_TOL
    assert rel_l2(xa.cpu().numpy(), operator.adjoint(y, st)) < OP_TOL


@pytest.mark.parametrize("tf32", [False, True])
@pytest.mark.parametrize("name", ["n64_zigzag", "n64_plain"])
def test_projector_packed_operand_matches_the_packing_pass(name, tf32):
    """With N a multiple of the K chunk (64 bins in bf16, 32 in tf32) the full-GEMM
    forward splits the projector's sums into the GEMM's hi + lo operand inside the
    projector; the projections through the stage entry points (stored, then split by the
    GEMM or its packing pass) give the same bits."""
    from paper_2511_06627_gb300 import PREC_TF32

    st, op = _make(name)
    op.set_path("full_gemm")
    if tf32:
        op.set_precision(PREC_TF32)
    x = _t(random_volume(st.nz, st.nx, seed=45).astype(np.float32))
    b = op.forward(x)
    b_stages = op.line_forward(op.project(x))
    op.sync_check()
    assert torch.equal(b, b_stages)
    assert torch.equal(op.forward(x), b)  # repeatable


def test_gemm_paths_take_every_shape():
    for name in CASES:
        st, op = _make(name)
        op.set_path("line_gemm")
        op.set_path("full_gemm")
        assert op.path == 3


@pytest.mark.parametrize("path", ["line_gemm", "full_gemm"])
@pytest.mark.parametrize("name", ["s128", "wide_band"])
def test_tf32_split_is_closer_to_the_oracle_than_bf16_split(name, path):
    """The tf32 hi + lo operands keep 22 mantissa bits against the bf16 split's 16,
    so the GEMM term of the error shrinks; both stay inside the operator tolerance."""
    from paper_2511_06627_gb300 import PREC_BF16X3, PREC_TF32

    st, op = _make(name)
    op.set_path(path)
    x = random_volume(st.nz, st.nx, seed=43).astype(np.float32)
    rng = np.random.default_rng(44)
    y = (rng.standard_normal(st.data_shape) + 1j * rng.standard_normal(st.data_shape)).astype(np.complex64)
    ref_f = to_interleaved(operator.forward(x, st))
    ref_a = operator.adjoint(y, st)
    err = {}
    for prec in (PREC_BF16X3, PREC_TF32):
        op.set_precision(prec)
        assert op.path == PATHS.index(path)
        b = op.forward(_t(x))
        xa = op.adjoint(_t(to_interleaved(y)))
        op.sync_check()
        err[prec] = (rel_l2(b.cpu().numpy(), ref_f), rel_l2(xa.cpu().numpy(), ref_a))
    for i in range(2):
        assert err[PREC_TF32][i] < OP_TOL
        assert err[PREC_TF32][i] <= err[PREC_BF16X3][i] * 1.01
    # switching between the GEMM paths keeps tf32
    op.set_path("line_gemm" if path == "full_gemm" else "full_gemm")
    assert op.precision == PREC_TF32


def test_tf32_is_refused_off_the_gemm_paths():
    from paper_2511_06627_gb300 import PREC_TF32, MpiFflError

    st, op = _make("tiny")
    for path in ("staged", "fused"):
        op.set_path(path)
        with pytest.raises(MpiFflError):
            op.set_precision(PREC_TF32)
