"""The tensor PSF (Appendix B, Eq. (31)) and the receive-coil map (operator B) on the
GPU against the FP64 oracle: A and A^T with the slice-coupled PSF on three shapes and
both operand splits (rel-L2 1e-5), the coil map on the collinear model, the adjoint
identity, switching models back and forth, and a sampled angle at the benchmark's
full size."""

import numpy as np
import pytest

from _helpers import OP_TOL, ensure_library, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Setup, operator, tensor_psf  # noqa: E402
from oracle.data import to_interleaved  # noqa: E402
from phantoms import config, phantom_for, random_volume  # noqa: E402

KEYS = ("nx", "nz", "n_angles", "S", "P", "A", "phi0", "zigzag", "Q", "fwhm", "k_min", "k_max", "half_width")
CASES = {
    "tiny": {k: config("tiny")[k] for k in KEYS},
    "ragged": dict(nx=21, nz=7, n_angles=5, S=24, P=10, A=3.5, phi0=0.3, zigzag=1, Q=4, fwhm=2.5,
                   k_min=1, k_max=3, half_width=2),
    "tall": dict(nx=20, nz=26, n_angles=3, S=32, P=20, A=4.0, phi0=0.0, zigzag=0, Q=8, fwhm=3.0,
                 k_min=2, k_max=5, half_width=1),
}


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


def _make(name, path="full_gemm"):
    from paper_2511_06627_gb300 import FFLOperator

    kw = dict(CASES[name])
    gains = np.linspace(0.95, 1.05, kw["n_angles"]).astype(np.float32)
    st = Setup(**kw, gains=gains.astype(np.float64))
    op = FFLOperator(**kw, gains=gains)
    op.set_path(path)
    return st, op


def _coil(st, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.4, 1.6, (st.nz, st.nx)).astype(np.float32)


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _data(st, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(st.data_shape) + 1j * rng.standard_normal(st.data_shape)


@pytest.mark.parametrize("precision", ["bf16x3", "tf32"])
@pytest.mark.parametrize("name", list(CASES))
def test_tensor_operator_and_transpose(name, precision):
    st, op = _make(name)
    if precision == "tf32":
        from paper_2511_06627_gb300._lib import PREC_TF32

        op.set_precision(PREC_TF32)
    coil = _coil(st, 21)
    op.set_psf_model("tensor")
    op.set_coil_map(coil)
    x = random_volume(st.nz, st.nx, seed=22).astype(np.float32)
    y = _data(st, 23).astype(np.complex64)
    b = op.forward(_t(x)).cpu().numpy()
    xa = op.adjoint(_t(to_interleaved(y))).cpu().numpy()
    op.sync_check()
    assert rel_l2(b, to_interleaved(tensor_psf.forward(x, st, coil.astype(np.float64)))) < OP_TOL
    assert rel_l2(xa, tensor_psf.adjoint(y, st, coil.astype(np.float64))) < OP_TOL


def test_tensor_with_more_angles_than_a_tile():
    """130 angles: one line per problem and A rows over two 128-row tiles."""
    from paper_2511_06627_gb300 import FFLOperator

    kw = dict(nx=16, nz=5, n_angles=130, S=24, P=10, A=3.0, phi0=0.2, zigzag=1, Q=4, fwhm=2.0,
              k_min=1, k_max=3, half_width=1)
    gains = np.linspace(0.9, 1.1, 130).astype(np.float32)
    st = Setup(**kw, gains=gains.astype(np.float64))
    op = FFLOperator(**kw, gains=gains)
    op.set_path("full_gemm")
    op.set_psf_model("tensor")
    coil = _coil(st, 31)
    op.set_coil_map(coil)
    x = random_volume(st.nz, st.nx, seed=32).astype(np.float32)
    y = _data(st, 33).astype(np.complex64)
    b = op.forward(_t(x)).cpu().numpy()
    xa = op.adjoint(_t(to_interleaved(y))).cpu().numpy()
    op.sync_check()
    assert rel_l2(b, to_interleaved(tensor_psf.forward(x, st, coil.astype(np.float64)))) < OP_TOL
    assert rel_l2(xa, tensor_psf.adjoint(y, st, coil.astype(np.float64))) < OP_TOL


def test_tensor_adjoint_identity_and_model_switch():
    st, op = _make("ragged")
    x = _t(random_volume(st.nz, st.nx, seed=24))
    g = torch.Generator(device="cuda").manual_seed(25)
    y = torch.randn(op.data_shape, device="cuda", generator=g)
    b_col = op.forward(x)
    op.set_psf_model("tensor")
    assert op.psf_model == 1
    b = op.forward(x)
    xa = op.adjoint(y)
    lhs, rhs = float(op.dot(b, y)), float(op.dot(x, xa))
    scale = (float(op.dot(b, b)) * float(op.dot(y, y))) ** 0.5
    assert abs(lhs - rhs) <= 1e-6 * scale
    assert rel_l2(b.cpu().numpy(), b_col.cpu().numpy()) > 1e-2  # the slices do couple
    op.set_psf_model("collinear")
    assert torch.equal(op.forward(x), b_col)
    op.sync_check()


def _collinear_with_coil(x, st, coil):
    """Oracle composition of the collinear model with B's coil map (before H)."""
    from oracle import projection

    out = np.empty(st.data_shape, dtype=np.complex128)
    for m in range(st.n_angles):
        ang = np.array([m])
        proj = tensor_psf.coil_apply(projection.project(x, st.angles[ang]), coil)
        sig = operator.resample_fwd(operator.psf_fwd(proj, st), st, ang)
        out[m] = operator.compress_fwd(sig, st)[0]
    return out


@pytest.mark.parametrize("path", ["staged", "full_gemm"])
def test_coil_map_on_the_collinear_model(path):
    from oracle import projection

    st, op = _make("tiny", path)
    coil = _coil(st, 26)
    op.set_coil_map(coil)
    x = random_volume(st.nz, st.nx, seed=27).astype(np.float32)
    ref = _collinear_with_coil(x.astype(np.float64), st, coil.astype(np.float64))
    assert rel_l2(op.forward(_t(x)).cpu().numpy(), to_interleaved(ref)) < OP_TOL
    y = _data(st, 28)
    vol = np.zeros((st.nz, st.nx, st.nx))
    for m in range(st.n_angles):
        ang = np.array([m])
        sig = operator.compress_adj(y[m:m + 1], st)
        pb = operator.psf_adj(operator.resample_adj(sig, st, ang), st)
        vol += projection.backproject(tensor_psf.coil_apply(pb, coil.astype(np.float64)), st.angles[ang], st.nx)
    xa = op.adjoint(_t(to_interleaved(y.astype(np.complex64)))).cpu().numpy()
    assert rel_l2(xa, vol) < OP_TOL
    op.set_coil_map(None)
    b0 = op.forward(_t(x)).cpu().numpy()
    assert rel_l2(b0, to_interleaved(operator.forward(x.astype(np.float64), st))) < OP_TOL
    op.sync_check()


def test_tensor_full_size_sampled_angle():
    """The 256^2 x 128, 36-angle workload with the tensor PSF: A x on the phantom and
    A^T y for y on one angle, against the oracle, for a column-marched angle."""
    from paper_2511_06627_gb300 import FFLOperator

    cfg = config("invivo")
    st = Setup.from_config(cfg)
    x = phantom_for(cfg)
    op = FFLOperator.from_config(cfg)
    op.set_path("full_gemm")
    op.set_psf_model("tensor")
    b = op.forward(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    m = 20
    ref = tensor_psf.forward_stages(x.astype(np.float64), st, None, angles=np.array([m]))["data"][0]
    assert rel_l2(b[m, ..., 0] + 1j * b[m, ..., 1], ref) < OP_TOL
    rng = np.random.default_rng(29)
    y = rng.standard_normal(ref.shape) + 1j * rng.standard_normal(ref.shape)
    y_full = np.zeros(st.data_shape, dtype=np.complex128)
    y_full[m] = y
    xa = op.adjoint(torch.from_numpy(to_interleaved(y_full).astype(np.float32)).cuda()).cpu().numpy()
    ref_x = tensor_psf.adjoint_stages(y[None], st, None, angles=np.array([m]))["vol"]
    assert rel_l2(xa, ref_x) < OP_TOL
    op.sync_check()
