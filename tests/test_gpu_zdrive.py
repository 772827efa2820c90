"""The z-drive scan of the dual-drive acquisition (Sec. 3.1) on the GPU against the
FP64 oracle: every z stage and its transpose, A_z and A_z^T end to end (rel-L2 1e-5),
the adjoint identity in FP64, and sampled angles at the benchmark's full size."""

import numpy as np
import pytest

from _helpers import OP_TOL, ensure_library, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Setup, zdrive  # noqa: E402
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


def _make(name):
    from paper_2511_06627_gb300 import FFLOperator

    kw = dict(CASES[name])
    gains = np.linspace(0.95, 1.05, kw["n_angles"]).astype(np.float32)
    st = Setup(**kw, gains=gains.astype(np.float64))
    op = FFLOperator(**kw, gains=gains)
    return st, op


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("name", list(CASES))
def test_z_stages_and_transposes(name):
    st, op = _make(name)
    rng = np.random.default_rng(11)
    M = st.n_angles
    proj = rng.standard_normal((M, st.nz, st.nx))
    cz = rng.standard_normal((M, st.nx, zdrive.n_fine_z(st)))
    sig = rng.standard_normal((M, st.nz, st.L))
    ang = np.arange(M)
    assert rel_l2(op.apply_stage_zdrive(1, _t(proj)).cpu().numpy(), zdrive.psf_fwd_z(proj, st)) < OP_TOL
    assert rel_l2(op.apply_stage_zdrive(1, _t(cz), transpose=True).cpu().numpy(), zdrive.psf_adj_z(cz, st)) < OP_TOL
    assert rel_l2(op.apply_stage_zdrive(2, _t(cz)).cpu().numpy(), zdrive.resample_fwd_z(cz, st, ang)) < OP_TOL
    got = op.apply_stage_zdrive(2, _t(sig), transpose=True).cpu().numpy()
    assert rel_l2(got, zdrive.resample_adj_z(sig, st, ang)) < OP_TOL
    op.sync_check()


@pytest.mark.parametrize("name", list(CASES))
def test_z_operator_and_transpose(name):
    st, op = _make(name)
    x = random_volume(st.nz, st.nx, seed=12).astype(np.float32)
    rng = np.random.default_rng(13)
    y = (rng.standard_normal(st.data_shape) + 1j * rng.standard_normal(st.data_shape)).astype(np.complex64)
    b = op.forward_zdrive(_t(x)).cpu().numpy()
    xa = op.adjoint_zdrive(_t(to_interleaved(y))).cpu().numpy()
    op.sync_check()
    assert rel_l2(b, to_interleaved(zdrive.forward_z(x, st))) < OP_TOL
    assert rel_l2(xa, zdrive.adjoint_z(y, st)) < OP_TOL


@pytest.mark.parametrize("name", list(CASES))
def test_fused_z_path_matches_the_staged_kernels(name):
    """A_z and A_z^T run E_z V_z B fused with S D F (the time signal is never stored);
    composed from the staged kernels they compute the same FP32 samples, up to the
    order of the sums."""
    st, op = _make(name)
    x = _t(random_volume(st.nz, st.nx, seed=16))
    b = op.forward_zdrive(x)
    staged = op.apply_stage(3, op.apply_stage_zdrive(2, op.apply_stage_zdrive(1, op.apply_stage(0, x))))
    assert rel_l2(b.cpu().numpy(), staged.cpu().numpy()) < 2e-6
    xa = op.adjoint_zdrive(b)
    s = op.apply_stage_zdrive(2, op.apply_stage(3, b, transpose=True), transpose=True)
    staged = op.apply_stage(0, op.apply_stage_zdrive(1, s, transpose=True), transpose=True)
    op.sync_check()
    assert rel_l2(xa.cpu().numpy(), staged.cpu().numpy()) < 2e-6


def test_fused_z_adjoint_is_deterministic():
    """The fused transpose sums every fine z cell in a fixed order: two calls agree bit
    for bit."""
    st, op = _make("ragged")
    g = torch.Generator(device="cuda").manual_seed(17)
    y = torch.randn(op.data_shape, device="cuda", generator=g)
    a = op.adjoint_zdrive(y)
    b = op.adjoint_zdrive(y)
    op.sync_check()
    assert torch.equal(a, b)


def test_z_adjoint_identity_and_zero_input():
    st, op = _make("tiny")
    x = torch.from_numpy(random_volume(st.nz, st.nx, seed=14).astype(np.float32)).cuda()
    g = torch.Generator(device="cuda").manual_seed(15)
    y = torch.randn(op.data_shape, device="cuda", generator=g)
    ax, aty = op.forward_zdrive(x), op.adjoint_zdrive(y)
    lhs, rhs = float(op.dot(ax, y)), float(op.dot(x, aty))
    scale = (float(op.dot(ax, ax)) * float(op.dot(y, y))) ** 0.5
    assert abs(lhs - rhs) <= 1e-6 * scale
    assert float(op.forward_zdrive(torch.zeros_like(x)).abs().max()) == 0.0


def test_z_full_size_sampled_angles():
    """The 256^2 x 128, 36-angle workload: A_z x on the phantom and A_z^T y for random
    y, for a row-marched and a column-marched angle, against the oracle."""
    from paper_2511_06627_gb300 import FFLOperator

    cfg = config("invivo")
    st = Setup.from_config(cfg)
    x = phantom_for(cfg)
    op = FFLOperator.from_config(cfg)
    b = op.forward_zdrive(torch.from_numpy(x).cuda()).cpu().numpy().astype(np.float64)
    rng = np.random.default_rng(16)
    for m in (0, 20):
        ref = zdrive.forward_stages_z(x.astype(np.float64), st, angles=np.array([m]))["data"][0]
        assert rel_l2(b[m, ..., 0] + 1j * b[m, ..., 1], ref) < OP_TOL
        y = rng.standard_normal(ref.shape) + 1j * rng.standard_normal(ref.shape)
        y_full = np.zeros(st.data_shape, dtype=np.complex128)
        y_full[m] = y
        xa = op.adjoint_zdrive(torch.from_numpy(to_interleaved(y_full).astype(np.float32)).cuda()).cpu().numpy()
        ref_x = zdrive.adjoint_stages_z(y[None], st, angles=np.array([m]))["vol"]
        assert rel_l2(xa, ref_x) < OP_TOL
    op.sync_check()
