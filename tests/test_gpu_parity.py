"""Parity of the CUDA path with the FP64 oracle, stage by stage and end to end.

Every case runs the library through its C ABI (via the Python binding) and
compares element by element with the oracle on the same seeded inputs; the
FP32 operator tolerance is rel-L2 1e-5.
"""

import math

import numpy as np
import pytest

from _helpers import OP_TOL, ensure_library, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import Setup, operator  # noqa: E402
from oracle.data import from_interleaved, to_interleaved  # noqa: E402
from phantoms import config, phantom_for, random_volume  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


CASES = {
    # the tiny recipe itself
    "tiny": dict(config("tiny")),
    # ragged sizes: odd N, odd N_z, S not a power of two, a 45 deg tie and 90 deg
    "ragged": dict(nx=21, nz=5, n_angles=7, S=24, P=10, A=3.5, phi0=0.3, zigzag=1, Q=4, fwhm=2.5,
                   k_min=1, k_max=3, half_width=2,
                   angles=[0.0, math.pi / 4, 0.9, math.pi / 2, 2.0, 3 * math.pi / 4, 3.0]),
    # no zig-zag, k_min > 1 (the paper keeps harmonics 2..5), non-identity D_Gamma
    "bands": dict(nx=24, nz=6, n_angles=5, S=32, P=16, A=4.0, phi0=0.0, zigzag=0, Q=8, fwhm=3.0,
                  k_min=2, k_max=5, half_width=3, gamma=True),
}


def _make(name):
    from paper_2511_06627_gb300 import FFLOperator

    c = dict(CASES[name])
    angles = c.pop("angles", None)
    gamma = c.pop("gamma", False)
    keys = ("nx", "nz", "n_angles", "S", "P", "A", "phi0", "zigzag", "Q", "fwhm", "k_min", "k_max", "half_width")
    kw = {k: c[k] for k in keys}
    nb = (kw["k_max"] - kw["k_min"] + 1) * (2 * kw["half_width"] + 1)
    dg = None
    if gamma:
        q = np.arange(nb)
        dg = (0.5 + 0.5 * np.cos(q)) * np.exp(0.7j * q)  # magnitude and phase per kept bin
    gains = np.linspace(0.9, 1.1, kw["n_angles"]).astype(np.float32).astype(np.float64)
    st = Setup(**kw, angles=None if angles is None else np.array(angles), gains=gains,
               d_gamma=None if dg is None else dg.astype(np.complex64).astype(np.complex128))
    op = FFLOperator(**kw, angles=angles, gains=gains, d_gamma=dg)
    return st, op


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _n(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("name", list(CASES))
def test_stages_forward(name):
    st, op = _make(name)
    x = random_volume(st.nz, st.nx, seed=11).astype(np.float32)
    ref = operator.forward_stages(x, st)
    # each stage fed with the oracle's own (float32-rounded) input
    proj = _n(op.apply_stage(0, _t(x)))
    assert rel_l2(proj, ref["proj"]) < OP_TOL
    fine = _n(op.apply_stage(1, _t(ref["proj"])))
    assert rel_l2(fine, operator.psf_fwd(ref["proj"].astype(np.float32), st)) < OP_TOL
    sig = _n(op.apply_stage(2, _t(ref["fine"])))
    assert rel_l2(sig, operator.resample_fwd(ref["fine"].astype(np.float32), st)) < OP_TOL
    data = _n(op.apply_stage(3, _t(ref["sig"])))
    exp = operator.compress_fwd(ref["sig"].astype(np.float32), st)
    assert rel_l2(data, to_interleaved(exp)) < OP_TOL
    b = _n(op.forward(_t(x)))
    assert rel_l2(b, to_interleaved(ref["data"])) < OP_TOL


@pytest.mark.parametrize("name", list(CASES))
def test_stages_adjoint(name):
    st, op = _make(name)
    rng = np.random.default_rng(12)
    y = (rng.standard_normal(st.data_shape) + 1j * rng.standard_normal(st.data_shape)).astype(np.complex64)
    ref = operator.adjoint_stages(y, st)
    sig = _n(op.apply_stage(3, _t(to_interleaved(y)), transpose=True))
    assert rel_l2(sig, ref["sig"]) < OP_TOL
    fine = _n(op.apply_stage(2, _t(ref["sig"]), transpose=True))
    assert rel_l2(fine, operator.resample_adj(ref["sig"].astype(np.float32), st)) < OP_TOL
    proj = _n(op.apply_stage(1, _t(ref["fine"]), transpose=True))
    assert rel_l2(proj, operator.psf_adj(ref["fine"].astype(np.float32), st)) < OP_TOL
    from oracle import projection

    vol = _n(op.apply_stage(0, _t(ref["proj"]), transpose=True))
    assert rel_l2(vol, projection.backproject(ref["proj"].astype(np.float32), st.angles, st.nx)) < OP_TOL
    x = _n(op.adjoint(_t(to_interleaved(y))))
    assert rel_l2(x, ref["vol"]) < OP_TOL


@pytest.mark.parametrize("name", list(CASES))
def test_adjoint_dot_product_on_gpu(name):
    st, op = _make(name)
    x = _t(random_volume(st.nz, st.nx, seed=13))
    y = _t(np.random.default_rng(14).standard_normal(op.data_shape))
    ax = op.forward(x)
    aty = op.adjoint(y)
    lhs = float((ax.double() * y.double()).sum())
    rhs = float((x.double() * aty.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * float(ax.double().norm() * y.double().norm())


def test_phantom_forward_and_adjoint_match_oracle():
    """The tiny recipe's phantom through A and A^T, end to end."""
    cfg = config("tiny")
    st, op = _make("tiny")
    x = phantom_for(cfg)
    b = _n(op.forward(_t(x)))
    bref = operator.forward(x, st)
    assert rel_l2(b, to_interleaved(bref)) < OP_TOL
    xa = _n(op.adjoint(_t(to_interleaved(bref))))
    assert rel_l2(xa, operator.adjoint(from_interleaved(to_interleaved(bref).astype(np.float32)), st)) < OP_TOL


def test_empty_volume_gives_zero_data():
    st, op = _make("ragged")
    b = _n(op.forward(torch.zeros(op.vol_shape, device="cuda")))
    assert np.all(b == 0.0)
    x = _n(op.adjoint(torch.zeros(op.data_shape, device="cuda")))
    assert np.all(x == 0.0)


def test_ttt_matches_oracle():
    from oracle import regularizer

    st, op = _make("ragged")
    x = random_volume(st.nz, st.nx, seed=15).astype(np.float32)
    assert rel_l2(_n(op.apply_ttt(_t(x))), regularizer.ttt(x)) < OP_TOL


def test_dot_f64_matches_numpy():
    st, op = _make("ragged")
    rng = np.random.default_rng(16)
    a = rng.standard_normal(100003).astype(np.float32)
    b = rng.standard_normal(100003).astype(np.float32)
    got = float(op.dot(_t(a), _t(b)).cpu())
    ref = float(np.dot(a.astype(np.float64), b.astype(np.float64)))
    assert abs(got - ref) <= 1e-12 * np.linalg.norm(a) * np.linalg.norm(b)
    assert float(op.dot(_t(a[:0]), _t(b[:0])).cpu()) == 0.0


@pytest.mark.parametrize("overlap", [False, True])
@pytest.mark.parametrize("pinned", [False, True])
def test_host_buffers_equal_device_buffers(overlap, pinned):
    """forward/adjoint given host tensors stage them through the handle and give the
    same bits as with device tensors, over several calls in a row (both staging slots,
    inputs changing between calls)."""
    from paper_2511_06627_gb300 import FFLOperator

    kw = {k: config("tiny")[k] for k in ("nx", "nz", "n_angles", "S", "P", "A", "phi0", "zigzag", "Q", "fwhm",
                                         "k_min", "k_max", "half_width")}
    op = FFLOperator(**kw)
    op.set_path("full_gemm")
    op.set_host_overlap(overlap)
    st = Setup(**kw)
    rng = np.random.default_rng(7)
    xs = [rng.random((st.nz, st.nx, st.nx), dtype=np.float32) for _ in range(4)]
    ys = [rng.standard_normal(op.data_shape).astype(np.float32) for _ in range(4)]

    def host(a):
        t = torch.from_numpy(a.copy())
        return t.pin_memory() if pinned else t

    hx, hy = [host(a) for a in xs], [host(a) for a in ys]
    hb = [host(np.zeros(op.data_shape, np.float32)) for _ in range(4)]
    hxa = [host(np.zeros((st.nz, st.nx, st.nx), np.float32)) for _ in range(4)]
    for k in range(4):
        op.forward(hx[k], out=hb[k])
        op.adjoint(hy[k], out=hxa[k])
    torch.cuda.synchronize()
    op.sync_check()
    for k in range(4):
        bd = op.forward(torch.from_numpy(xs[k]).cuda())
        xd = op.adjoint(torch.from_numpy(ys[k]).cuda())
        torch.cuda.synchronize()
        assert np.array_equal(hb[k].numpy(), bd.cpu().numpy())
        assert np.array_equal(hxa[k].numpy(), xd.cpu().numpy())
    # mixed: device in, host out and host in, device out
    b_dev = op.new_data()
    op.forward(hx[0], out=b_dev)
    out_h = host(np.zeros((st.nz, st.nx, st.nx), np.float32))
    op.adjoint(b_dev, out=out_h)
    torch.cuda.synchronize()
    ref = op.adjoint(op.forward(torch.from_numpy(xs[0]).cuda()))
    torch.cuda.synchronize()
    assert np.array_equal(out_h.numpy(), ref.cpu().numpy())


def test_compression_analysis_matches_the_oracle():
    """I(s, S) of Eq. (30) from the GPU band energies, for every sub-band (harmonics
    1..K, |delta| <= w) of the kept bins, against the oracle's literal Eq. (30) on the
    symmetric bin set S u (L - S) of its FP64 time signal."""
    from paper_2511_06627_gb300 import FFLOperator

    cfg = config("tiny")
    kw = {k: cfg[k] for k in ("nx", "nz", "n_angles", "S", "P", "A", "phi0", "zigzag", "Q", "fwhm",
                              "k_min", "k_max", "half_width")}
    st = Setup(**kw)
    x = phantom_for(cfg)
    op = FFLOperator(**kw)
    Ks = list(range(cfg["k_min"], cfg["k_max"] + 1))
    ws = list(range(0, cfg["half_width"] + 1))
    got = op.information_retained(torch.from_numpy(x).cuda(), Ks, ws)
    sig = operator.forward_stages(x.astype(np.float64), st)["sig"]
    L = st.S * st.P
    for a, K in enumerate(Ks):
        for c, w in enumerate(ws):
            k = np.arange(cfg["k_min"], K + 1)
            d = np.arange(-w, w + 1)
            bins = (k[:, None] * st.P + d[None, :]).reshape(-1)
            ref = operator.information_retained(sig, np.concatenate([bins, L - bins]))
            assert abs(got[a, c] - ref) <= 1e-5 * ref, (K, w, got[a, c], ref)
    # monotone in both the harmonic count and the bandwidth, and at most 1
    assert np.all(np.diff(got, axis=0) >= 0) and np.all(np.diff(got, axis=1) >= 0) and got.max() <= 1.0


@pytest.mark.parametrize("n", [300, 320, 512])
def test_projector_pair_on_wide_detectors(n):
    """Above 256 bins the interleaved projector stages each march line with two tensor
    copies (boxes of at most 256 positions, zero fill past the line's end), and N = 300 is
    not a multiple of the 32 rays of a warp: P and P^T (Sec. 2.2, Eq. (19)) against the
    oracle, with a 45 deg tie and 90 deg among the angles and a ragged slice block."""
    from oracle import projection
    from paper_2511_06627_gb300 import FFLOperator

    nz = 9
    angles = [0.0, 0.3, math.pi / 4, 1.2, math.pi / 2, 2.5]
    kw = dict(nx=n, nz=nz, n_angles=len(angles), S=32, P=16, A=4.0, phi0=0.0, zigzag=1, Q=4, fwhm=2.5,
              k_min=1, k_max=3, half_width=2)
    op = FFLOperator(**kw, angles=angles)
    x = random_volume(nz, n, seed=47).astype(np.float32)
    p = _n(op.project(_t(x)))
    assert rel_l2(p, projection.project(x.astype(np.float64), angles)) < OP_TOL
    rng = np.random.default_rng(48)
    q = rng.standard_normal((len(angles), nz, n)).astype(np.float32)
    v = _n(op.backproject(_t(q)))
    assert rel_l2(v, projection.backproject(q.astype(np.float64), angles, n)) < OP_TOL
