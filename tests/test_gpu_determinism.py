"""Run-to-run determinism on the GPU: every kernel of A, A^T and the solve sums in a
fixed order (no atomics), so repeating a call on the same input must give the same
bits. Checked at the full 256^2 x 128, 36-angle size on every path (staged, fused,
line-GEMM, full-GEMM), stage by stage, for a short solve, for the tensor-PSF operator and for the
z-drive scan."""

import pytest

from _helpers import ensure_library

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from phantoms import config, phantom_for  # noqa: E402


@pytest.fixture(scope="module")
def op_x():
    ensure_library()
    from paper_2511_06627_gb300 import FFLOperator

    cfg = config("invivo")
    op = FFLOperator.from_config(cfg)
    x = torch.from_numpy(phantom_for(cfg)).cuda()
    yield op, x
    op.close()


def _repeat(fn, n=3):
    first = fn().clone()
    bad = {}
    for k in range(1, n):
        out = fn()
        if not torch.equal(out, first):
            diff = (out - first).abs()
            bad[k] = (int((diff != 0).sum()), float(diff.max()))
    return bad


@pytest.mark.parametrize("path", ["staged", "fused", "line_gemm", "full_gemm"])
def test_operators_repeat_bit_for_bit(op_x, path):
    op, x = op_x
    op.set_path(path)
    b = op.forward(x).clone()
    p = op.project(x).clone()
    checks = {
        "project": lambda: op.project(x),
        "backproject": lambda: op.backproject(p),
        "line_forward": lambda: op.line_forward(p),
        "line_adjoint": lambda: op.line_adjoint(b),
        "forward": lambda: op.forward(x),
        "adjoint": lambda: op.adjoint(b),
    }
    bad = {name: r for name, fn in checks.items() if (r := _repeat(fn))}
    op.sync_check()
    assert not bad, f"results changed between calls (elements, max |diff|): {bad}"


def test_solve_repeats_bit_for_bit(op_x):
    op, x = op_x
    op.set_path("full_gemm")
    b = op.forward(x).clone()
    norms = [op.power_norm(20, 1234) for _ in range(2)]
    assert norms[0] == norms[1]
    bad = _repeat(lambda: op.solve(b, iters=30, ata_norm=norms[0], report=False)[0], n=2)
    op.sync_check()
    assert not bad, f"solve changed between calls: {bad}"


def test_tensor_psf_and_zdrive_repeat_bit_for_bit(op_x):
    """The slice-coupled tensor-PSF GEMMs (pre-split A staged by bulk copies, fixed-order
    sum of the K splits) and the fused z-drive kernels at the same size."""
    op, x = op_x
    op.set_path("full_gemm")
    op.set_psf_model("tensor")
    try:
        b = op.forward(x).clone()
        bad = {name: r for name, fn in {"tensor forward": lambda: op.forward(x),
                                        "tensor adjoint": lambda: op.adjoint(b)}.items() if (r := _repeat(fn))}
    finally:
        op.set_psf_model("collinear")
    bz = op.forward_zdrive(x).clone()
    bad.update({name: r for name, fn in {"z forward": lambda: op.forward_zdrive(x),
                                         "z adjoint": lambda: op.adjoint_zdrive(bz)}.items() if (r := _repeat(fn))})
    op.sync_check()
    assert not bad, f"results changed between calls (elements, max |diff|): {bad}"
