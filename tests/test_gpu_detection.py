"""The detection-limit analysis (Sec. 4.2, Fig. 5) on the GPU: box statistics against
the FP64 oracle (bit-equal repeats), and the detection limit of a reconstructed
synthetic sensitivity series against the oracle's analysis of the same volume."""

import math

import numpy as np
import pytest

from _helpers import ensure_library

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import detection  # noqa: E402
from phantoms import config, scaled_config  # noqa: E402
from phantoms.generators import sensitivity_series  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


def test_box_stats_match_the_oracle():
    from paper_2511_06627_gb300.operator import box_stats

    rng = np.random.default_rng(41)
    vol = rng.standard_normal((13, 21, 37)).astype(np.float32)
    boxes = [(0, 13, 0, 21, 0, 37), (2, 5, 3, 9, 30, 37), (12, 13, 20, 21, 36, 37), (4, 11, 0, 21, 5, 6)]
    dv = torch.from_numpy(vol).cuda()
    for pooled in (False, True):
        got = box_stats(dv, boxes, pooled)
        ref = detection.box_stats(vol, boxes, pooled)
        assert np.array_equal(got[:, 0], ref[:, 0]) and np.array_equal(got[:, 3], ref[:, 3])
        assert np.allclose(got[:, 1:3], ref[:, 1:3], rtol=1e-12, atol=1e-14)
        assert np.array_equal(box_stats(dv, boxes, pooled), got)  # fixed summation order


def test_box_stats_reject_boxes_outside_the_volume():
    from paper_2511_06627_gb300 import MpiFflError
    from paper_2511_06627_gb300.operator import box_stats

    dv = torch.zeros((4, 5, 6), device="cuda")
    for bad in [(0, 5, 0, 5, 0, 6), (1, 1, 0, 5, 0, 6), (0, 4, -1, 5, 0, 6)]:
        with pytest.raises(MpiFflError):
            box_stats(dv, [bad])


def test_detection_limit_of_a_reconstructed_series():
    """Synthetic sensitivity series (5-50 units) at 64^2 x 32, 12 angles: b = A x plus
    complex noise at 0.5% of max |b|, 60 iterations of Eq. (26), then the analysis on
    the GPU against the oracle's analysis of the same reconstruction."""
    from paper_2511_06627_gb300 import FFLOperator
    from paper_2511_06627_gb300.operator import box_stats, detection_limit

    cfg = scaled_config("phantom", nx=64, nz=32, n_angles=12)
    amounts = [5.0, 10.0, 25.0, 50.0]
    vol, sboxes, vboxes = sensitivity_series(cfg["nx"], cfg["nz"], amounts, seed=3)
    op = FFLOperator.from_config(cfg)
    op.set_path("full_gemm")
    b = op.forward(torch.from_numpy(vol).cuda())
    rng = np.random.default_rng(5)
    sigma = 0.005 * float(b.abs().max())
    b += torch.from_numpy((sigma / math.sqrt(2) * rng.standard_normal(b.shape)).astype(np.float32)).cuda()
    x, _ = op.solve(b, iters=60)
    values = box_stats(x, sboxes)[:, 1]
    noise = box_stats(x, vboxes, pooled=True)[0, 2]
    got = detection_limit(amounts, values, noise)
    ref = detection.analyse(x.cpu().numpy(), sboxes, amounts, vboxes)
    assert np.allclose(values, ref["values"], rtol=1e-12)
    assert math.isclose(noise, ref["noise"], rel_tol=1e-12)
    assert math.isclose(got["limit"], ref["limit"], rel_tol=1e-9)
    assert got["slope"] > 0 and math.isfinite(got["limit"])
    op.sync_check()
