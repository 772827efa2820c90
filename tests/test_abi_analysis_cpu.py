"""The host-only least-squares crossing of the detection-limit analysis (Sec. 4.2,
Fig. 5) through the C ABI, against the oracle's fit, without a GPU."""

import math

import numpy as np
import pytest

from _helpers import ensure_library
from oracle import detection


@pytest.fixture(scope="module", autouse=True)
def _lib():
    ensure_library()


def test_detection_limit_matches_the_oracle():
    from paper_2511_06627_gb300.operator import detection_limit

    rng = np.random.default_rng(31)
    for _ in range(10):
        amounts = np.sort(rng.uniform(1, 60, rng.integers(2, 7)))
        values = 0.3 + 0.07 * amounts + rng.normal(0, 0.05, amounts.size)
        noise = rng.uniform(0.01, 0.2)
        got = detection_limit(amounts, values, noise)
        lim, s, a = detection.detection_limit(amounts, values, noise)
        assert math.isclose(got["slope"], s, rel_tol=1e-10) and math.isclose(got["intercept"], a, rel_tol=1e-10)
        assert math.isclose(got["limit"], lim, rel_tol=1e-9, abs_tol=1e-12)


def test_detection_limit_rejects_degenerate_input():
    from paper_2511_06627_gb300 import MpiFflError
    from paper_2511_06627_gb300.operator import detection_limit

    with pytest.raises(MpiFflError):
        detection_limit([1.0], [2.0], 0.1)
    with pytest.raises(MpiFflError):
        detection_limit([2.0, 2.0], [1.0, 3.0], 0.1)
    assert math.isnan(detection_limit([1.0, 2.0], [3.0, 1.0], 0.1)["limit"])  # falling line
