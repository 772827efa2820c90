"""Pins of the detection-limit analysis (Sec. 4.2, Fig. 5): hand-computed mean
absolute deviations, an exact line and its crossing, and the synthetic sensitivity
series' sample masses."""

import math

import numpy as np

from oracle import detection
from phantoms.generators import sensitivity_series


def test_mean_absolute_deviation_by_hand():
    vol = np.zeros((1, 2, 2))
    vol[0] = [[1.0, 2.0], [3.0, 4.0]]  # mean 2.5, |dev| = 1.5, 0.5, 0.5, 1.5
    st = detection.box_stats(vol, [(0, 1, 0, 2, 0, 2)])
    assert st.tolist() == [[4.0, 2.5, 1.0, 4.0]]


def test_pooled_boxes_are_one_region():
    vol = np.zeros((1, 1, 4))
    vol[0, 0] = [0.0, 0.0, 4.0, 4.0]  # boxes {0, 0} and {4, 4}: each MAD 0, pooled MAD 2
    boxes = [(0, 1, 0, 1, 0, 2), (0, 1, 0, 1, 2, 4)]
    assert detection.box_stats(vol, boxes)[:, 2].tolist() == [0.0, 0.0]
    assert detection.box_stats(vol, boxes, pooled=True)[0].tolist() == [4.0, 2.0, 2.0, 4.0]


def test_exact_line_and_its_crossing():
    amounts = np.array([5.0, 10.0, 25.0, 50.0])
    values = 0.02 + 0.4 * amounts
    a, s = detection.linear_fit(amounts, values)
    assert math.isclose(a, 0.02, abs_tol=1e-12) and math.isclose(s, 0.4, rel_tol=1e-12)
    limit, _, _ = detection.detection_limit(amounts, values, noise=0.1)
    assert math.isclose(limit, (0.3 - 0.02) / 0.4, rel_tol=1e-12)


def test_least_squares_of_scattered_points_by_hand():
    # points (0, 1), (1, 2), (2, 2): slope 1/2, intercept 7/6 (normal equations)
    a, s = detection.linear_fit([0.0, 1.0, 2.0], [1.0, 2.0, 2.0])
    assert math.isclose(s, 0.5, rel_tol=1e-12) and math.isclose(a, 7.0 / 6.0, rel_tol=1e-12)
    assert math.isnan(detection.detection_limit([0.0, 1.0], [1.0, 1.0], 0.1)[0])  # flat: no crossing


def test_sensitivity_series_masses_and_boxes():
    amounts = [5.0, 10.0, 25.0, 50.0]
    vol, sboxes, vboxes = sensitivity_series(64, 32, amounts, seed=2)
    assert len(sboxes) == 4 and len(vboxes) == 5
    # the blobs integrate to their amounts (a sampled Gaussian of sigma 1.2 sums to its
    # integral within exp(-2 pi^2 sigma^2)); each sample's box (half-width 3 sigma + 1,
    # over 4 sigma per axis) holds its own amount but for tails below 1e-3
    assert math.isclose(vol.astype(np.float64).sum(), sum(amounts), rel_tol=1e-6)
    for amt, b in zip(amounts, sboxes):
        z0, z1, y0, y1, x0, x1 = b
        assert math.isclose(vol[z0:z1, y0:y1, x0:x1].astype(np.float64).sum(), amt, rel_tol=1e-3)
    peak = float(vol.max())
    for b in vboxes:  # voids are away from the samples: at most their far Gaussian tails
        assert detection.box_stats(vol, [b])[0, 3] < 1e-5 * peak
