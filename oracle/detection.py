"""Detection-limit analysis of a reconstruction (oracle, float64).

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline use this module; the product path never does.

Sec. 4.2 (Fig. 5). Fit a least-squares line to the image value of each sample
against its iron amount. Take the background noise as the mean absolute deviation
(MAD) of void regions. The detection limit is the amount at which the line reaches
three times the noise.

Readings (the paper describes the procedure in words):
  - The image value of a sample is the mean reconstructed value over a box around it
    (an ROI mean, which stays linear in the amount when the reconstruction spreads a
    sample over several voxels).
  - The noise is the mean absolute deviation about their mean of all voxels of the
    void boxes taken together.
  - The fit is ordinary least squares v = a + s * amount over the samples given.
    The limit is (k * noise - a) / s with k = 3, undefined unless s > 0.
"""

import numpy as np


def box_voxels(vol, box):
    z0, z1, y0, y1, x0, x1 = box
    return np.asarray(vol, dtype=np.float64)[z0:z1, y0:y1, x0:x1].reshape(-1)


def box_stats(vol, boxes, pooled=False):
    """Per box (or for all boxes together): (count, mean, mean absolute deviation, max)."""
    groups = [np.concatenate([box_voxels(vol, b) for b in boxes])] if pooled else [box_voxels(vol, b) for b in boxes]
    out = []
    for v in groups:
        mean = v.mean()
        out.append((v.size, mean, np.abs(v - mean).mean(), v.max()))
    return np.array(out, dtype=np.float64)


def linear_fit(amounts, values):
    """(intercept a, slope s) of the least-squares line values ~ a + s * amounts."""
    A = np.stack([np.ones(len(amounts)), np.asarray(amounts, dtype=np.float64)], axis=1)
    coef, *_ = np.linalg.lstsq(A, np.asarray(values, dtype=np.float64), rcond=None)
    return float(coef[0]), float(coef[1])


def detection_limit(amounts, values, noise, k=3.0):
    """Amount at which the fitted line reaches k * noise (NaN if the slope is not positive)."""
    a, s = linear_fit(amounts, values)
    return (k * noise - a) / s if s > 0 else float("nan"), s, a


def analyse(vol, sample_boxes, amounts, void_boxes, k=3.0):
    """Sample values, noise and the detection limit of one reconstruction."""
    values = box_stats(vol, sample_boxes)[:, 1]
    noise = box_stats(vol, void_boxes, pooled=True)[0, 2]
    limit, s, a = detection_limit(amounts, values, noise, k)
    return dict(values=values, noise=noise, limit=limit, slope=s, intercept=a)
