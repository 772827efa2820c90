"""Regularised reconstruction by accelerated projected gradient descent (oracle).

Sec. 3.3, Eq. (25): minimise ||A x - b||^2 + lambda ||T x||^2.
Eq. (26): y^{k+1} = x^k + (k-1)/(k+2) (x^k - x^{k-1}),
          x^{k+1} = y^{k+1} - tau [A^*(A y^{k+1} - b) + lambda T^*T y^{k+1}],
tau = (||A^*A||_2 + lambda ||T^*T||_2)^{-1}; the iterate is projected to
real, non-negative values inside every iteration.

Readings used here:
* x^1 = x^0 = x0 (zero by default) and k = 1..K, so the first momentum
  coefficient is 0; the projection max(0, .) is applied to each update.
* ||A^*A||_2 comes from power iteration on A^T A (start vector from the
  counter-based SplitMix64 generator below, Rayleigh quotient of the last
  iterate); ||T^*T||_2 from its closed form.
* lambda defaults to 1e-3 ||A^T A|| / ||T^T T|| (the paper gives no value).
* Optional early stop when the residual norm changes by at most `stop_rel`
  (relative) between iterations.
"""

import numpy as np

from . import regularizer

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64_uniform(seed, n):
    """u_i in [-1, 1) from SplitMix64 (Steele, Lea, Flood 2014) at counter i.

    z = seed + (i + 1) * 0x9E3779B97F4A7C15;  z = (z ^ z>>30) * 0xBF58476D1CE4E5B9;
    z = (z ^ z>>27) * 0x94D049BB133111EB;  z ^= z>>31;  u = (z >> 11) * 2^-52 - 1.
    """
    with np.errstate(over="ignore"):
        i = np.arange(1, n + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * 2.0**-52 - 1.0


def power_norm(apply_ata, shape, n_iter=50, seed=1234):
    """||A^T A||_2 by power iteration; returns the last Rayleigh quotient."""
    v = splitmix64_uniform(seed, int(np.prod(shape))).reshape(shape)
    v /= np.linalg.norm(v)
    mu = 0.0
    for _ in range(n_iter):
        w = apply_ata(v)
        mu = float(np.vdot(v, w).real)
        nw = np.linalg.norm(w)
        if nw == 0.0:
            return 0.0
        v = w / nw
    return mu


def default_lambda(ata_norm, shape):
    return 1e-3 * ata_norm / regularizer.ttt_norm(shape)


def step_size(ata_norm, lam, shape):
    return 1.0 / (ata_norm + lam * regularizer.ttt_norm(shape))


def solve(apply_a, apply_at, b, shape, tau, lam, iters, x0=None, nonneg=True,
          stop_rel=0.0, apply_ttt=regularizer.ttt):
    """Run Eq. (26); returns (x, residual_history)."""
    x = np.zeros(shape) if x0 is None else np.array(x0, dtype=np.float64)
    x_prev = x.copy()
    hist = []
    for k in range(1, iters + 1):
        beta = (k - 1.0) / (k + 2.0)
        y = x + beta * (x - x_prev)
        r = apply_a(y) - b
        hist.append(float(np.sqrt(np.sum(np.abs(r) ** 2))))
        g = apply_at(r) + lam * apply_ttt(y)
        x_new = y - tau * g
        if nonneg:
            x_new = np.maximum(x_new, 0.0)
        x_prev, x = x, x_new
        if stop_rel > 0.0 and k > 1 and abs(hist[-2] - hist[-1]) <= stop_rel * hist[-2]:
            break
    return x, hist
