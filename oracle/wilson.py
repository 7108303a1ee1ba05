"""Wilson score interval (Eq. 4), Wilson sample size (Eq. 5) and the
iterative sample-size procedure (Fig. 2), written out in FP64.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Readings of the paper used here:
  * alpha = 1 - confidence, z = Phi^{-1}(1 - alpha/2) (Sec. 3.3).
  * epsilon is the half-width ("width 2 epsilon", Sec. 3.3.1).
  * The sample size of Eq. 5 is rounded up (ceil): Table 1's conservative
    N = 2648 = ceil(Wilson_sample(0.5, 0.025, 0.99)).
  * In Fig. 2, "pest" is the cumulative frequency yes / N_tot.
  * The interval is clipped to [0, 1]; at p_hat = 0 the lower end is 0 and at
    p_hat = 1 the upper end is 1.
"""
from __future__ import annotations

import math
from typing import Callable, Tuple

from . import normal_quantile


def z_value(confidence: float) -> float:
    alpha = 1.0 - confidence
    return normal_quantile(1.0 - alpha / 2.0)


def wilson_interval(yes: int, n: int, confidence: float) -> Tuple[float, float, float]:
    """Eq. 4: [L, U] = (p + z^2/(2n) -+ z sqrt(p(1-p)/n + z^2/(4n^2))) / (1 + z^2/n).
    Returns (p_hat, L, U)."""
    if n <= 0:
        return (float('nan'), 0.0, 1.0)
    z = z_value(confidence)
    p = yes / n
    z2 = z * z
    centre = p + z2 / (2.0 * n)
    half = z * math.sqrt(p * (1.0 - p) / n + z2 / (4.0 * n * n))
    den = 1.0 + z2 / n
    lo = (centre - half) / den
    hi = (centre + half) / den
    if yes == 0:
        lo = 0.0
    if yes == n:
        hi = 1.0
    return p, max(0.0, lo), min(1.0, hi)


def wilson_sample_real(p: float, eps: float, confidence: float) -> float:
    """Eq. 5: N >= z^2 (p(1-p) - 2 eps^2 + sqrt(p^2 (1-p)^2 + 4 eps^2 (p - 1/2)^2)) / (2 eps^2)."""
    z = z_value(confidence)
    e2 = eps * eps
    q = p * (1.0 - p)
    return z * z * (q - 2.0 * e2 + math.sqrt(q * q + 4.0 * e2 * (p - 0.5) ** 2)) / (2.0 * e2)


def wilson_sample(p: float, eps: float, confidence: float) -> int:
    return int(math.ceil(wilson_sample_real(p, eps, confidence)))


def iterative(run: Callable[[int, int], Tuple[int, int]], eps: float, confidence: float,
              start_p: float = 1.0, max_iter: int = 1000):
    """Fig. 2.  ``run(begin, count)`` performs trajectories begin..begin+count-1
    and returns (yes, n_decided).  ``start_p`` = 1 gives the iterative method,
    0.5 the conservative one (which performs a single batch).

    Returns dict(p_hat, lo, hi, n_tot, yes, iterations, sizes)."""
    n_tot = 0
    yes_tot = 0
    dec_tot = 0
    N = wilson_sample(start_p, eps, confidence)
    sizes = []
    it = 0
    while True:
        it += 1
        y, d = run(n_tot, N)
        sizes.append(N)
        n_tot += N
        yes_tot += y
        dec_tot += d
        p_est = yes_tot / dec_tot if dec_tot else 0.0
        if start_p == 0.5:
            break
        p_prime = p_est + eps if p_est <= 0.5 else p_est - eps
        n_prime = wilson_sample(p_prime, eps, confidence)
        n_new = n_prime - n_tot
        if n_new > 0 and it < max_iter:
            N = n_new
            continue
        break
    p, lo, hi = wilson_interval(yes_tot, dec_tot, confidence)
    return dict(p_hat=p, lo=lo, hi=hi, n_tot=n_tot, yes=yes_tot, decided=dec_tot,
                iterations=it, sizes=sizes)
