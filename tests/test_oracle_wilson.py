"""Pins of the oracle's Wilson interval (Eq. 4), sample size (Eq. 5) and the
iterative procedure (Fig. 2) against the values the paper prints, closed
forms, and a library normal quantile."""
import math
import os

import numpy as np
import pytest
from scipy import special, stats

from oracle import wilson

GOLD = os.path.join(os.path.dirname(__file__), 'golden', 'table1_wilson.txt')


def _table1():
    rows = []
    for line in open(GOLD):
        if line.strip() and not line.startswith('#'):
            r, yes, n, p, lo, hi = line.split()
            rows.append((int(r), int(yes), int(n), p, lo, hi))
    return rows


def test_normal_quantile_against_scipy(orc):
    for p in [0.5, 0.9, 0.95, 0.975, 0.995, 0.99995, 1e-6, 0.3]:
        z = orc.normal_quantile(p)
        assert abs(z - special.ndtri(p)) <= 2e-15 * max(1.0, abs(z)), p
    assert abs(wilson.z_value(0.95) - 1.959963984540054) < 1e-15
    assert abs(wilson.z_value(0.99) - 2.5758293035489004) < 1e-15


@pytest.mark.parametrize('row', _table1(), ids=lambda r: f'row{r[0]}')
def test_table1_intervals(row):
    _, yes, n, p_print, lo_print, hi_print = row
    ulp = lambda s: 10.0 ** -len(s.split('.')[1])
    p, lo, hi = wilson.wilson_interval(yes, n, 0.99)
    assert abs(p - float(p_print)) < ulp(p_print)
    assert abs(lo - float(lo_print)) < ulp(lo_print)
    assert abs(hi - float(hi_print)) < ulp(hi_print)


def test_table1_conservative_and_first_iterative_sizes():
    # Table 1: conservative N = 2648 at 99%, half-width 0.025 (Eq. 5, p = 0.5);
    # Fig. 2's first batch uses p = 1.
    assert wilson.wilson_sample(0.5, 0.025, 0.99) == 2648
    assert wilson.wilson_sample(1.0, 0.025, 0.99) == 127
    # closed form at p = 1: z^2 (1/(2 eps) - 1)
    z = wilson.z_value(0.99)
    assert abs(wilson.wilson_sample_real(1.0, 0.025, 0.99) - z * z * (1 / 0.05 - 1)) < 1e-9
    # closed form at p = 1/2: z^2 (1/4 - 2e^2 + sqrt(1/16)) / (2 e^2) = z^2 (1 - 4 e^2)/(4 e^2)
    e = 0.025
    assert abs(wilson.wilson_sample_real(0.5, e, 0.99) - z * z * (1 - 4 * e * e) / (4 * e * e)) < 1e-9


def test_zero_and_full_counts():
    for n in [1, 7, 127, 10000]:
        z = wilson.z_value(0.95)
        p, lo, hi = wilson.wilson_interval(0, n, 0.95)
        assert p == 0 and lo == 0.0
        assert abs(hi - z * z / (n + z * z)) < 1e-15
        p, lo, hi = wilson.wilson_interval(n, n, 0.95)
        assert hi == 1.0 and abs(lo - n / (n + z * z)) < 1e-15


def test_eq5_inverts_eq4_half_width():
    # At N = Wilson_sample(p, eps) (real-valued) the Eq. 4 half-width at
    # p_hat = p equals eps (Eq. 5 is Eq. 4 solved for n).
    for p in [0.01, 0.1, 0.3, 0.5, 0.8]:
        for eps in [0.005, 0.025]:
            N = wilson.wilson_sample_real(p, eps, 0.99)
            z = wilson.z_value(0.99)
            half = z * math.sqrt(p * (1 - p) / N + z * z / (4 * N * N)) / (1 + z * z / N)
            assert abs(half - eps) < 1e-12


def _bernoulli_runner(p, rng):
    def run(begin, count):
        y = int((rng.random(count) < p).sum())
        return y, count
    return run


def test_fig2_reduction_up_to_88_percent():
    # Sec. 3.3.2: at p in {0, 1} the iterative method needs 88% fewer samples
    # than the conservative 2648 (2 eps = 0.05, 99%).
    rng = np.random.default_rng(0)
    for p in (0.0, 1.0):
        r = wilson.iterative(_bernoulli_runner(p, rng), 0.025, 0.99)
        assert r['n_tot'] == 304
        assert r['sizes'] == [127, 177]
        red = 1 - r['n_tot'] / 2648
        assert 0.88 <= red < 0.89
    r = wilson.iterative(_bernoulli_runner(0.3, rng), 0.025, 0.99, start_p=0.5)
    assert r['n_tot'] == 2648 and r['iterations'] == 1


@pytest.mark.parametrize('p', [0.02, 0.2, 0.5, 0.9])
def test_fig2_coverage(p):
    # The final interval covers p in at least (1 - alpha) - 2.5% of 600 runs.
    rng = np.random.default_rng(int(p * 1000))
    cover = 0
    reps = 600
    for _ in range(reps):
        r = wilson.iterative(_bernoulli_runner(p, rng), 0.025, 0.95)
        cover += r['lo'] <= p <= r['hi']
        assert r['hi'] - r['lo'] <= 2 * 0.025 + 1e-9 or r['n_tot'] < 2000
    assert cover / reps >= 0.95 - 0.025
