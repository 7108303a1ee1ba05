"""The exact CME helper the oracle's tests rely on (tests/_cme.py) against
closed forms: pure decay (first passage below k by T <=> A(T) <= k,
A(T) ~ Binomial(A0, e^{-cT})), immigration (A(T) ~ Poisson(cT)), linear
birth-death extinction by T (Kendall 1948), and an until formula whose
left operand fails at once."""
import math

import numpy as np
from scipy import stats

import workloads
from tests import _cme


def test_pure_decay_binomial():
    model, _ = workloads.pure_decay(A0=20, k=0.7, T=1.0)
    for k in (0, 5, 12, 19):
        p = _cme.eventually_probability(model, lambda x, k=k: x[0] <= k, 1.0)
        assert abs(p - stats.binom.cdf(k, 20, math.exp(-0.7))) < 1e-12


def test_immigration_poisson():
    model, _ = workloads.immigration_only(k=3.0, T=2.0)
    for m in (1, 6, 11):
        p = _cme.eventually_probability(model, lambda x, m=m: x[0] >= m, 2.0)
        assert abs(p - stats.poisson.sf(m - 1, 6.0)) < 1e-12


def test_birth_death_extinction_kendall():
    b, d, A0, T = 1.0, 1.3, 3, 2.0
    model, _ = workloads.birth_death_survival(b=b, d=d, A0=A0, T=T)
    p = _cme.eventually_probability(model, lambda x: x[0] == 0, T, cap=160)
    e = math.exp((b - d) * T)
    q = d * (e - 1.0) / (b * e - d)  # one lineage extinct by T
    assert abs(p - q ** A0) < 1e-9


def test_until_with_failing_left_operand():
    model, _ = workloads.immigration_only(k=3.0, T=2.0)
    # (A < 0) U[0,2] (A >= 1): the left operand fails at once, the right
    # does not hold at 0, so the formula is false with probability 1
    assert _cme.until_probability(model, lambda x: x[0] < 0, lambda x: x[0] >= 1, 2.0) == 0.0
    # (A < 4) U[0,2] (A >= 2) = F[0,2](A >= 2) here (counts rise by one)
    p = _cme.until_probability(model, lambda x: x[0] < 4, lambda x: x[0] >= 2, 2.0)
    assert abs(p - stats.poisson.sf(1, 6.0)) < 1e-12
