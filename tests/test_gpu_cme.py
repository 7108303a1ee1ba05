"""Exact time-bounded reachability by uniformisation on the GPU
(smc_cme_reach): against SciPy's matrix exponential of the same chain
(tests/_cme.py), against closed forms, with truncation reported, and --
the comparison of Sec. 5 / Fig. 4 -- against the statistical estimate."""
import math

import numpy as np
import pytest
from scipy import stats

import workloads
from tests import _cme

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def smc():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no GPU')
    import paper_0912_2551_gb300 as smc
    return smc


def _exact(smc, m, p, **kw):
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        return ctx.cme_reach(**kw)


def test_immigration_death_against_expm_and_the_known_value(smc):
    m, p = workloads.immigration_death()
    r = _exact(smc, m, p, cap=1000)
    ref = _cme.eventually_probability(m, lambda x: x[0] >= 130, 100.0)
    assert abs(r['p'] - ref) < 1e-9, (r, ref)
    assert abs(r['p'] - 0.0912186) < 5e-8
    assert r['n_states'] == 131 and r['truncated'] == 0.0 and r['poisson_tail'] < 1e-12


@pytest.mark.parametrize('name', ['mm_degradation', 'autorepressor'])
def test_rate_law_models_against_expm(smc, name):
    m, p = getattr(workloads, name)()
    a = p.atoms[0]
    goal = (lambda x: x[0] <= a.bound) if a.op == '<=' else (lambda x: x[0] >= a.bound)
    r = _exact(smc, m, p, cap=300)
    ref = _cme.eventually_probability(m, goal, p.formula[2], cap=300)
    assert abs(r['p'] - ref) < 1e-9, (r, ref)


def test_always_is_the_complement_and_matches_the_binomial(smc):
    # pure decay A -> 0 (k A) from 1000: A is non-increasing, so
    # G[0,1](A >= 360) holds iff A(1) >= 360, and A(1) ~ Binomial(1000, e^-1)
    m, _ = workloads.pure_decay(1000, 1.0, 1.0)
    p = workloads.Property([workloads.atom(['A'], 'A', '>=', 360)], ('G', 0.0, 1.0, ('atom', 0)))
    r = _exact(smc, m, p, cap=2000)
    ref = stats.binom.sf(359, 1000, math.exp(-1.0))
    assert abs(r['p'] - ref) < 1e-9, (r, ref)


def test_until_with_a_left_operand(smc):
    m, _ = workloads.dimerisation()
    sp = m.species
    p = workloads.Property([workloads.atom(sp, 'A', '<=', 100), workloads.atom(sp, 'B', '>=', 25)],
                           ('U', 0.0, 20.0, ('atom', 0), ('atom', 1)))
    r = _exact(smc, m, p, cap=400)
    ref = _cme.until_probability(m, lambda x: x[0] <= 100, lambda x: x[1] >= 25, 20.0, cap=400)
    assert 0.05 < ref < 0.95
    assert abs(r['p'] - ref) < 1e-9, (r, ref)


def test_truncation_is_reported_and_bounds_the_error(smc):
    m, p = workloads.immigration_death()
    p2 = workloads.Property([workloads.atom(['A'], 'A', '>=', 130)], ('F', 0.0, 100.0, ('atom', 0)))
    exact = _exact(smc, m, p2, cap=1000)['p']
    # goal beyond the cap: every path to it crosses a capped state
    r = _exact(smc, m, p2, cap=120)
    assert r['truncated'] > 0.0 and r['p'] <= exact <= r['p'] + r['truncated'] + 1e-12, (r, exact)


def test_unsupported_shapes_and_sizes(smc):
    from paper_0912_2551_gb300 import _native as N
    m, p = workloads.mapk_cascade(1, seed=5)  # nested F: not time-bounded reachability
    with pytest.raises(smc.SmcError) as e:
        _exact(smc, m, p)
    assert e.value.code == N.SMC_E_UNSUPPORTED
    m, p = workloads.immigration_death()
    with pytest.raises(smc.SmcError) as e:
        _exact(smc, m, p, cap=1000, max_states=50)
    assert e.value.code == N.SMC_E_UNSUPPORTED


@pytest.mark.parametrize('name', ['immigration_death', 'autorepressor', 'mm_degradation'])
def test_statistical_estimate_covers_the_exact_value(smc, name):
    # Sec. 5 / Fig. 4: the iterative Wilson estimate against the numerical
    # solution of the same chain, FP64 and mixed paths
    m, p = getattr(workloads, name)()
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        exact = ctx.cme_reach(cap=1000)['p']
        for prec in ('plain', 'mixed'):
            r = ctx.estimate(0.9999, 0.005, seed=21, precision=prec, sampling='iterative')[0]
            assert r['lo'] <= exact <= r['hi'], (name, prec, r, exact)
