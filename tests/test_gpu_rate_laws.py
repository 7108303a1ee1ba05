"""Rate-law factors (smc_load_rate_factors): propensities c h(x) times
rational factors (a0 + a1 x^n) / (b0 + b1 x^n) of single species.  The FP64
path must reproduce the oracle trajectory by trajectory -- the same
operations in the same order -- through the model-specialized kernel and
through the generic one (for the 10-species chain, with dependency-graph
updates that include a factor's species); the mixed path must cover the exact value
(CME) within its interval; bad factors are rejected."""
import ctypes
import math

import numpy as np
import pytest

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


def _run(smc, m, p, precision, n, seed, jit=1, outputs=('verdict', 'status', 'events', 't_final')):
    import torch
    with smc.Context(0) as ctx:
        ctx.set_option('jit', jit)
        ctx.load_model(m)
        ctx.load_property(p)
        out = ctx.simulate(precision, seed=seed, n_traj=n, outputs=outputs)
        torch.cuda.synchronize()
        spec = all(s['specialized'] for s in ctx.launch_shapes(precision))
        return {k: v.cpu().numpy() for k, v in out.items()}, spec


@pytest.mark.parametrize('jit', [1, 0])
@pytest.mark.parametrize('name', ['mm_degradation', 'autorepressor', 'factor_chain'])
def test_fp64_matches_oracle_per_trajectory(smc, orc, name, jit):
    m, p = getattr(workloads, name)()
    n = 4000
    g, spec = _run(smc, m, p, 'plain', n, seed=13, jit=jit)
    assert spec == (jit == 1)
    r = orc.run(m, p, seed=13, n_traj=n)
    v = g['verdict'][0]
    assert (v == r['verdict']).mean() >= 0.9999
    ev = g['events'][0].astype(np.uint64) == r['events']
    assert ev.mean() >= 0.9999
    same = ev & (v == r['verdict'])
    rel = np.abs(g['t_final'][0][same] - r['t_final'][same]) / np.maximum(np.abs(r['t_final'][same]), 1e-300)
    assert (rel <= 1e-12).mean() >= 0.9999
    assert (g['status'][0] == r['status']).all()


@pytest.mark.parametrize('name', ['mm_degradation', 'autorepressor'])
def test_mixed_covers_exact_value(smc, name):
    m, p = getattr(workloads, name)()
    atom = p.atoms[0]
    goal = (lambda x: x[0] <= atom.bound) if atom.op == '<=' else (lambda x: x[0] >= atom.bound)
    exact = _cme.eventually_probability(m, goal, p.formula[2], cap=300)
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        res = ctx.estimate(0.9999, 0.005, seed=3, precision='mixed', sampling='iterative')[0]
    assert res['lo'] <= exact <= res['hi'], (res, exact)


def test_invalid_factors_are_rejected(smc):
    from paper_0912_2551_gb300 import _native as N
    m, p = workloads.autorepressor()
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        bad = [[(0, 0, 0, 1.0, 0.0, 1.0, 1.0)],           # power 0
               [(0, 0, 5, 1.0, 0.0, 1.0, 1.0)],           # power > 4
               [(0, 0, 1, 1.0, 0.0, 0.0, 1.0)],           # b0 = 0
               [(0, 0, 1, -1.0, 0.0, 1.0, 1.0)],          # a0 < 0
               [(2, 0, 1, 1.0, 0.0, 1.0, 1.0)],           # reaction out of range
               [(0, 1, 1, 1.0, 0.0, 1.0, 1.0)],           # species out of range
               [(0, 0, 1, 1.0, 0.0, 1.0, 1.0)] * 3,       # three factors on one reaction
               [(0, 0, 1, math.inf, 0.0, 1.0, 1.0)]]      # not finite
        for f in bad:
            with pytest.raises(smc.SmcError) as e:
                ctx.load_rate_factors(f)
            assert e.value.code == N.SMC_E_INVALID_ARG, f
    b = workloads.random_networks(4, seed=3)
    with smc.Context(0) as ctx:
        ctx.load_batch(b)
        with pytest.raises(smc.SmcError) as e:
            ctx.load_rate_factors([(0, 0, 1, 1.0, 0.0, 1.0, 1.0)])
        assert e.value.code == N.SMC_E_UNSUPPORTED
