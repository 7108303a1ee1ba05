"""Arithmetic atoms on the GPU (smc_set_atom_expression): the FP64 path
reproduces the oracle trajectory by trajectory through the model-specialized
and the generic kernel (the same FP64 operations in the same order), the
mixed path and the exact solver agree with the CME solution of the paper's
example formula, and malformed programs are rejected."""
import math

import numpy as np
import pytest

import workloads
from tests import _cme

pytestmark = pytest.mark.gpu
SP = ['X1', 'X2', 'X3']


@pytest.fixture(scope='module')
def smc():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no GPU')
    import paper_0912_2551_gb300 as smc
    return smc


def _quotient_model():
    """Division, powers and a multi-species left side on the same network:
    (X1^2 + X3 < 3 X2 / (1 + X3)) U[0,15] (X2 - X1 >= 12)."""
    m, _ = workloads.sqrt_race()
    left = workloads.expr_atom(SP, [('x', 'X1'), ('pow', 2), ('x', 'X3'), ('+',)], '<',
                               [('c', 3.0), ('x', 'X2'), ('*',), ('c', 1.0), ('x', 'X3'), ('+',), ('/',)])
    right = workloads.expr_atom(SP, [('x', 'X2'), ('x', 'X1'), ('-',)], '>=', [('c', 12.0)])
    return m, workloads.Property([left, right], ('U', 0.0, 15.0, ('atom', 0), ('atom', 1)))


MODELS = {'sqrt_race': workloads.sqrt_race, 'quotient': _quotient_model}


@pytest.mark.parametrize('jit', [1, 0])
@pytest.mark.parametrize('name', sorted(MODELS))
def test_fp64_matches_oracle_per_trajectory(smc, orc, name, jit):
    import torch
    m, p = MODELS[name]()
    n = 6000
    with smc.Context(0) as ctx:
        ctx.set_option('jit', jit)
        ctx.load_model(m)
        ctx.load_property(p)
        g = ctx.simulate('plain', seed=5, n_traj=n, outputs=('verdict', 'status', 'events', 't_final'))
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in g.items()}
        assert all(s['specialized'] == bool(jit) for s in ctx.launch_shapes('plain'))
    r = orc.run(m, p, seed=5, n_traj=n)
    assert 0.05 < r['verdict'].mean() < 0.95
    assert (g['verdict'][0] == r['verdict']).mean() >= 0.9999
    assert (g['events'][0].astype(np.uint64) == r['events']).mean() >= 0.9999
    assert (g['status'][0] == r['status']).all()


def test_mixed_and_exact_solver_against_cme(smc):
    m, p = workloads.sqrt_race()
    exact = _cme.until_probability(m, lambda x: x[0] < math.sqrt(x[1]), lambda x: x[1] >= 10 + x[2],
                                   p.formula[2], cap=20)
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        ex = ctx.cme_reach(cap=20)
        assert abs(ex['p'] - exact) < 1e-9, (ex, exact)
        r = ctx.estimate(0.9999, 0.005, seed=9, precision='mixed', sampling='iterative')[0]
        assert r['lo'] <= exact <= r['hi'], (r, exact)


def test_malformed_programs_are_rejected(smc):
    from paper_0912_2551_gb300 import _native as N
    m, p = workloads.sqrt_race()
    bad = [([('+',)], [('c', 1.0)]),                          # operator without operands
           ([('x', 0), ('x', 1)], [('c', 1.0)]),              # two values left
           ([('x', 5)], [('c', 1.0)]),                        # species out of range
           ([('x', 0), ('pow', 17)], [('c', 1.0)]),           # power out of range
           ([('c', math.inf)], [('c', 1.0)]),                 # constant not finite
           ([('c', 1.0)] * 9 + [('+',)] * 8, [('c', 1.0)])]   # deeper than 8
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        for lhs, rhs in bad:
            with pytest.raises(smc.SmcError) as e:
                ctx.set_atom_expression(0, '<', lhs, rhs)
            assert e.value.code == N.SMC_E_INVALID_ARG, lhs
        with pytest.raises(smc.SmcError) as e:
            ctx.monitor_replay([(np.zeros((1, 3)), np.zeros(1), 1.0, True)], 3)
        assert e.value.code == N.SMC_E_UNSUPPORTED
