"""The Next operator X[a,b] on the GPU: a closed form, per-trajectory parity
with the oracle (FP64, both kernels) inside boolean combinations with other
temporal operators, and nested in a temporal operand or over one (the trace
monitor's shapes)."""
import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu
A = lambda k: ('atom', k)  # noqa: E731


@pytest.fixture(scope='module')
def smc():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no GPU')
    import paper_0912_2551_gb300 as smc
    return smc


def _id(formula):
    m, _ = workloads.immigration_death()
    atoms = [workloads.atom(['A'], 'A', '>=', 1), workloads.atom(['A'], 'A', '>=', 130)]
    return m, workloads.Property(atoms, formula)


FORMULAS = {
    'next': ('X', 0.05, 0.2, A(0)),
    'next_and_eventually': ('and', ('X', 0.05, 0.2, A(0)), ('F', 0.0, 100.0, A(1))),
    'not_next_or': ('or', ('not', ('X', 0.0, 0.1, A(0))), ('F', 0.0, 100.0, A(1))),
}


def test_next_closed_form(smc):
    m, p = _id(FORMULAS['next'])
    exact = math.exp(-0.5) - math.exp(-2.0)
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        for prec in ('plain', 'mixed'):
            r = ctx.estimate(0.9999, 0.003, seed=3, precision=prec, sampling='iterative')[0]
            assert r['lo'] <= exact <= r['hi'], (prec, r, exact)


@pytest.mark.parametrize('jit', [1, 0])
@pytest.mark.parametrize('name', sorted(FORMULAS))
def test_fp64_matches_oracle_per_trajectory(smc, orc, name, jit):
    import torch
    m, p = _id(FORMULAS[name])
    n = 4000
    with smc.Context(0) as ctx:
        ctx.set_option('jit', jit)
        ctx.load_model(m)
        ctx.load_property(p)
        g = ctx.simulate('plain', seed=8, n_traj=n, outputs=('verdict', 'status', 'events', 't_final'))
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in g.items()}
    r = orc.run(m, p, seed=8, n_traj=n)
    assert (g['verdict'][0] == r['verdict']).mean() >= 0.9999
    assert (g['events'][0].astype(np.uint64) == r['events']).mean() >= 0.9999


def test_next_nested_shapes_run_on_the_trace_monitor(smc, orc):
    # X inside a temporal operand, and a temporal operator under X: beyond
    # the monitor's units, decided by the trace monitor, per trajectory as
    # the oracle decides them
    import torch
    for f in [('F', 0.0, 10.0, ('X', 0.0, 1.0, A(0))),      # X inside a right operand
              ('X', 0.0, 1.0, ('F', 0.0, 1.0, A(0)))]:      # temporal operand
        m, p = _id(f)
        n = 2000
        with smc.Context(0) as ctx:
            ctx.load_model(m)
            ctx.load_property(p)
            assert ctx.monitor_kind == 'trace', f
            g = ctx.simulate('plain', seed=8, n_traj=n, outputs=('verdict', 'status', 'events', 't_final'))
            torch.cuda.synchronize()
            g = {k: v.cpu().numpy() for k, v in g.items()}
        r = orc.run(m, p, seed=8, n_traj=n)
        assert (g['verdict'][0] == r['verdict']).all(), f
        assert (g['events'][0].astype(np.uint64) == r['events']).all(), f
