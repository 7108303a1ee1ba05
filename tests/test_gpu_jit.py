"""Model-specialized kernels (SMC_OPT_JIT): the run-time compiled kernel of a
network structure must reproduce the generic kernel bit for bit -- same
random numbers, same arithmetic in the same order -- on the FP64 path, and on
the mixed path for small networks (S, R <= 8, where both recompute every
propensity per event): per-trajectory verdicts, statuses, event counts,
final clocks and states, snapshots, and the device-side counts and Wilson
interval.  For larger networks the generic mixed kernel updates a_0
incrementally in FP32 (renormalised in FP64 every 2^k events) while the
specialized one recomputes it per event, so their FP32 roundings differ and
trajectories may part at a selection boundary: there the comparison is
statistical.  The FP64 path's agreement with the oracle is covered by the
parity tests, which run through the specialized kernel by default."""
import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def smc():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no GPU')
    import paper_0912_2551_gb300 as smc
    return smc


def _nested_lv():
    """Lotka-Volterra with a nested monitor (candidate clocks in use):
    (X < 3000) U[0,10] (Y >= 1500 & F[0,0.5] Y < 1000)."""
    m, _ = workloads.lotka_volterra(1)
    sp = m.species
    p = workloads.Property([workloads.atom(sp, 'X', '<', 3000), workloads.atom(sp, 'Y', '>=', 1500),
                            workloads.atom(sp, 'Y', '<', 1000)],
                           ('U', 0.0, 10.0, ('atom', 0), ('and', ('atom', 1), ('F', 0.0, 0.5, ('atom', 2)))))
    return m, p


def _weighted_atom():
    """Dimerisation watched through a multi-term atom A + 2B (conserved up to
    immigration) with a lower window bound: F[2,20](A + 2B >= 160)."""
    m, _ = workloads.dimerisation(1)
    sp = m.species
    p = workloads.Property([workloads.atom(sp, {'A': 1, 'B': 2}, '>=', 160)], ('F', 2.0, 20.0, ('atom', 0)))
    return m, p


MODELS = {
    'lotka_volterra': lambda: workloads.lotka_volterra(1),
    'lv_family': lambda: workloads.lotka_volterra_family(6, seed=4),
    'immigration_death': lambda: workloads.immigration_death(1),
    'dimerisation': lambda: workloads.dimerisation(1),
    'pure_decay': lambda: workloads.pure_decay(),
    'nested_lv': _nested_lv,
    'weighted_atom': _weighted_atom,
    'mm_degradation': lambda: workloads.mm_degradation(),
    'autorepressor': lambda: workloads.autorepressor(),
    # medium networks: net changes from the shared-memory table, rates per warp
    'cascade_literal': lambda: workloads.mapk_cascade(2, seed=5),
    'cascade_variant': lambda: workloads.mapk_cascade(2, seed=5, variant=True),
    'factor_chain': lambda: workloads.factor_chain(),
    'sqrt_race': lambda: workloads.sqrt_race(),  # arithmetic atoms (the paper's example formula)
    'next': lambda: (workloads.immigration_death()[0],  # the Next operator with F
                     workloads.Property([workloads.atom(['A'], 'A', '>=', 1), workloads.atom(['A'], 'A', '>=', 130)],
                                        ('and', ('X', 0.05, 0.2, ('atom', 0)), ('F', 0.0, 100.0, ('atom', 1))))),
}
SIZES = {'lotka_volterra': 1500, 'cascade_literal': 512, 'cascade_variant': 256}
MEDIUM = {'cascade_literal', 'cascade_variant', 'factor_chain'}
OUTPUTS = ('verdict', 'status', 'events', 't_final', 'x_final')


def _run(smc, model, prop, jit, precision, n, t_max=math.inf):
    import torch
    with smc.Context(0) as ctx:
        ctx.set_option('jit', jit)
        ctx.load_model(model)
        ctx.load_property(prop, t_max=t_max)
        out = ctx.simulate(precision, seed=17, traj_begin=1000, n_traj=n, confidence=0.95, outputs=OUTPUTS)
        torch.cuda.synchronize()
        shapes = ctx.launch_shapes(precision)
        return {k: v.cpu().numpy() for k, v in out.items()}, shapes


@pytest.mark.parametrize('precision', ['plain', 'mixed'])
@pytest.mark.parametrize('name', sorted(MODELS))
def test_specialized_kernel_reproduces_generic(smc, name, precision):
    model, prop = MODELS[name]()
    n = SIZES.get(name, 3000)
    spec, s1 = _run(smc, model, prop, 1, precision, n)
    gen, s0 = _run(smc, model, prop, 0, precision, n)
    assert all(s['specialized'] for s in s1), s1
    assert not any(s['specialized'] for s in s0)
    assert spec['counts'][:, 1].sum() + spec['counts'][:, 3].sum() == model.n_inst * n
    if precision == 'mixed' and name in MEDIUM:
        assert (spec['verdict'] == gen['verdict']).mean() >= 0.95
        p1, p2 = spec['verdict'].mean(), gen['verdict'].mean()
        pm = 0.5 * (p1 + p2)
        assert abs(p1 - p2) <= 4 * math.sqrt(max(pm * (1 - pm), 1e-4) / spec['verdict'].size) + 1e-3
        e1, e2 = spec['events'].astype(float).mean(), gen['events'].astype(float).mean()
        assert abs(e1 - e2) <= 0.02 * e2, (e1, e2)
        assert (spec['status'] == gen['status']).mean() >= 0.95
        return
    for k in OUTPUTS + ('counts',):
        assert np.array_equal(spec[k], gen[k]), (k, np.argwhere(spec[k] != gen[k])[:5])
    assert np.array_equal(spec['wilson'], gen['wilson'])


@pytest.mark.parametrize('name', ['lotka_volterra', 'immigration_death', 'nested_lv', 'next'])
def test_cooperative_tail_reproduces_generic(smc, name):
    # a handful of trajectories: warps run out of work at once, and a warp's
    # last trajectory is advanced by its 32 lanes speculating over the
    # reactions (FP64 path): the trajectories must be the sequential ones
    model, prop = MODELS[name]()
    for n in (1, 3, 37):
        spec, _ = _run(smc, model, prop, 1, 'plain', n)
        gen, _ = _run(smc, model, prop, 0, 'plain', n)
        for k in OUTPUTS + ('counts',):
            assert np.array_equal(spec[k], gen[k]), (name, n, k, np.argwhere(spec[k] != gen[k])[:5])


@pytest.mark.parametrize('precision', ['plain', 'mixed'])
def test_specialized_snapshots_reproduce_generic(smc, precision):
    import torch
    model, prop = workloads.lotka_volterra_family(4, seed=9)
    res = []
    for jit in (1, 0):
        with smc.Context(0) as ctx:
            ctx.set_option('jit', jit)
            ctx.load_model(model)
            ctx.load_property(prop)
            for stop in (False, True):
                o = ctx.simulate_snapshot(precision, seed=3, traj_begin=0, n_traj=2048, t_snap=0.6, stop=stop)
                torch.cuda.synchronize()
                res.append({k: v.cpu().numpy() for k, v in o.items()})
    for a, b in zip(res[:2], res[2:]):
        for k in a:
            assert np.array_equal(a[k], b[k]), k
    assert (res[0]['snap'] == 0).any() and (res[0]['snap'] == 1).any()


def test_ineligible_models_run_generic(smc):
    import torch
    # more than 32 reactions: one network of the random batch, loaded alone
    b = workloads.random_networks(64, seed=3)
    i = next(k for k, mm in enumerate(b.models) if mm.n_reactions > 32)
    m, p = b.models[i], b.properties[i]
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        ctx.simulate('mixed', seed=1, n_traj=64, outputs=())
        torch.cuda.synchronize()
        assert not any(s['specialized'] for s in ctx.launch_shapes('mixed'))
    # heterogeneous batch
    b = workloads.random_networks(16, seed=3)
    with smc.Context(0) as ctx:
        ctx.load_batch(b)
        ctx.load_property(b.properties)
        ctx.simulate('mixed', seed=1, n_traj=64, outputs=())
        torch.cuda.synchronize()
        assert not any(s['specialized'] for s in ctx.launch_shapes('mixed'))


def test_specialized_estimate_matches_generic(smc):
    """The graph-captured Fig. 2 loop through the specialized kernel."""
    model, prop = workloads.immigration_death(1)
    res = []
    for jit in (1, 0):
        with smc.Context(0) as ctx:
            ctx.set_option('jit', jit)
            ctx.load_model(model)
            ctx.load_property(prop)
            r = ctx.estimate(0.99, 0.01, seed=5, precision='plain', sampling='iterative')[0]
            res.append((r['yes'], r['n'], r['events'], r['iterations'], r['p_hat'], r['lo'], r['hi']))
    assert res[0] == res[1]
