"""Formulas nested beyond the monitor's units (Sec. 3.1's grammar: U, F, G
and X in either operand, to any depth), run on the GPU by the trace
monitor (smc_nest.h: each lane records its trajectory, the formula's
verdict and decision point come from the recording).

FP64 path: per trajectory the verdict, status, event count, final state
and clock (to 1e-12 relative) equal the oracle's, whose evaluator
recurses over the whole trace (oracle/smc_oracle.c).  Mixed path: its
estimate falls within the combined intervals of the FP64 one.  The
recording's capacity bound gives status 3 and counts the trajectory as
undecided.  The replay of tiny paths through the same evaluator is
tests/test_gpu_parity.py::test_monitor_replay_matches_oracle (its
formula list includes these shapes)."""
import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

A = lambda k: ('atom', k)


@pytest.fixture(scope='module')
def smc():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no GPU')
    import paper_0912_2551_gb300 as smc
    return smc


@pytest.fixture()
def ctx(smc):
    c = smc.Context(0)
    yield c
    c.close()


def _model(kind, formula):
    if kind == 'id':  # immigration-death: 0 -> A (10), A -> 0 (0.1 A), A0 = 0
        m, _ = workloads.immigration_death()
        sp = ['A']
        atoms = [workloads.atom(sp, 'A', '>=', 100), workloads.atom(sp, 'A', '>=', 120),
                 workloads.atom(sp, 'A', '>=', 10), workloads.atom(sp, 'A', '>=', 80),
                 workloads.atom(sp, 'A', '>=', 75), workloads.atom(sp, 'A', '<=', 150)]
    else:  # Lotka-Volterra, X0 = Y0 = 1000
        m, _ = workloads.lotka_volterra()
        sp = ['X', 'Y']
        atoms = [workloads.atom(sp, {'X': 1, 'Y': -1}, '>', 0), workloads.atom(sp, 'X', '<', 100),
                 workloads.atom(sp, 'Y', '<', 700)]
    return m, workloads.Property(atoms, formula)


CASES = [
    # (name, model, formula, t_max of the pessimistic rule, trajectories)
    ('id_next_inside_F', 'id', ('F', 10.0, 40.0, ('X', 0.0, 0.02, A(0))), math.inf, 4000),
    ('id_F_inside_U_left', 'id', ('U', 0.0, 30.0, ('F', 0.0, 2.0, A(2)), A(1)), math.inf, 4000),
    ('id_depth_4', 'id', ('G', 0.0, 20.0, ('implies', A(3), ('F', 0.0, 3.0, ('G', 0.0, 1.0, A(4))))),
     math.inf, 4000),
    ('id_unbounded_next_inside_U', 'id', ('U', 0.0, math.inf, ('X', 0.0, 1.0, A(5)), A(1)), 50.0, 4000),
    ('id_G_with_lower_bound_inside_F', 'id', ('F', 5.0, 30.0, ('G', 0.5, 2.0, A(0))), math.inf, 4000),
    ('lv_next_inside_U_left', 'lv', ('U', 0.0, 15.0, ('X', 0.0, 0.05, ('not', A(2))), A(1)), math.inf, 2000),
]


def _run(ctx, m, prop, t_max, n, precision, seed):
    import torch
    ctx.load_model(m)
    ctx.load_property(prop, t_max=t_max)
    assert ctx.monitor_kind == 'trace'
    out = ctx.simulate(precision, seed=seed, n_traj=n,
                       outputs=('verdict', 'status', 'events', 't_final', 'x_final'))
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


@pytest.mark.parametrize('case', CASES, ids=[c[0] for c in CASES])
def test_nested_formula_plain_matches_oracle(ctx, orc, case):
    _, kind, formula, t_max, n = case
    m, prop = _model(kind, formula)
    g = _run(ctx, m, prop, t_max, n, 'plain', seed=7)
    r = orc.run(m, prop, seed=7, n_traj=n, t_max=t_max, want_x=True)
    S = m.n_species
    v, st, ev, tf = g['verdict'][0], g['status'][0], g['events'][0].astype(np.uint64), g['t_final'][0]
    xf = g['x_final'][0][:, :S]
    same = (v == r['verdict']) & (st == r['status']) & (ev == r['events']) & np.all(xf == r['x_final'], axis=1)
    rel = np.abs(tf - r['t_final']) / np.maximum(np.abs(r['t_final']), 1e-300)
    same &= rel <= 1e-12
    bad = np.nonzero(~same)[0]
    for k in bad[:10]:
        print(f'trajectory {k}: gpu verdict {v[k]} status {st[k]} events {ev[k]} t {tf[k]!r} x {xf[k].tolist()}; '
              f'oracle {r["verdict"][k]} {r["status"][k]} {r["events"][k]} {r["t_final"][k]!r} '
              f'{r["x_final"][k].tolist()}')
    print(f'{case[0]}: {n - bad.size} of {n} equal, p = {v.mean():.4f}')
    assert bad.size <= n // 1000
    assert (r['status'] == 0).all()  # every trajectory decided within the horizon
    yes, dec = int(g['counts'][0, 0]), int(g['counts'][0, 1])
    assert dec == n and yes == int(v.sum()) and int(g['counts'][0, 2]) == int(ev.astype(np.int64).sum())


@pytest.mark.parametrize('case', [CASES[0], CASES[2], CASES[4]], ids=[CASES[i][0] for i in (0, 2, 4)])
def test_nested_formula_mixed_agrees_with_plain(ctx, case):
    from oracle import wilson
    _, kind, formula, t_max, n = case
    m, prop = _model(kind, formula)
    n *= 4
    gp = _run(ctx, m, prop, t_max, n, 'plain', seed=11)
    gm = _run(ctx, m, prop, t_max, n, 'mixed', seed=11)
    yp, ym = int(gp['verdict'][0].sum()), int(gm['verdict'][0].sum())
    assert int(gm['counts'][0, 1]) == n
    _, lo_p, hi_p = wilson.wilson_interval(yp, n, 0.999)
    _, lo_m, hi_m = wilson.wilson_interval(ym, n, 0.999)
    assert abs(ym - yp) / n <= (hi_p - lo_p) / 2 + (hi_m - lo_m) / 2
    # both draw the same random numbers: most trajectories reach the same verdict
    assert (gp['verdict'][0] == gm['verdict'][0]).mean() >= 0.95


def test_trace_capacity_bound_gives_status_3(ctx):
    import torch
    _, kind, formula, t_max, _ = CASES[0]
    m, prop = _model(kind, formula)
    ctx.set_option('trace_cap', 16)  # immigration-death reaches its verdicts after ~475 events
    try:
        g = _run(ctx, m, prop, t_max, 512, 'plain', seed=3)
    finally:
        ctx.set_option('trace_cap', 4096)
    st, c = g['status'][0], g['counts'][0]
    # a trajectory decided within its first 16 positions may still finish
    assert (st == 3).mean() > 0.99 and set(np.unique(st)) <= {0, 3}
    assert int(c[3]) == int((st == 3).sum()) and int(c[1]) == int((st == 0).sum())
    torch.cuda.synchronize()


def test_trace_monitor_refuses_the_snapshot_paths(ctx, smc):
    _, kind, formula, t_max, _ = CASES[0]
    m, prop = _model(kind, formula)
    ctx.load_model(m)
    ctx.load_property(prop, t_max=t_max)
    assert ctx.monitor_kind == 'trace'
    with pytest.raises(smc.SmcError):
        ctx.simulate_snapshot('plain', seed=1, n_traj=64, t_snap=5.0)
    # and a formula of the units' fragment is not moved to the trace monitor
    m2, p2 = workloads.immigration_death()
    ctx.load_property(p2)
    assert ctx.monitor_kind == 'units'


def _ext_cases():
    # rate-law factors (Hill repression) and arithmetic atoms: the trace
    # monitor's kernel variant with the EXT code
    from tests.test_gpu_expr import _quotient_model
    m1, p1 = workloads.autorepressor()
    yield 'autorepressor_next_inside_F', m1, workloads.Property(p1.atoms, ('F', 5.0, 40.0, ('X', 0.0, 0.5, A(0))))
    m2, p2 = _quotient_model()
    yield 'quotient_F_inside_U_left', m2, workloads.Property(p2.atoms, ('U', 0.0, 15.0, ('F', 0.0, 1.0, A(0)), A(1)))


@pytest.mark.parametrize('name', ['autorepressor_next_inside_F', 'quotient_F_inside_U_left'])
def test_nested_formula_with_rate_laws_and_expressions(ctx, orc, name):
    m, prop = next((mm, pp) for nm, mm, pp in _ext_cases() if nm == name)
    n = 3000
    g = _run(ctx, m, prop, math.inf, n, 'plain', seed=5)
    r = orc.run(m, prop, seed=5, n_traj=n)
    same = (g['verdict'][0] == r['verdict']) & (g['events'][0].astype(np.uint64) == r['events'])
    print(f'{name}: {int(same.sum())} of {n} equal, p = {g["verdict"][0].mean():.4f}')
    assert same.mean() >= 0.999
    assert (g['status'][0] == r['status']).all()


def test_nested_formula_on_a_batch(ctx, orc):
    # per-instance atoms of the random-network batch, one nested formula shape
    import torch
    b = workloads.random_networks(4096, seed=3)
    idx = [i for i, mm in enumerate(b.models) if mm.n_reactions <= 24][:48]
    sub = workloads.Batch([b.models[i] for i in idx],
                          [workloads.Property(b.properties[i].atoms, ('F', 0.0, 30.0, ('G', 0.5, 1.5, A(0))))
                           for i in idx])
    n = 64
    ctx.load_batch(sub)
    ctx.load_property(sub.properties)
    assert ctx.monitor_kind == 'trace'
    out = ctx.simulate('plain', seed=9, n_traj=n, outputs=('verdict', 'status', 'events'))
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    agree = total = 0
    for row in range(len(idx)):
        r = orc.run(sub.models[row], sub.properties[row], seed=9, instance=row, n_traj=n)
        agree += int(((g['verdict'][row] == r['verdict']) &
                      (g['events'][row].astype(np.uint64) == r['events'])).sum())
        total += n
    print(f'batch: {agree} of {total} equal')
    assert agree / total >= 0.999


def test_nested_formula_at_the_event_budget(ctx, orc):
    # a budget below the events a verdict needs: undecided trajectories stop
    # at the budget with status 1, decided ones keep their decision point
    import torch
    _, kind, formula, t_max, _ = CASES[4]  # G with a lower bound inside F[5, 30]
    m, prop = _model(kind, formula)
    n, budget = 2000, 300
    ctx.load_model(m)
    ctx.load_property(prop, t_max=t_max)
    ctx.set_option('event_budget', budget)
    out = ctx.simulate('plain', seed=13, n_traj=n, outputs=('verdict', 'status', 'events', 't_final'))
    torch.cuda.synchronize()
    g = {k: v.cpu().numpy() for k, v in out.items()}
    r = orc.run(m, prop, seed=13, n_traj=n, budget=budget)
    assert (r['status'] == 1).mean() > 0.2  # the budget binds for many trajectories
    assert (g['status'][0] == r['status']).all()
    assert (g['events'][0].astype(np.uint64) == r['events']).all()
    assert (g['verdict'][0] == r['verdict']).all()
    assert int(g['counts'][0, 3]) == int((r['status'] == 1).sum())


def test_nested_formula_on_absorbing_paths(ctx, orc):
    # pure decay A -> 0 from A0 = 6: paths absorb at A = 0 (no further
    # position), which decides a nested formula at the closed end
    m, _ = workloads.pure_decay(A0=6, k=1.0)
    sp = ['A']
    atoms = [workloads.atom(sp, 'A', '>=', 3), workloads.atom(sp, 'A', '<=', 0)]
    prop = workloads.Property(atoms, ('or', ('F', 0.0, 3.0, ('X', 0.0, 0.3, A(1))),
                                      ('U', 0.0, 4.0, ('F', 0.0, 0.5, A(0)), A(1))))
    n = 4000
    g = _run(ctx, m, prop, math.inf, n, 'plain', seed=2)
    r = orc.run(m, prop, seed=2, n_traj=n, want_x=True)
    assert 0.02 < r['verdict'].mean() < 0.98
    assert (g['verdict'][0] == r['verdict']).all()
    assert (g['events'][0].astype(np.uint64) == r['events']).all()
    assert (g['x_final'][0][:, :1] == r['x_final']).all()
