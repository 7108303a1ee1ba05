"""Parity of the CUDA path (called through the C ABI) with the CPU oracle on the
same seeded inputs.

FP64 path: per-trajectory verdicts must agree on >= 99.99% of trajectories
(in practice all: the reaction sequence is bit-identical, only the FP64
path's table-driven log and glibc's may differ in the last bit of the clock), event counts likewise,
|p_hat difference| <= 1e-3, and the Wilson bounds computed on the device from
the integer counts agree with Eq. 4 to 1e-12 relative.
Mixed path: statistical agreement (p_hat inside the combined intervals) and a
high per-trajectory agreement rate with the FP64 path, since both draw the
same random numbers.
"""
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


@pytest.fixture()
def ctx(smc):
    c = smc.Context(0)
    yield c
    c.close()


def _gpu(ctx, model, prop, n, seed, precision='plain', begin=0, outputs=('verdict', 'status', 'events', 't_final'),
         confidence=0.95, t_max=math.inf):
    import torch
    ctx.load_model(model)
    ctx.load_property(prop, t_max=t_max)
    out = ctx.simulate(precision, seed=seed, traj_begin=begin, n_traj=n, confidence=confidence, outputs=outputs)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _compare_plain(g, r, inst=0, min_agree=0.9999):
    v, rv = g['verdict'][inst], r['verdict']
    agree = (v == rv).mean()
    assert agree >= min_agree, agree
    ev_eq = (g['events'][inst].astype(np.uint64) == r['events'])
    assert ev_eq.mean() >= min_agree
    same = ev_eq & (v == rv)
    tf, rtf = g['t_final'][inst][same], r['t_final'][same]
    rel = np.abs(tf - rtf) / np.maximum(np.abs(rtf), 1e-300)
    assert (rel <= 1e-12).mean() >= min_agree, rel.max()
    assert (g['status'][inst] == r['status']).all()
    return agree


def test_immigration_death_plain_full_config(ctx, orc):
    # F[0,100](A >= 130), 10,000 trajectories, Philox seed 0, Wilson 95%.
    from oracle import wilson
    m, p = workloads.immigration_death()
    n = 10000
    g = _gpu(ctx, m, p, n, seed=0)
    r = orc.run(m, p, seed=0, n_traj=n)
    _compare_plain(g, r)
    yes, dec = int(g['counts'][0, 0]), int(g['counts'][0, 1])
    assert dec == n and yes == int(g['verdict'][0].sum())
    assert abs(yes / n - r['verdict'].mean()) <= 1e-3
    assert int(g['counts'][0, 2]) == int(g['events'][0].sum())
    p_hat, lo, hi = wilson.wilson_interval(yes, dec, 0.95)
    assert abs(g['wilson'][0, 0] - p_hat) <= 1e-15
    assert abs(g['wilson'][0, 1] - lo) <= 1e-12 * lo and abs(g['wilson'][0, 2] - hi) <= 1e-12 * hi


def test_lotka_volterra_plain(ctx, orc):
    m, p = workloads.lotka_volterra()
    n = 20000
    g = _gpu(ctx, m, p, n, seed=7)
    r = orc.run(m, p, seed=7, n_traj=n)
    _compare_plain(g, r)
    assert abs(g['verdict'][0].mean() - r['verdict'].mean()) <= 1e-3


def _report_mismatches(ctx, orc, m, p, seed, g, r, inst=0, limit=20):
    """Indices where verdict, status, event count or clock (beyond 1e-12
    relative) differ, each with the first event at which the GPU and oracle
    states part (tests/_parity.py), printed for the log."""
    from tests._parity import first_divergence, ulps_apart
    v, ev, tf, st = g['verdict'][inst], g['events'][inst].astype(np.uint64), g['t_final'][inst], g['status'][inst]
    rel = np.abs(tf - r['t_final']) / np.maximum(np.abs(r['t_final']), 1e-300)
    bad = np.nonzero((v != r['verdict']) | (ev != r['events']) | (st != r['status']) | (rel > 1e-12))[0]
    found = []
    for k in bad[:limit]:
        d = first_divergence(ctx, orc, m, p, seed, int(k), instance=inst)
        if d['event'] is not None:
            d['clock_ulps'] = ulps_apart(d['gpu']['t'], d['oracle']['t'])
        print(f'trajectory {k}: verdict {v[k]} / {r["verdict"][k]}, events {ev[k]} / {r["events"][k]}, '
              f'first divergence {d}')
        found.append((int(k), d))
    return bad, found


def test_lotka_volterra_full_size_all_trajectories(ctx, orc):
    # the benchmark's workload at full size (10^6 trajectories of one launch,
    # in the launch shape the autotuner picks, as bench.py times it), every
    # trajectory recomputed by the oracle on all host cores: verdicts, event
    # counts, statuses and clocks per trajectory (>= 99.99% equal)
    from oracle import wilson
    m, p = workloads.lotka_volterra()
    n = 1_000_000
    g = _gpu(ctx, m, p, n, seed=0, confidence=0.99)
    v, ev = g['verdict'][0], g['events'][0]
    r = orc.run(m, p, seed=0, n_traj=n)
    bad, found = _report_mismatches(ctx, orc, m, p, 0, g, r)
    print(f'full-size parity: {n - bad.size} of {n} trajectories equal in verdict, events, status and clock; '
          f'verdicts equal {(v == r["verdict"]).sum()}')
    _compare_plain(g, r)
    assert bad.size <= n // 10000
    for _, d in found:  # any divergence is a clock apart in its last bits, never a different reaction
        assert d['event'] is not None and d['gpu']['x'] == d['oracle']['x'] and d['clock_ulps'] <= 4
    # properties of the whole launch: counts, events, the interval from them
    yes, dec = int(g['counts'][0, 0]), int(g['counts'][0, 1])
    assert dec == n and yes == int(v.sum()) and int(g['counts'][0, 2]) == int(ev.astype(np.int64).sum())
    p_hat, lo, hi = wilson.wilson_interval(yes, dec, 0.99)
    assert abs(g['wilson'][0, 1] - lo) <= 1e-12 * lo and abs(g['wilson'][0, 2] - hi) <= 1e-12 * hi
    assert 2.0e-4 < p_hat < 7.0e-4 and abs(ev.mean() - 2358.7) < 5.0
    # the chosen (mixed) path on the same launch: same random numbers, so the
    # verdicts mostly agree, and the estimates lie within the 99.9% intervals
    gm = _gpu(ctx, m, p, n, seed=0, precision='mixed', outputs=('verdict',))
    vm = gm['verdict'][0]
    assert (vm == v).mean() >= 0.99
    ym = int(gm['counts'][0, 0])
    assert ym == int(vm.sum()) and int(gm['counts'][0, 1]) == n
    _, lo_p, hi_p = wilson.wilson_interval(yes, n, 0.999)
    _, lo_m, hi_m = wilson.wilson_interval(ym, n, 0.999)
    assert abs(ym - yes) / n <= (hi_p - lo_p) / 2 + (hi_m - lo_m) / 2


@pytest.mark.parametrize('name', ['dimerisation', 'hetero', 'decay'])
def test_small_networks_plain_with_final_states(ctx, orc, name):
    if name == 'dimerisation':
        m, p = workloads.dimerisation()
    elif name == 'hetero':
        sp = ['A', 'B', 'C']
        m = workloads.Model('hetero', sp, [[0, 1], [0, -1]], [[-1, -1, 1], [-1, 0, 0]], [[0.05, 0.4]], [[6, 4, 0]])
        p = workloads.Property([workloads.atom(sp, 'C', '>=', 2)], ('F', 0.0, 1.5, ('atom', 0)))
    else:
        m, p = workloads.pure_decay(1000, 1.0, 1.0)
    n = 3000
    g = _gpu(ctx, m, p, n, seed=3, outputs=('verdict', 'status', 'events', 't_final', 'x_final'))
    r = orc.run(m, p, seed=3, n_traj=n, want_x=True)
    _compare_plain(g, r)
    same = g['events'][0].astype(np.uint64) == r['events']
    assert (g['x_final'][0][same][:, :m.n_species] == r['x_final'][same]).all()


def test_ranges_chain_and_offsets(ctx, orc):
    # trajectories [500, 1500) in two calls equal one call; counts accumulate
    import torch
    m, p = workloads.immigration_death()
    ctx.load_model(m)
    ctx.load_property(p)
    a = ctx.simulate('plain', seed=5, traj_begin=500, n_traj=1000)
    b1 = ctx.simulate('plain', seed=5, traj_begin=500, n_traj=400)
    b2 = ctx.simulate('plain', seed=5, traj_begin=900, n_traj=600, counts=b1['counts'])
    torch.cuda.synchronize()
    va = a['verdict'].cpu().numpy()[0]
    vb = np.concatenate([b1['verdict'].cpu().numpy()[0], b2['verdict'].cpu().numpy()[0]])
    assert (va == vb).all()
    assert (a['counts'].cpu().numpy() == b2['counts'].cpu().numpy()).all()
    r = orc.run(m, p, seed=5, traj_begin=500, n_traj=1000)
    assert (va == r['verdict']).mean() >= 0.9999
    # a single trajectory and an empty range
    one = ctx.simulate('plain', seed=5, traj_begin=777, n_traj=1)
    torch.cuda.synchronize()
    assert one['verdict'].cpu().numpy()[0, 0] == va[277]
    zero = ctx.simulate('plain', seed=5, traj_begin=0, n_traj=0, outputs=())
    torch.cuda.synchronize()
    assert int(zero['counts'].sum()) == 0


def test_launch_shape_does_not_change_results(ctx):
    import torch
    m, p = workloads.lotka_volterra()
    ctx.load_model(m)
    ctx.load_property(p)
    ref = None
    for warps, refill, bps in [(4, 1, 0), (1, 1, 1), (8, 8, 0), (2, 32, 3)]:
        ctx.set_option('warps_per_block', warps)
        ctx.set_option('refill', refill)
        ctx.set_option('blocks_per_sm', bps)
        for prec in ('plain', 'mixed'):
            o = ctx.simulate(prec, seed=11, traj_begin=0, n_traj=4000, outputs=('verdict', 'events'))
            torch.cuda.synchronize()
            got = (o['verdict'].cpu().numpy(), o['events'].cpu().numpy())
            if ref is None:
                ref = {}
            if prec not in ref:
                ref[prec] = got
            else:
                assert (got[0] == ref[prec][0]).all() and (got[1] == ref[prec][1]).all()


def test_event_budget(ctx, orc):
    m, p = workloads.immigration_death()
    ctx.load_model(m)
    ctx.load_property(p)
    ctx.set_option('event_budget', 100)
    import torch
    o = ctx.simulate('plain', seed=0, traj_begin=0, n_traj=300)
    torch.cuda.synchronize()
    r = orc.run(m, p, seed=0, n_traj=300, budget=100)
    assert (o['status'].cpu().numpy()[0] == r['status']).all()
    c = o['counts'].cpu().numpy()[0]
    assert int(c[3]) == int((r['status'] == 1).sum()) and int(c[1]) + int(c[3]) == 300


def test_unbounded_formula_pessimistic_rule(ctx, orc):
    # F[0,inf)(A >= 5) on pure decay from 3 absorbs (false); on immigration
    # the pessimistic rule at t_max decides the undecided ones false.
    m, _ = workloads.pure_decay(3, 1.0, 1.0)
    p = workloads.Property([workloads.atom(['A'], 'A', '>=', 5)], ('F', 0.0, math.inf, ('atom', 0)))
    g = _gpu(ctx, m, p, 200, seed=1, t_max=10.0)
    r = orc.run(m, p, seed=1, n_traj=200, t_max=10.0)
    assert (g['verdict'][0] == r['verdict']).all() and (g['events'][0].astype(np.uint64) == r['events']).all()
    m2, _ = workloads.immigration_only(0.3, 10.0)
    g = _gpu(ctx, m2, p, 2000, seed=2, t_max=10.0)
    r = orc.run(m2, p, seed=2, n_traj=2000, t_max=10.0)
    _compare_plain(g, r)


def test_mixed_path_statistics(ctx, orc):
    from oracle import wilson
    for mk, n in [(workloads.immigration_death, 20000), (workloads.lotka_volterra, 40000)]:
        m, p = mk()
        gp = _gpu(ctx, m, p, n, seed=21, precision='plain')
        gm = _gpu(ctx, m, p, n, seed=21, precision='mixed')
        agree = (gp['verdict'][0] == gm['verdict'][0]).mean()
        assert agree >= 0.99, agree
        yp, ym = int(gp['verdict'][0].sum()), int(gm['verdict'][0].sum())
        _, lo_p, hi_p = wilson.wilson_interval(yp, n, 0.999)
        _, lo_m, hi_m = wilson.wilson_interval(ym, n, 0.999)
        assert abs(ym - yp) / n <= (hi_p - lo_p) / 2 + (hi_m - lo_m) / 2


def _oracle_decision_point(orc, prop, S, x, t, tmin, closed):
    n = len(t)
    for q in range(2 * n):
        k = q // 2
        if q % 2 == 0:
            v = orc.eval_prefix(prop, S, x[:k + 1], t[:k + 1], t[k], False)
        elif k + 1 < n:
            # after the draw the next entry time is known exactly
            v = orc.eval_prefix(prop, S, x[:k + 1], t[:k + 1], t[k + 1], False, tmin_exact=True)
        else:
            v = orc.eval_prefix(prop, S, x, t, tmin, closed)
        if v != 2:
            return v, q
    return 2, -1


def test_monitor_replay_matches_oracle(ctx, orc):
    # The compiled monitor (the device code the SSA kernel steps) against
    # the oracle's trace semantics on exhaustive tiny paths: the verdict and
    # the point at which it becomes fixed.
    import random
    from tests.test_oracle_monitor import FORMULAS, _atoms, _paths
    sp = ['A']
    m = workloads.Model('one', sp, [[0, -1]], [[-1]], [[1.0]], [[3]])
    for fi, f in enumerate(FORMULAS):
        prop = workloads.Property(_atoms(), f)
        ctx.load_model(m)
        ctx.load_property(prop)
        rng = random.Random(1000 + fi)
        paths = []
        for xs, ts in _paths(rng, 400):
            closed = rng.random() < 0.3
            tmin = math.inf if closed else ts[-1] + rng.choice([0.0, 0.5, 1.0, 3.0])
            paths.append((np.asarray(xs), np.asarray(ts, float), tmin, closed))
        v, q = ctx.monitor_replay(paths, 1)
        for i, (xs, ts, tmin, closed) in enumerate(paths):
            ov, oq = _oracle_decision_point(orc, prop, 1, xs, ts, tmin, closed)
            want = {0: 1, 1: 2, 2: 0}[ov]
            assert (v[i], q[i]) == (want, oq), (f, xs.tolist(), ts.tolist(), tmin, closed, v[i], q[i], ov, oq)


def test_iterative_estimate_matches_oracle_fig2(ctx, orc):
    # smc_estimate (Fig. 2 on the host, kernels per batch) against the
    # oracle's Fig. 2 driven by oracle trajectories: same batches, counts
    # and interval.
    from oracle import wilson
    m, p = workloads.lotka_volterra()
    ctx.load_model(m)
    ctx.load_property(p)
    res = ctx.estimate(0.95, 0.01, seed=4, precision='plain', sampling='iterative')[0]

    def run(begin, count):
        r = orc.run(m, p, seed=4, traj_begin=begin, n_traj=count)
        return int(r['verdict'].sum()), int((r['status'] == 0).sum())

    ref = wilson.iterative(run, 0.01, 0.95)
    assert res['launched'] == ref['n_tot'] and res['yes'] == ref['yes']
    assert res['iterations'] == ref['iterations']
    assert abs(res['lo'] - ref['lo']) <= 1e-12 * max(ref['lo'], 1e-300) + 1e-300
    assert abs(res['hi'] - ref['hi']) <= 1e-12 * ref['hi']
    cons = ctx.estimate(0.99, 0.025, seed=4, precision='plain', sampling='conservative')[0]
    assert cons['launched'] == 2648 and cons['iterations'] == 1


def test_fixed_estimate_records_verdicts(ctx, orc):
    m, p = workloads.immigration_death()
    ctx.load_model(m)
    ctx.load_property(p)
    ctx.set_option('record', 1)
    res = ctx.estimate(0.95, 0.01, seed=0, precision='plain', sampling='fixed', fixed_n=5000)[0]
    v = ctx.get_verdicts(5000)
    r = orc.run(m, p, seed=0, n_traj=5000)
    assert (v == r['verdict']).mean() >= 0.9999 and res['yes'] == int(v.sum())


def test_invalid_arguments_are_rejected(ctx, smc):
    m, p = workloads.immigration_death()
    bad = workloads.Model('bad', ['A'], [[-1, -1], [0, -1]], [[1], [-1]], [[10.0, -0.1]], [[0]])
    with pytest.raises(smc.SmcError) as e:
        ctx.load_model(bad)
    assert e.value.code == -1
    ctx.load_model(m)
    # F nested in the left operand of U: beyond the units, on the trace monitor
    ctx.load_property(workloads.Property(p.atoms, ('U', 0, 5, ('F', 0, 1, ('atom', 0)), ('atom', 0))))
    assert ctx.monitor_kind == 'trace'
    deep = ('atom', 0)
    for _ in range(10):  # a formula tree 11 nodes high: beyond the trace monitor too
        deep = ('F', 0.0, 1.0, deep)
    with pytest.raises(smc.SmcError) as e:
        ctx.load_property(workloads.Property(p.atoms, ('U', 0, 5, deep, ('atom', 0))))
    assert e.value.code == -4
    with pytest.raises(smc.SmcError) as e:  # interval with lo > hi
        ctx.load_property(workloads.Property(p.atoms, ('F', 5.0, 1.0, ('atom', 0))))
    assert e.value.code == -1
    with smc.Context(0) as fresh:  # estimate before the property
        fresh.load_model(m)
        with pytest.raises(smc.SmcError) as e:
            fresh.estimate(0.95, 0.01, sampling='iterative')
        assert e.value.code == -5
