"""Batched heterogeneous networks (random mass-action networks of uneven size,
one property shape with per-instance atoms) through smc_load_model_batch:
per-trajectory parity with the oracle on a subsample of instances, the
full-size workload (4096 instances x 10,000 trajectories, graph-captured
estimate, mixed path) checked on sampled trajectories, and independence of
the results from the autotuner's launch choice."""
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


@pytest.fixture(scope='module')
def batch():
    return workloads.random_networks(4096, seed=3)


def _sub(batch, idx):
    return workloads.Batch([batch.models[i] for i in idx], [batch.properties[i] for i in idx])


def test_batch_plain_matches_oracle_per_trajectory(smc, orc, batch):
    import torch
    idx = list(range(0, 4096, 21))  # 196 instances of every size class
    sub = _sub(batch, idx)
    n = 96
    with smc.Context(0) as ctx:
        ctx.load_batch(sub)
        ctx.load_property(sub.properties)
        out = ctx.simulate('plain', seed=9, traj_begin=0, n_traj=n,
                           outputs=('verdict', 'status', 'events', 't_final'))
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in out.items()}
    agree = ev_eq = total = 0
    for row, m in enumerate(idx):
        # instance row `row` of the batch keys its random numbers by `row`
        r = orc.run(sub.models[row], sub.properties[row], seed=9, instance=row, n_traj=n)
        agree += int((g['verdict'][row] == r['verdict']).sum())
        ev_eq += int((g['events'][row].astype(np.uint64) == r['events']).sum())
        total += n
        assert int(g['counts'][row, 1] + g['counts'][row, 3]) == n
    assert agree / total >= 0.9999, agree / total
    assert ev_eq / total >= 0.9999, ev_eq / total
    sizes = {sub.models[i].n_reactions for i in range(len(idx))}
    assert min(sizes) <= 8 and max(sizes) > 32  # small and generic paths both ran


def test_batch_full_size_sampled(smc, orc, batch):
    # the configuration the benchmark times: 4096 instances x 10,000
    # trajectories, one graph-captured estimate, mixed path; sampled
    # trajectories against the oracle (agreement of the mixed path with
    # FP64) and the per-instance estimates against the plain path
    n = 10000
    with smc.Context(0) as ctx:
        ctx.load_batch(batch)
        ctx.load_property(batch.properties)
        ctx.set_option('record', 1)
        res = ctx.estimate(0.95, 0.01, seed=1, precision='mixed', sampling='fixed', fixed_n=n)
        v = ctx.get_verdicts(4096 * n).reshape(4096, n)
        resp = ctx.estimate(0.95, 0.01, seed=1, precision='plain', sampling='fixed', fixed_n=n)
        vp = ctx.get_verdicts(4096 * n).reshape(4096, n)
    assert all(r['launched'] == n for r in res)
    assert sum(r['budget_hits'] for r in res) == 0
    rng = np.random.default_rng(0)
    inst = rng.choice(4096, 48, replace=False)
    agree = agree_p = total = 0
    for m in inst:
        ks = np.sort(rng.choice(n, 40, replace=False))
        want = np.array([orc.run(batch.models[m], batch.properties[m], seed=1, instance=int(m),
                                 traj_begin=int(k), n_traj=1, threads=1)['verdict'][0] for k in ks])
        agree += int((v[m, ks] == want).sum())
        agree_p += int((vp[m, ks] == want).sum())
        total += len(ks)
    assert agree_p / total >= 0.9999, agree_p / total
    assert agree / total >= 0.99, agree / total
    # per-instance p_hat of the mixed path within the plain path's interval
    # widened by the mixed one's (both 95%, 10,000 trajectories)
    pm = np.array([r['p_hat'] for r in res])
    pp = np.array([r['p_hat'] for r in resp])
    hw = np.array([(r['hi'] - r['lo']) / 2 for r in resp]) + np.array([(r['hi'] - r['lo']) / 2 for r in res])
    assert (np.abs(pm - pp) <= hw + 1e-12).mean() >= 0.99


def test_autotuned_and_fixed_shapes_give_identical_counts(smc, batch):
    sub = _sub(batch, list(range(0, 4096, 8)))
    results = []
    for autotune in (1, 0):
        with smc.Context(0) as ctx:
            ctx.load_batch(sub)
            ctx.load_property(sub.properties)
            ctx.set_option('autotune', autotune)
            if not autotune:
                ctx.set_option('warps_per_block', 2)
            res = ctx.estimate(0.95, 0.02, seed=5, precision='mixed', sampling='iterative')
            results.append([(r['yes'], r['n'], r['events'], r['launched']) for r in res])
    assert results[0] == results[1]


def test_launch_shapes_cover_instances_and_survive_reload(smc, batch):
    sub = _sub(batch, list(range(0, 4096, 16)))
    with smc.Context(0) as ctx:
        ctx.load_batch(sub)
        ctx.load_property(sub.properties)
        first = ctx.estimate(0.95, 0.05, seed=7, precision='mixed', sampling='fixed', fixed_n=64)
        shapes = ctx.launch_shapes('mixed')
        assert sum(s['n_instances'] for s in shapes) == len(sub.models)
        for s in shapes:
            assert s['warps_per_block'] in (2, 4, 8) and s['refill'] in (1, 8) and s['blocks_per_sm'] >= 1
        # same structure loaded again: the tuned shapes are kept (no new trials)
        ctx.load_batch(sub)
        ctx.load_property(sub.properties)
        again = ctx.estimate(0.95, 0.05, seed=7, precision='mixed', sampling='fixed', fixed_n=64)
        assert ctx.launch_shapes('mixed') == shapes
        assert [(r['yes'], r['events']) for r in again] == [(r['yes'], r['events']) for r in first]
        # an explicit shape replaces the tuned one
        ctx.set_option('warps_per_block', 2)
        ctx.set_option('refill', 4)
        ctx.estimate(0.95, 0.05, seed=7, precision='mixed', sampling='fixed', fixed_n=64)
        fixed = ctx.launch_shapes('mixed')
        assert all(s['warps_per_block'] == 2 and s['refill'] == 4 for s in fixed)
        assert sum(s['n_instances'] for s in fixed) == len(sub.models)


@pytest.fixture(scope='module')
def large():
    return workloads.random_networks_large(96, seed=8)


def test_large_networks_selection_modes_and_oracle(smc, orc, large):
    # networks of 65 to 255 reactions: the FP64 path's selection by running
    # sums checkpointed every 16 reactions (automatic above 64 reactions, and
    # forced from 17) gives the linear scan's trajectories bit for bit, and
    # both match the oracle per trajectory
    import torch
    n = 64
    outs = {}
    for sel in (1, 0, 2):
        with smc.Context(0) as ctx:
            ctx.set_option('selection', sel)
            ctx.load_batch(large)
            ctx.load_property(large.properties)
            out = ctx.simulate('plain', seed=4, traj_begin=0, n_traj=n,
                               outputs=('verdict', 'status', 'events', 't_final'))
            torch.cuda.synchronize()
            outs[sel] = {k: v.cpu().numpy() for k, v in out.items()}
    for sel in (0, 2):
        for k in ('verdict', 'status', 'events', 't_final', 'counts'):
            assert np.array_equal(outs[sel][k], outs[1][k]), (sel, k)
    g = outs[0]
    agree = ev_eq = total = 0
    for row in range(len(large.models)):
        r = orc.run(large.models[row], large.properties[row], seed=4, instance=row, n_traj=n)
        agree += int((g['verdict'][row] == r['verdict']).sum())
        ev_eq += int((g['events'][row].astype(np.uint64) == r['events']).sum())
        total += n
    assert agree / total >= 0.9999 and ev_eq / total >= 0.9999, (agree / total, ev_eq / total)
    assert max(m.n_reactions for m in large.models) > 200 and int(g['counts'][:, 2].sum()) > 10 ** 7


def test_large_networks_mixed_selection_modes_agree(smc, large):
    # the mixed path keeps FP32 block sums along the dependency graph: its
    # estimates with checkpoints and with the linear scan agree within their
    # combined intervals, instance by instance
    from oracle import wilson
    n = 4000
    res = {}
    for sel in (1, 2):
        with smc.Context(0) as ctx:
            ctx.set_option('selection', sel)
            ctx.load_batch(large)
            ctx.load_property(large.properties)
            res[sel] = ctx.estimate(0.95, 0.01, seed=6, precision='mixed', sampling='fixed', fixed_n=n)
    for a, b in zip(res[1], res[2]):
        assert a['n'] == b['n'] == n
        _, lo_a, hi_a = wilson.wilson_interval(a['yes'], n, 0.9999)
        _, lo_b, hi_b = wilson.wilson_interval(b['yes'], n, 0.9999)
        assert abs(a['yes'] - b['yes']) / n <= (hi_a - lo_a) / 2 + (hi_b - lo_b) / 2, (a, b)
