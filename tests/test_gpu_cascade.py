"""The three-tier phosphorylation cascade (22 species, 30 reactions, counts
up to about 6,000, about 1.4e5 events per trajectory under the variant),
256 rate-perturbed instances, with the literal property (KPP<500) U[0,200]
(KPP>=2000 & F[0,50] KPP<500), which is false on every path (every reaction
moves KPP by at most 1, so the first state with KPP >= 500 has KPP = 500 and
satisfies neither operand), and the variant with left operand KPP<2000
(nested F window exercised; its probability differs from instance to
instance).  FP64 path against the oracle per trajectory on 1,000-trajectory
subsamples; the literal property's exact value 0 at the configured size;
the control variate on the variant, unbiased against the plain estimator."""
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


@pytest.mark.parametrize('variant,instances,n', [(False, range(8), 200), (True, (0, 2, 4, 6), 1000)])
def test_cascade_plain_matches_oracle(smc, orc, variant, instances, n):
    # FP64 path, per trajectory against the oracle: verdicts, statuses, event
    # counts, final states and clocks (the literal formula on 8 instances x
    # 200 trajectories, the variant on a 1,000-trajectory subsample of four
    # instances); any trajectory whose event count differs must part from the
    # oracle only by a clock a few ulps apart (tests/_parity.py), which is logged
    import torch
    from tests._parity import first_divergence, ulps_apart
    n_inst = 8
    m, p = workloads.mapk_cascade(n_inst, seed=5, variant=variant)
    kpp = workloads.MAPK_SPECIES.index('KPP')
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        out = ctx.simulate('plain', seed=2, traj_begin=0, n_traj=n,
                           outputs=('verdict', 'status', 'events', 't_final', 'x_final'))
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in out.items()}
        n_bad = 0
        for inst in instances:
            r = orc.run(m, p, seed=2, instance=inst, n_traj=n, want_x=True)
            ev = g['events'][inst].astype(np.uint64)
            same = ev == r['events']
            assert (g['verdict'][inst] != r['verdict']).sum() <= 1
            assert (g['status'][inst] == r['status']).all()
            assert (g['x_final'][inst][same][:, :22] == r['x_final'][same]).all()
            rel = np.abs(g['t_final'][inst][same] - r['t_final'][same]) / r['t_final'][same]
            assert (rel <= 1e-12).all(), rel.max()
            for k in np.nonzero(~same | (g['verdict'][inst] != r['verdict']))[0]:
                n_bad += 1
                d = first_divergence(ctx, orc, m, p, 2, int(k), instance=inst)
                d['clock_ulps'] = ulps_apart(d['gpu']['t'], d['oracle']['t']) if d['event'] else None
                print(f'instance {inst} trajectory {k}: events {ev[k]} / {r["events"][k]}, first divergence {d}')
                assert d['event'] is not None and d['gpu']['x'] == d['oracle']['x'] and d['clock_ulps'] <= 4
            if not variant:
                assert (r['verdict'] == 0).all() and (r['x_final'][:, kpp] == 500).all()
            print(f'instance {inst}: {same.sum()} of {n} event counts equal, mean events {r["events"].mean():.0f}, '
                  f'p {r["verdict"].mean():.3f}')
        assert n_bad <= 2
    assert int(g['counts'][:, 3].sum()) == 0


def test_cascade_literal_is_zero_at_scale(smc):
    # the configured size: 256 rate-perturbed instances x 100,000
    # trajectories in one batched launch (mixed path): every verdict false,
    # so every interval is Eq. 4 at 0 / 10^5
    m, p = workloads.mapk_cascade(256, seed=5, variant=False)
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        res = ctx.estimate(0.95, 0.01, seed=3, precision='mixed', sampling='fixed', fixed_n=100_000)
    assert all(r['yes'] == 0 and r['n'] == 100_000 and r['budget_hits'] == 0 for r in res)
    assert max(r['hi'] for r in res) < 4e-5


# the surrogate's inputs on the cascade: the active forms along the chain and
# the time (22 counts and 30 rates would exceed the network's 16 inputs)
CASCADE_FEATURES = ('KKKs', 'KKP', 'KKPP', 'KP', 'KPP', 'KP_KKPP', 'KPP_KPase')


@pytest.mark.gpu
def test_cascade_variant_control_variate(smc):
    # A network trained on prefixes of the 256-instance batch at t_c = 30
    # (labelled by their verdicts) serves as the control variate on held-out
    # instances: the estimate agrees with a plain estimate of 2 x 10^4
    # trajectories within their combined error, for any network.
    import math
    import torch
    m, p = workloads.mapk_cascade(256, seed=5, variant=True)
    idx = [workloads.MAPK_SPECIES.index(s) for s in CASCADE_FEATURES]
    t_c, xs, ts = 30.0, np.full(len(idx), 2000.0, np.float32), 200.0
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        ctx.set_features(species=idx, with_rates=False)
        o = ctx.simulate_snapshot('mixed', seed=21, traj_begin=0, n_traj=800, t_snap=t_c)
        feat = ctx.snapshot_features(o['x_snap'], t_c, xs, ts)
        alive = (o['snap'] == 0).reshape(-1)
        x = feat[alive].contiguous()
        y = o['verdict'].reshape(-1)[alive].to(torch.float32).contiguous()
        torch.cuda.synchronize()
        assert x.shape[0] > 100_000 and 0.05 < float(y.mean()) < 0.95, (x.shape, float(y.mean()))
        net = smc.Mlp(len(idx) + 1, seed=5)
        loss = net.train(x, y, epochs=4, batch=8192, lr=1e-3, seed=6)
        assert loss[-1] < loss[0], loss
    for i in (0, 4):
        with smc.Context(0) as ctx:
            ctx.load_model(m.instance(i))
            ctx.load_property(p)
            ctx.set_features(species=idx, with_rates=False)
            cv = ctx.estimate_cv(net, 0.95, 0.02, seed=31 + i, precision='mixed', t_snap=t_c, x_scale=xs,
                                 t_scale=ts, beta=1.0, pilot=1000)
            big = ctx.estimate(0.95, 0.02, seed=41 + i, precision='mixed', sampling='fixed', fixed_n=20_000)[0]
        sd_big = math.sqrt(max(big['p_hat'] * (1 - big['p_hat']), 1e-12) / big['n'])
        assert abs(cv['p_hat'] - big['p_hat']) <= 4 * math.sqrt(cv['var']) + 4 * sd_big, (cv, big)
        print(f'instance {i}: p (2e4 plain) {big["p_hat"]:.4f}, cv {cv["p_hat"]:.4f} (n_eff {cv["n_eff"]:.0f}, '
              f'full {cv["n_full"]}, prefix {cv["n_prefix"]}, events {cv["events_full"] + cv["events_prefix"]:.3g})')
