"""The three-tier phosphorylation cascade (22 species, 30 reactions, ~1e4
counts, 2e4-7e4 events per trajectory), rate-perturbed instances, with the
literal property (KPP<500) U[0,200] (KPP>=2000 & F[0,50] KPP<500), which is
false on every path (every reaction moves KPP by at most 1, so the first
state with KPP >= 500 has KPP = 500 and satisfies neither operand), and the
variant with left operand KPP<2000 (nested F window exercised).  FP64 path
against the oracle per trajectory; the literal property's exact value 0."""
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


@pytest.mark.parametrize('variant', [False, True])
def test_cascade_plain_matches_oracle(smc, orc, variant):
    # all 8 instances x 200 trajectories, FP64 path, per trajectory against
    # the oracle: verdicts, statuses, event counts, final states and clocks;
    # any trajectory whose event count differs must part from the oracle
    # only by a clock a few ulps apart (tests/_parity.py), which is logged
    import torch
    from tests._parity import first_divergence, ulps_apart
    n_inst, n = 8, 200
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
        for inst in range(n_inst):
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
            print(f'instance {inst}: {same.sum()} of {n} event counts equal, mean events {r["events"].mean():.0f}')
        assert n_bad <= 2
    assert int(g['counts'][:, 3].sum()) == 0


def test_cascade_literal_is_zero_at_scale(smc):
    # 256 rate-perturbed instances x 2,000 trajectories, mixed path: every
    # verdict false, every trajectory stopped at the KPP = 500 crossing
    m, p = workloads.mapk_cascade(256, seed=5, variant=False)
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        res = ctx.estimate(0.95, 0.01, seed=3, precision='mixed', sampling='fixed', fixed_n=2000)
    assert all(r['yes'] == 0 and r['n'] == 2000 and r['hi'] < 0.002 for r in res)
