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
    import torch
    m, p = workloads.mapk_cascade(8, seed=5, variant=variant)
    n = 12
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        out = ctx.simulate('plain', seed=2, traj_begin=0, n_traj=n,
                           outputs=('verdict', 'status', 'events', 't_final', 'x_final'))
        torch.cuda.synchronize()
        g = {k: v.cpu().numpy() for k, v in out.items()}
    kpp = workloads.MAPK_SPECIES.index('KPP')
    for inst in range(0, 8, 3):
        r = orc.run(m, p, seed=2, instance=inst, n_traj=n, want_x=True)
        assert (g['verdict'][inst] == r['verdict']).all()
        assert (g['events'][inst].astype(np.uint64) == r['events']).mean() >= 0.9
        same = g['events'][inst].astype(np.uint64) == r['events']
        assert (g['x_final'][inst][same][:, :22] == r['x_final'][same]).all()
        if not variant:
            assert (r['verdict'] == 0).all() and (r['x_final'][:, kpp] == 500).all()
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
