"""The surrogate control variate: BF16 tensor-core network against the FP64
oracle network (forward and gradients), training, checkpoint snapshots
against the oracle's trajectories, and the control-variate estimator
(unbiased with an untrained network, tighter with a trained one) against the
exact value of the immigration-death workload."""
import math

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu

EXACT_C1 = 0.0912186  # P(F[0,100] A >= 130), CME solve (tests/_cme.py)


@pytest.fixture(scope='module')
def env():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no GPU')
    import paper_0912_2551_gb300 as smc
    return torch, smc


def _bf16_weights(theta):
    from oracle import mlp as om
    t = np.asarray(theta, np.float64).copy()
    for name in ('W1', 'W2', 'W3'):
        o, s = om.OFF[name]
        t[o:o + s] = om.bf16_round(t[o:o + s])
    return t


def test_network_matches_oracle(env):
    torch, smc = env
    from oracle import mlp as om
    rng = np.random.default_rng(0)
    n = 3000
    x = rng.normal(size=(n, 6)).astype(np.float32)
    y = (rng.random(n) < 1 / (1 + np.exp(-x[:, 0] + x[:, 1]))).astype(np.float32)
    net = smc.Mlp(6, seed=3)
    theta = net.get_params()
    xt, yt = torch.tensor(x, device='cuda'), torch.tensor(y, device='cuda')
    torch.cuda.synchronize()
    g_gpu = net.predict(xt).cpu().numpy()
    tb = _bf16_weights(theta)
    xb = om.bf16_round(x)
    z_ref, _ = om.forward(tb, xb)
    g_ref = 1 / (1 + np.exp(-z_ref))
    assert np.max(np.abs(g_gpu - g_ref)) < 0.02
    grad, loss = net.gradient(xt, yt)
    gref = om.gradient(tb, xb, y)
    assert abs(loss - om.loss(tb, xb, y)) < 0.01 * om.loss(tb, xb, y)
    for name in ('W1', 'b1', 'W2', 'b2', 'W3', 'b3', 'w4', 'b4'):
        o, s = om.OFF[name]
        a, b = grad[o:o + s].astype(np.float64), gref[o:o + s]
        if name in ('W1',):
            a, b = a.reshape(128, 16)[:, :6], b.reshape(128, 16)[:, :6]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-12)
        cos = float(np.dot(a.ravel(), b.ravel()) / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))
        assert rel < 0.06 and cos > 0.998, (name, rel, cos)


def _forward_bf16_activations(theta, x):
    """The oracle network's layers with every hidden activation rounded to
    BF16, as the library's kernels store them between layers."""
    from oracle import mlp as om
    P = om.unpack(theta)
    h = om.pad(om.bf16_round(x))
    for W, b in (('W1', 'b1'), ('W2', 'b2'), ('W3', 'b3')):
        h = om.bf16_round(np.maximum(h @ P[W].T + P[b], 0.0))
    z = h @ P['w4'] + P['b4'][0]
    return 1 / (1 + np.exp(-z))


@pytest.mark.parametrize('n', [1, 127, 128, 129, 3000, 100_003])
def test_inference_tiles_and_mask(env, n):
    """Inference kernel (128-row tensor-core tiles, persistent over the
    tiles): exact tile sizes, ragged tails, more tiles than CTAs, and a mask
    that skips single rows and whole tiles, whose outputs must stay as they
    were."""
    torch, smc = env
    rng = np.random.default_rng(n)
    x = rng.normal(size=(n, 6)).astype(np.float32)
    net = smc.Mlp(6, seed=11)
    theta = _bf16_weights(net.get_params())
    g_ref = _forward_bf16_activations(theta, x)
    xt = torch.tensor(x, device='cuda')
    g = net.predict(xt).cpu().numpy()
    assert np.all(np.isfinite(g))
    err = np.abs(g.astype(np.float64) - g_ref)
    assert err.max() < 5e-3 and err.mean() < 5e-4, (err.max(), err.mean())
    skip = (rng.random(n) < 0.3).astype(np.uint8)
    skip[128:256] = 1  # a whole tile skipped
    sentinel = np.float32(-7.0)
    out = torch.full((n,), float(sentinel), dtype=torch.float32, device='cuda')
    gm = net.predict(xt, skip=torch.tensor(skip, device='cuda'), out=out).cpu().numpy()
    assert np.all(gm[skip == 1] == sentinel)
    assert np.array_equal(gm[skip == 0], g[skip == 0])


def test_training_learns_a_logistic_target(env):
    torch, smc = env
    rng = np.random.default_rng(1)
    n = 60000
    x = rng.normal(size=(n, 4)).astype(np.float32)
    p = 1 / (1 + np.exp(-(2 * x[:, 0] - x[:, 1] * x[:, 2])))
    y = (rng.random(n) < p).astype(np.float32)
    net = smc.Mlp(4, seed=2)
    xt, yt = torch.tensor(x, device='cuda'), torch.tensor(y, device='cuda')
    torch.cuda.synchronize()
    loss = net.train(xt, yt, epochs=6, batch=2048, lr=2e-3, seed=5)
    ent = float(np.mean(-(p * np.log(p) + (1 - p) * np.log(1 - p))))
    assert loss[-1] < loss[0] and loss[-1] < ent + 0.03, (loss, ent)
    g = net.predict(xt).cpu().numpy()
    assert np.corrcoef(g, p)[0, 1] > 0.95


def test_snapshots_match_oracle(env, orc):
    torch, smc = env
    m, p = workloads.lotka_volterra()
    t_snap, n = 0.5, 2000
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        full = ctx.simulate_snapshot('plain', seed=4, n_traj=n, t_snap=t_snap)
        pre = ctx.simulate_snapshot('plain', seed=4, n_traj=n, t_snap=t_snap, stop=True)
        torch.cuda.synchronize()
        f = {k: v.cpu().numpy() for k, v in full.items()}
        q = {k: v.cpu().numpy() for k, v in pre.items()}
    # the state occupied at t_snap: the oracle run under G[0,t_snap](true)
    always = workloads.Property([workloads.atom(m.species, 'X', '>=', 0)], ('G', 0.0, t_snap, ('atom', 0)))
    r = orc.run(m, always, seed=4, n_traj=n, want_x=True)
    alive = f['snap'][0] == 0
    assert alive.sum() > n // 2
    assert (f['x_snap'][0][alive] == r['x_final'][alive]).all()
    rp = orc.run(m, p, seed=4, n_traj=n)
    assert (rp['t_final'][~alive] <= t_snap).all()  # decided at a state entered before t_snap
    # prefix-only runs see the same snapshots and stop there, uncounted
    assert (q['snap'] == f['snap']).all() and (q['x_snap'][0][alive] == f['x_snap'][0][alive]).all()
    assert (q['status'][0][alive] == 2).all()
    assert int(q['counts'][0, 1]) == int((~alive).sum())


def _c1_features(t_snap):
    return np.array([100.0], np.float32), 100.0


def test_control_variate_untrained_is_unbiased(env):
    torch, smc = env
    m, p = workloads.immigration_death()
    net = smc.Mlp(4, seed=11)  # random network: g is an arbitrary function
    xs, ts = _c1_features(50.0)
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        res = ctx.estimate_cv(net, 0.9999, 0.01, seed=7, precision='plain', t_snap=50.0, x_scale=xs,
                              t_scale=ts, beta=1.0, pilot=4000)
    assert res['lo'] <= EXACT_C1 <= res['hi'], res
    assert res['n_full'] >= 4000


def test_control_variate_with_one_verdict_stops_like_fig2(env):
    # p = 0 (the threshold is never reached): while the full runs hold only
    # one verdict the variance estimate says nothing about Y, so n_eff is the
    # full sample and the loop stops where Fig. 2 stops at p_hat = 0
    torch, smc = env
    m, _ = workloads.immigration_death()
    never = workloads.Property([workloads.atom(['A'], 'A', '>=', 100000)], ('F', 0.0, 100.0, ('atom', 0)))
    net = smc.Mlp(4, seed=11)
    xs, ts = _c1_features(50.0)
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(never)
        res = ctx.estimate_cv(net, 0.95, 0.01, seed=7, precision='mixed', t_snap=50.0, x_scale=xs,
                              t_scale=ts, beta=1.0, pilot=100)
        plain = ctx.estimate(0.95, 0.01, seed=7, precision='mixed', sampling='iterative')[0]
    assert plain['p_hat'] == 0.0
    assert res['n_full'] <= plain['n'] and res['n_prefix'] == 0, (res, plain)
    assert res['n_eff'] == res['n_full'] and res['lo'] <= 0.0 + 1e-12 and res['hi'] <= 0.01, res


def _held_out_beta(ctx, net, t_snap, xs, ts, seed):
    """beta = Cov(Y, G) / Var(G) and the residual share Var(Y - beta G) / Var(Y)
    on held-out trajectories (a seed disjoint from training and estimation)."""
    h = ctx.simulate_snapshot('mixed', seed=seed, n_traj=50000, t_snap=t_snap)
    gh = net.predict(ctx.snapshot_features(h['x_snap'], t_snap, xs, ts)).cpu().numpy()
    yh = h['verdict'][0].cpu().numpy().astype(float)
    decided = h['snap'][0].cpu().numpy() == 1
    G = np.where(decided, yh, gh)
    beta = float(np.cov(yh, G)[0, 1] / np.var(G, ddof=1))
    calib = abs(float(gh[~decided].mean() - yh[~decided].mean()))
    return beta, float(np.var(yh - beta * G) / np.var(yh)), calib


def test_control_variate_trained_gains(env):
    # Train g on snapshots at t = 80 labelled by their verdicts, then compare
    # with an untrained network: the trained one explains more of the
    # verdict's variance on held-out trajectories, and its estimate reaches a
    # larger effective sample size per full trajectory; both stay unbiased.
    torch, smc = env
    m, p = workloads.immigration_death()
    t_snap = 80.0
    xs, ts = _c1_features(t_snap)
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        o = ctx.simulate_snapshot('mixed', seed=123, n_traj=200000, t_snap=t_snap)
        feat = ctx.snapshot_features(o['x_snap'], t_snap, xs, ts)
        alive = (o['snap'][0] == 0)
        x_train = feat[alive].contiguous()
        y_train = o['verdict'][0][alive].to(torch.float32).contiguous()
        torch.cuda.synchronize()
        trained = smc.Mlp(4, seed=1)
        loss = trained.train(x_train, y_train, epochs=8, batch=4096, lr=2e-3, seed=2)
        assert loss[-1] < loss[0]
        untrained = smc.Mlp(4, seed=1)
        out = {}
        for name, net in (('trained', trained), ('untrained', untrained)):
            beta, resid, calib = _held_out_beta(ctx, net, t_snap, xs, ts, 321)
            res = ctx.estimate_cv(net, 0.95, 0.005, seed=9, precision='mixed', t_snap=t_snap, x_scale=xs,
                                  t_scale=ts, beta=beta, pilot=3000)
            assert abs(res['p_hat'] - EXACT_C1) < 4 * math.sqrt(res['var']) + 2e-4, (name, res)
            out[name] = (resid, calib, res)
    # the trained network explains most of the verdict's variance and is
    # calibrated on the trajectories still undecided at the checkpoint
    assert out['trained'][0] < 0.5 and out['trained'][0] < out['untrained'][0], out
    assert out['trained'][1] < 0.02, out
    # a prefix to t = 80 costs most of a run (the chain is stationary long
    # before): prefix runs cannot pay against the explained variance, so the
    # cost-optimal estimator draws none and n_eff is the full sample's
    res = out['trained'][2]
    assert res['n_prefix'] == 0 and abs(res['n_eff'] / res['n_full'] - 1) < 0.1, res


def test_control_variate_pays_where_the_fate_is_settled_early(env):
    # Linear birth-death survival, G[0,20](A > 0): survivors grow like e^{0.2 t},
    # so a prefix to t = 8 costs ~7% of a run while A(8) settles most of the
    # verdict.  The trained control variate must stay unbiased against the
    # closed form and need fewer events per effective sample than the plain
    # estimator (the cost-optimal split predicts about half).
    torch, smc = env
    from tests.test_oracle_ssa import birth_death_survival_exact
    m, p = workloads.birth_death_survival(1)
    exact = birth_death_survival_exact(1.0, 0.8, 5, 20.0)
    t_snap = 8.0
    xs, ts = np.array([50.0], np.float32), 20.0
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        o = ctx.simulate_snapshot('mixed', seed=31, n_traj=200000, t_snap=t_snap)
        feat = ctx.snapshot_features(o['x_snap'], t_snap, xs, ts)
        alive = (o['snap'][0] == 0)
        x_train = feat[alive].contiguous()
        y_train = o['verdict'][0][alive].to(torch.float32).contiguous()
        e_pre = o['e_snap'][0].double().sum().item()
        e_full = o['counts'][0, 2].double().item()
        torch.cuda.synchronize()
        assert e_pre / e_full < 0.15, e_pre / e_full
        net = smc.Mlp(4, seed=5)
        net.train(x_train, y_train, epochs=6, batch=4096, lr=2e-3, seed=6)
        beta, resid, calib = _held_out_beta(ctx, net, t_snap, xs, ts, 32)
        assert resid < 0.4 and calib < 0.02, (resid, calib)
        res = ctx.estimate_cv(net, 0.95, 0.003, seed=33, precision='mixed', t_snap=t_snap, x_scale=xs,
                              t_scale=ts, beta=beta, pilot=2000)
    assert abs(res['p_hat'] - exact) < 4 * math.sqrt(res['var']), (res, exact)
    assert res['n_prefix'] > res['n_full'], res
    plain_cost = res['n_eff'] * res['events_full'] / res['n_full']
    assert (res['events_full'] + res['events_prefix']) < 0.8 * plain_cost, res
