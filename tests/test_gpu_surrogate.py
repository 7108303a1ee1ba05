"""The surrogate control variate: BF16 tensor-core network against the FP64
oracle network (forward and gradients), training, checkpoint snapshots
against the oracle's trajectories, and the control-variate estimator
(unbiased with an untrained network, tighter with a trained one) against the
exact value of the immigration-death workload."""
import math

import numpy as np
import pytest

import workloads

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


# Element-wise tolerance of a sum S = sum_r t_r computed by the library's
# kernels (BF16 operands, FP32 accumulation) against the same sum in FP64
# over the oracle's BF16-stored operands (oracle/mlp.py with bf16=True).
# The two differ only where an operand, stored in BF16, rounded to the other
# neighbour because the FP32 and FP64 sums before that rounding differed
# (or where such a difference propagated from an earlier layer): each row's
# term then carries an error of at most about one BF16 unit, 2^-8 |t_r| per
# rounding stage upstream, independently across rows (rows never mix before
# the sum).  By Hoeffding's inequality the sum's error stays below
# LAMBDA * 2^-8 * sqrt(STAGES * sum_r t_r^2) except with probability
# 2 exp(-LAMBDA^2 / 2) (3e-8 per element for LAMBDA = 6); FP32 accumulation
# adds at most n 2^-24 sum_r |t_r| (n terms), taken here as 2^-12 sum |t_r|.
LAMBDA, U_BF16 = 6.0, 2.0 ** -8


def _sum_tolerance(t2, tabs, stages):
    return LAMBDA * U_BF16 * np.sqrt(stages * t2) + 2.0 ** -12 * tabs


def _gradient_tolerance(theta, x, y):
    """Per-parameter tolerance (layout of oracle.mlp) for the gradient of the
    mean cross-entropy, from the row terms of each parameter's sum."""
    from oracle import mlp as om
    z, (xp, a1, h1, a2, h2, a3, h3, P) = om.forward(theta, x, bf16=True)
    n = xp.shape[0]
    dz = (1 / (1 + np.exp(-z)) - np.asarray(y, np.float64)) / n
    d3 = om.bf16_round(np.outer(dz, P['w4']) * (a3 > 0))
    d2 = om.bf16_round((d3 @ P['W3']) * (a2 > 0))
    d1 = om.bf16_round((d2 @ P['W2']) * (a1 > 0))
    tol = np.zeros(om.NPARAM)

    def put(name, v):
        o, s = om.OFF[name]
        tol[o:o + s] = np.ravel(v)

    # weight W_l[o][i] = sum_r d_l[r, o] h_{l-1}[r, i]; stages: the forward
    # layers below h_{l-1} and above, and the backward roundings above d_l
    for name, d, h, st in (('W3', d3, h2, 5), ('W2', d2, h1, 6), ('W1', d1, xp, 7)):
        put(name, _sum_tolerance((d ** 2).T @ (h ** 2), np.abs(d).T @ np.abs(h), st))
    for name, d, st in (('b3', d3, 4), ('b2', d2, 5), ('b1', d1, 6)):
        put(name, _sum_tolerance((d ** 2).sum(axis=0), np.abs(d).sum(axis=0), st))
    put('w4', _sum_tolerance((dz ** 2) @ (h3 ** 2), np.abs(dz) @ np.abs(h3), 4))
    put('b4', [2.0 ** -12 * np.abs(dz).sum()])
    return tol


@pytest.mark.gpu
def test_network_matches_oracle_elementwise(env):
    """Forward outputs and every gradient entry of the library's BF16 network
    against the oracle network with the same BF16 storage, element by element
    within the tolerance derived above."""
    torch, smc = env
    from oracle import mlp as om
    rng = np.random.default_rng(0)
    n = 3000
    x = rng.normal(size=(n, 6)).astype(np.float32)
    y = (rng.random(n) < 1 / (1 + np.exp(-x[:, 0] + x[:, 1]))).astype(np.float32)
    net = smc.Mlp(6, seed=3)
    theta = net.get_params().astype(np.float64)
    xt, yt = torch.tensor(x, device='cuda'), torch.tensor(y, device='cuda')
    torch.cuda.synchronize()
    # forward (inference kernel): z = sum_k w4_k h3[r, k] + b4 per row, 3 stages
    g_gpu = net.predict(xt).cpu().numpy().astype(np.float64)
    z_ref, cache = om.forward(theta, x, bf16=True)
    h3, P = cache[6], cache[7]
    t = h3 * P['w4']
    tol_z = _sum_tolerance((t ** 2).sum(axis=1), np.abs(t).sum(axis=1), 3) + 1e-6
    g_ref = 1 / (1 + np.exp(-z_ref))
    err_g = np.abs(g_gpu - g_ref)
    assert np.all(err_g <= 0.25 * tol_z + 2e-7), np.max(err_g / (0.25 * tol_z + 2e-7))  # |sigmoid'| <= 1/4
    # gradient (training kernels), every entry
    grad, loss = net.gradient(xt, yt)
    grad = grad.astype(np.float64)
    gref = om.gradient(theta, x, y, bf16=True)
    tol = _gradient_tolerance(theta, x, y)
    lref = om.loss(theta, x, y, bf16=True)
    assert abs(loss - lref) <= 1e-4 * lref, (loss, lref)
    err = np.abs(grad - gref)
    worst = {}
    for name in ('W1', 'b1', 'W2', 'b2', 'W3', 'b3', 'w4', 'b4'):
        o, s = om.OFF[name]
        e, tl = err[o:o + s], tol[o:o + s] + 1e-9
        worst[name] = float(np.max(e / tl))
        bad = np.nonzero(e > tl)[0]
        assert bad.size == 0, (name, bad[:8], e[bad[:8]], tl[bad[:8]], grad[o + bad[:8]], gref[o + bad[:8]])
    # the padded inputs' weights get exactly zero gradient
    W1g = grad[om.OFF['W1'][0]:om.OFF['W1'][0] + 128 * 16].reshape(128, 16)
    assert np.all(W1g[:, 6:] == 0.0)
    print('largest error / tolerance per block:', worst)


def _gradient_fp32(theta, x, y):
    """The oracle network's gradient with the same BF16 storage but every sum
    accumulated in FP32 (NumPy's own summation order): what a correct kernel
    may differ by."""
    from oracle import mlp as om

    def r(a):
        return om.bf16_round(a).astype(np.float32)

    P = {k: v.astype(np.float32) for k, v in om.unpack(theta, True).items()}
    n = x.shape[0]
    xp = om.pad(r(x)).astype(np.float32)
    h1 = r(np.maximum(xp @ P['W1'].T + P['b1'], 0))
    h2 = r(np.maximum(h1 @ P['W2'].T + P['b2'], 0))
    h3 = r(np.maximum(h2 @ P['W3'].T + P['b3'], 0))
    z = h3 @ P['w4'] + P['b4'][0]
    dz = ((1 / (1 + np.exp(-z)) - y) / n).astype(np.float32)
    d3 = r(np.outer(dz, P['w4']) * (h3 > 0))
    d2 = r((d3 @ P['W3']) * (h2 > 0))
    d1 = r((d2 @ P['W2']) * (h1 > 0))
    g = np.zeros(om.NPARAM)
    for name, v in (('w4', h3.T @ dz), ('b4', [dz.sum()]), ('W3', d3.T @ h2), ('b3', d3.sum(0)),
                    ('W2', d2.T @ h1), ('b2', d2.sum(0)), ('W1', d1.T @ xp), ('b1', d1.sum(0))):
        o, s = om.OFF[name]
        g[o:o + s] = np.ravel(v)
    return g


def test_gradient_tolerance_accepts_fp32_and_rejects_planted_mistakes():
    """The tolerance admits a correct FP32-accumulated computation and is
    tight enough to reject the mistakes a kernel could make: a transposed
    weight block, a dropped bias, a wrong mask, and a single row 10% off,
    each planted in a copy of the oracle's gradient on the CPU."""
    from oracle import mlp as om
    rng = np.random.default_rng(0)
    n = 3000
    x = rng.normal(size=(n, 6)).astype(np.float32)
    y = (rng.random(n) < 1 / (1 + np.exp(-x[:, 0] + x[:, 1]))).astype(np.float32)
    theta = np.zeros(om.NPARAM)
    for name, fan_out, fan_in, used in (('W1', 128, 16, 6), ('W2', 128, 128, 128), ('W3', 128, 128, 128),
                                        ('w4', 1, 128, 128)):
        o, s = om.OFF[name]
        lim = np.sqrt(6.0 / used)
        w = rng.uniform(-lim, lim, (fan_out, fan_in))
        w[:, used:] = 0.0
        theta[o:o + s] = w.ravel()
    for name in ('b1', 'b2', 'b3'):
        o, s = om.OFF[name]
        theta[o:o + s] = rng.normal(0.0, 0.1, s)
    theta = theta.astype(np.float32).astype(np.float64)
    g = om.gradient(theta, x, y, bf16=True)
    tol = _gradient_tolerance(theta, x, y)
    assert np.all(np.abs(_gradient_fp32(theta, x, y) - g) <= 0.1 * tol)

    def rejected(g2):
        return np.any(np.abs(g2 - g) > tol + 1e-9)

    o, s = om.OFF['W2']
    g2 = g.copy()
    g2[o:o + s] = g[o:o + s].reshape(128, 128).T.ravel()
    assert rejected(g2)
    g2 = g.copy()
    g2[o + 5 * 128:o + 6 * 128] *= 1.1  # one row 10% off
    assert rejected(g2)
    # gradient of a network whose second layer has no bias
    t2 = theta.copy()
    t2[om.OFF['b2'][0]:om.OFF['b2'][0] + 128] = 0.0
    assert rejected(om.gradient(t2, x, y, bf16=True))
    # gradient with the layer-3 mask dropped
    z, (xp, a1, h1, a2, h2, a3, h3, P) = om.forward(theta, x, bf16=True)
    dz = (1 / (1 + np.exp(-z)) - y) / n
    d3 = om.bf16_round(np.outer(dz, P['w4']))
    g2 = g.copy()
    o, s = om.OFF['W3']
    g2[o:o + s] = (d3.T @ h2).ravel()
    assert rejected(g2)


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


@pytest.mark.gpu
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


@pytest.mark.gpu
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


@pytest.mark.gpu
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


@pytest.mark.gpu
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


@pytest.mark.gpu
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


@pytest.mark.gpu
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


@pytest.mark.gpu
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


def _family_snapshots(ctx, torch, t_snap, want, xs, ts, seed):
    """`want` snapshot features at t_snap of trajectories still undecided
    there, labelled by their verdicts (full runs), over every instance."""
    feats, labels, got, begin = [], [], 0, 0
    while got < want:
        o = ctx.simulate_snapshot('mixed', seed=seed, traj_begin=begin, n_traj=4096, t_snap=t_snap)
        f = ctx.snapshot_features(o['x_snap'], t_snap, xs, ts)
        alive = (o['snap'] == 0).reshape(-1)
        feats.append(f[alive])
        labels.append(o['verdict'].reshape(-1)[alive].to(torch.float32))
        got += int(alive.sum().item())
        begin += 4096
    return torch.cat(feats)[:want].contiguous(), torch.cat(labels)[:want].contiguous(), begin


@pytest.mark.gpu
def test_control_variate_lotka_volterra_family(env):
    # The surrogate workload as configured: the Lotka-Volterra family (rates
    # times log-uniform factors in [0.7, 1.3]), G[0,30](X>0 & Y>0), a network
    # trained on 2M prefixes at t_c = 5 labelled by their verdicts, 95% Wilson
    # half-width 0.002.  On held-out instances the control-variate estimate
    # must agree with a plain estimate of 10^6 trajectories within its own
    # error (unbiased for any network); the plain iterative estimate to the
    # same half-width runs beside it and the gain is reported, whatever it is.
    torch, smc = env
    fam, p = workloads.lotka_volterra_family(512, seed=1)
    test, _ = workloads.lotka_volterra_family(2, seed=2)
    t_c, xs, ts = 5.0, np.array([1000.0, 1000.0], np.float32), 30.0
    ref = np.log(np.asarray(fam.rates, np.float64)).mean(axis=0)
    with smc.Context(0) as ctx:
        ctx.load_model(fam)
        ctx.load_property(p)
        ctx.set_features(log_rate_ref=ref)
        x, y, used = _family_snapshots(ctx, torch, t_c, 2_000_000, xs, ts, seed=11)
        torch.cuda.synchronize()
        assert x.shape == (2_000_000, 6) and 0.0 < float(y.mean()) < 1.0
        net = smc.Mlp(6, seed=7)
        loss = net.train(x, y, epochs=4, batch=8192, lr=1e-3, seed=3)
        assert loss[-1] < loss[0], loss
    for i in range(test.n_inst):
        with smc.Context(0) as ctx:
            ctx.load_model(test.instance(i))
            ctx.load_property(p)
            ctx.set_features(log_rate_ref=ref)
            beta, resid, calib = _held_out_beta(ctx, net, t_c, xs, ts, 40 + i)
            cv = ctx.estimate_cv(net, 0.95, 0.002, seed=50 + i, precision='mixed', t_snap=t_c, x_scale=xs,
                                 t_scale=ts, beta=beta, pilot=2000)
            plain = ctx.estimate(0.95, 0.002, seed=60 + i, precision='mixed', sampling='iterative')[0]
            big = ctx.estimate(0.95, 0.002, seed=70 + i, precision='plain', sampling='fixed', fixed_n=1_000_000)[0]
        sd_big = math.sqrt(max(big['p_hat'] * (1 - big['p_hat']), 1e-12) / big['n'])
        assert abs(cv['p_hat'] - big['p_hat']) <= 4 * math.sqrt(cv['var']) + 4 * sd_big, (cv, big)
        assert cv['hi'] - cv['lo'] <= 2 * 0.002 * 1.01, cv
        plain_events = plain['events']
        cv_events = cv['events_full'] + cv['events_prefix']
        print(f'instance {i}: p(10^6) {big["p_hat"]:.5f}, cv {cv["p_hat"]:.5f} (n_eff {cv["n_eff"]:.0f}, '
              f'full {cv["n_full"]}, prefix {cv["n_prefix"]}), plain {plain["p_hat"]:.5f} (n {plain["n"]}); '
              f'residual variance share {resid:.3f}, calibration {calib:.4f}, '
              f'events cv / plain {cv_events / plain_events:.3f}')
