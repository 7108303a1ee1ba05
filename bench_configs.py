"""The other measured workloads of bench.py (``--config``), one JSON line each.

* immigration_death: 0 -> A (10), A -> 0 (0.1 A), F[0,100](A >= 130), 10,000
  trajectories per step, FP64 path, Wilson 95%; exact P = 0.0912186.
* random_networks: 4096 random mass-action networks (S in 2..32, R in 4..64)
  x 10,000 trajectories, F[0,50](X_k >= theta), one graph-captured estimate
  per step, mixed path.
* surrogate: Lotka-Volterra family (rates x log-uniform [0.7, 1.3]),
  G[0,30](X>0 & Y>0): for each checkpoint t_c in {0.5, 1, 2, 5}, 1,000,000
  snapshots at t_c of trajectories still undecided there, labelled by their
  verdicts, train the BF16 network; then reach a 95% Wilson half-width of
  0.002 on held-out instances with the plain estimator (Fig. 2, FP64 and
  mixed) and with the control-variate estimator; value = effective verified
  trajectories per second of the latter at the best t_c.  The same on a
  linear birth-death survival problem, where the checkpoint pays.
* cascade: three-tier phosphorylation cascade, 256 rate-perturbed instances,
  literal and variant properties, mixed path.
* surrogate_inference: the control variate's network (6 -> 128 x 3 -> 1,
  BF16, FP32 accumulation) on 6,000,000 rows of Lotka-Volterra-family
  features (x / x_scale, t_c / t_scale, centred log rates: 6 per row), one
  tcgen05 launch per step; rows/s and TFLOP/s against the measured BF16
  peak.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

import bench


def _line(metric_value, unit, steps, warmup, ms, dtype, workload, extra):
    line = {'metric': bench.METRIC, 'value': metric_value, 'unit': unit, 'n_gpus': 1, 'steps': steps,
            'warmup': warmup, 'ms_per_step': ms, 'higher_is_better': True, 'scaling': 'weak',
            'vs_baseline': None, 'dtype': dtype, 'data': 'synthetic', 'config': {'workload': workload}}
    line.update(extra)
    print(json.dumps(line), flush=True)


def _issue_roofline(events_per_s, ops_per_event, kernel):
    pk, src = bench.peaks()
    f = float(pk.get('sm_max_mhz', 2070.0)) * 1e6
    import torch
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    peak = n_sm * 4 * 32 * f
    ach = events_per_s * ops_per_event
    return {'bound': 'alu', 'kernel': kernel, 'achieved': ach / 1e9, 'peak': peak / 1e9, 'unit': 'Gop/s',
            'frac': ach / peak, 'traffic': None, 'ops_per_event': ops_per_event,
            'peak_source': f'{n_sm} SMs x 4 x 32 lanes x {f / 1e6:.0f} MHz ({src})'}


def _timed_simulate(ctx, precision, n, steps, warmup, seed=0, confidence=0.95, label='steps', warm_n=None):
    """Device time per step of `steps` simulate calls of n trajectories per
    instance, after `warmup` calls of warm_n (default n) trajectories."""
    import torch
    dev = torch.device('cuda', 0)
    stream = torch.cuda.Stream(dev)
    counts = torch.zeros((ctx.n_inst, 4), dtype=torch.int64, device=dev)
    wil = torch.zeros((ctx.n_inst, 3), dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            ctx.simulate(precision, seed=seed, traj_begin=0, n_traj=warm_n or n, confidence=confidence,
                         outputs=(), counts=counts, wilson=wil, stream=stream)
    torch.cuda.synchronize()
    counts.zero_()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    clocks = bench.Clocks(0)
    clocks.start()
    bench.nvtx_push(f'{label}_{precision}_steps')
    with torch.cuda.stream(stream):
        for s in range(steps):
            ev[s][0].record(stream)
            ctx.simulate(precision, seed=seed, traj_begin=0, n_traj=n, confidence=confidence, outputs=(),
                         counts=counts, wilson=wil, stream=stream)
            ev[s][1].record(stream)
    bench.nvtx_pop()
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    return ms, counts.cpu().numpy() // steps, wil.cpu().numpy(), clk


def immigration_death(args):
    import oracle
    import paper_0912_2551_gb300 as smc
    import workloads
    m, p = workloads.immigration_death()
    n = 10000
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        ms, c, wil, clk = _timed_simulate(ctx, 'plain', n, args.steps, args.warmup, seed=0)
        kname = bench.kernel_name(ctx, 'plain')
        it = ctx.estimate(0.95, 0.005, seed=0, precision='plain', sampling='iterative')[0]
        t0 = time.perf_counter()
        ex = ctx.cme_reach(cap=1000)  # the exact side of Fig. 4 (uniformisation on the GPU)
        t_ex = time.perf_counter() - t0
    t0 = time.perf_counter()
    r = oracle.run(m, p, seed=0, n_traj=n)
    cpu = time.perf_counter() - t0
    ev = float(c[0, 2])
    _line(n / (ms / 1e3), 'trajectories/s', args.steps, args.warmup, ms, 'f64',
          'immigration-death, F[0,100](A>=130), 10,000 trajectories, Philox seed 0, Wilson 95%',
          {'events_per_s': ev / (ms / 1e3), 'clocks': clk,
           'exact_uniformisation': {'p': ex['p'], 'n_states': ex['n_states'], 'iterations': ex['iterations'],
                                    'truncated': ex['truncated'], 'seconds': t_ex},
           'result': {'p_hat': wil[0, 0], 'lo': wil[0, 1], 'hi': wil[0, 2], 'exact': 0.0912186,
                      'oracle_p_hat': float(r['verdict'].mean()),
                      'iterative_eps_0.005': {'n': it['launched'], 'p_hat': it['p_hat'], 'lo': it['lo'],
                                              'hi': it['hi']}},
           'roofline': _issue_roofline(ev / (ms / 1e3), bench.algorithmic_ops_per_event(m, 1, True), kname),
           'cpu_baseline': {'value': n / cpu, 'unit': 'trajectories/s', 'cores': os.cpu_count(),
                            'kind': 'oracle', 'sample': f'the full {n} trajectories, {cpu:.2f} s'}})


def random_networks(args):
    import oracle
    import paper_0912_2551_gb300 as smc
    import workloads
    b = workloads.random_networks(4096, seed=3)
    n = args.traj or 10000
    steps = max(1, min(args.steps, 3))
    with smc.Context(0) as ctx:
        ctx.load_batch(b)
        ctx.load_property(b.properties)
        ctx.estimate(0.95, 0.01, seed=99, precision='mixed', sampling='fixed', fixed_n=500)  # tune + warm
        clocks = bench.Clocks(0)
        clocks.start()
        t0 = time.perf_counter()
        tot = None
        bench.nvtx_push('batch_mixed_steps')
        for s in range(steps):
            res = ctx.estimate(0.95, 0.01, seed=1 + s, precision='mixed', sampling='fixed', fixed_n=n)
            ev = sum(r['events'] for r in res)
            tot = ev if tot is None else tot + ev
        bench.nvtx_pop()
        dt = (time.perf_counter() - t0) / steps
        clk = clocks.stop()
        ev_step = tot / steps
        shapes = ctx.launch_shapes('mixed')
    # oracle on a bounded sample: 2 trajectories of every 16th instance
    t0 = time.perf_counter()
    k = 0
    for i in range(0, 4096, 16):
        oracle.run(b.models[i], b.properties[i], seed=1, instance=i, n_traj=2)
        k += 2
    cpu = time.perf_counter() - t0
    R = np.array([mm.n_reactions for mm in b.models])
    ops = 40 + 4 + 1 + 2 + float(np.mean(R + 1)) + 2.5 + 3 * 6 + 2 + 2
    _line(4096 * n / dt, 'trajectories/s', steps, 1, 1e3 * dt, 'mixed (f32 propensities, f64 clock)',
          f'4096 random mass-action networks (S 2..32, R 4..64) x {n:,} trajectories, F[0,50](X_k>=theta), '
          'one graph-captured estimate per step',
          {'events_per_s': ev_step / dt, 'events_per_trajectory': ev_step / (4096 * n), 'clocks': clk,
           'roofline': _issue_roofline(ev_step / dt, ops, 'ssa_kernel<mixed>'),
           'note': 'host-timed smc_estimate (graph launch, ranges up, counts down); at 10,000 trajectories '
                   'per instance (6.2e10 events per step) the heaviest networks\' trajectories (up to ~8e5 '
                   'events each) add about 0.7 s of tail; the marginal rate from 1e4 to 2e4 per instance '
                   'is higher',
           'launch': shapes,
           'cpu_baseline': {'value': k / cpu, 'unit': 'trajectories/s', 'cores': os.cpu_count(),
                            'kind': 'oracle', 'sample': f'2 trajectories of every 16th instance, {cpu:.1f} s'}})


def nested(args):
    """A formula nested beyond the monitor's units on the trace monitor:
    immigration-death, G[0,20](A >= 80 -> F[0,3] G[0,1] A >= 75) (depth 4),
    10^5 trajectories per step, FP64 and mixed paths; the same formula's
    oracle on a 2,000-trajectory sample."""
    import oracle
    import paper_0912_2551_gb300 as smc
    import workloads
    m, _ = workloads.immigration_death()
    sp = ['A']
    atoms = [workloads.atom(sp, 'A', '>=', 80), workloads.atom(sp, 'A', '>=', 75)]
    A = lambda k: ('atom', k)  # noqa: E731
    p = workloads.Property(atoms, ('G', 0.0, 20.0, ('implies', A(0), ('F', 0.0, 3.0, ('G', 0.0, 1.0, A(1))))))
    n = args.traj or 100000
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        assert ctx.monitor_kind == 'trace'
        if args.trace_cap:
            ctx.set_option('trace_cap', args.trace_cap)
        ms, c, wil, clk = _timed_simulate(ctx, 'plain', n, args.steps, args.warmup, seed=0, label='nested')
        ms_m, c_m, _, clk_m = _timed_simulate(ctx, 'mixed', n, args.steps, args.warmup, seed=0, label='nested')
        kname = bench.kernel_name(ctx, 'plain')
    k = 2000
    r, cpu = None, None
    if not args.no_cpu_baseline:
        t0 = time.perf_counter()
        r = oracle.run(m, p, seed=0, n_traj=k)
        cpu = time.perf_counter() - t0
    ev = float(c[0, 2])
    _line(n / (ms / 1e3), 'trajectories/s', args.steps, args.warmup, ms, 'f64',
          'immigration-death, G[0,20](A>=80 -> F[0,3] G[0,1] A>=75) on the trace monitor, '
          f'{n:,} trajectories per step',
          {'events_per_s': ev / (ms / 1e3), 'events_per_trajectory': ev / n, 'clocks': clk,
           'mixed': {'value': n / (ms_m / 1e3), 'ms_per_step': ms_m, 'events_per_s': float(c_m[0, 2]) / (ms_m / 1e3),
                     'clocks': clk_m},
           'result': {'p_hat': wil[0, 0], 'lo': wil[0, 1], 'hi': wil[0, 2],
                      'oracle_p_hat_2000': float(r['verdict'].mean()) if r else None},
           'roofline': _issue_roofline(ev / (ms / 1e3), bench.algorithmic_ops_per_event(m, 2, True), kname),
           'note': 'the issue roofline counts the SSA\'s work per event only; the trace monitor adds the '
                   'recording and its checks',
           'cpu_baseline': None if r is None else
           {'value': k / cpu, 'unit': 'trajectories/s', 'cores': os.cpu_count(),
            'kind': 'oracle', 'sample': f'{k} trajectories, {cpu:.2f} s'}})


def _collect_snapshots(ctx, torch, t_c, want, per_call, x_scale, t_scale, seed):
    """Snapshots at t_c of trajectories still undecided there, labelled by
    their verdicts (full runs)."""
    xs, ys = [], []
    got, begin = 0, 0
    while got < want:
        o = ctx.simulate_snapshot('mixed', seed=seed, traj_begin=begin, n_traj=per_call, t_snap=t_c)
        f = ctx.snapshot_features(o['x_snap'], t_c, x_scale, t_scale)
        alive = (o['snap'] == 0).reshape(-1)
        xs.append(f[alive])
        ys.append(o['verdict'].reshape(-1)[alive].to(torch.float32))
        got += int(alive.sum().item())
        begin += per_call
    x = torch.cat(xs)[:want].contiguous()
    y = torch.cat(ys)[:want].contiguous()
    return x, y, begin


def _held_out(ctx, net, t_c, x_scale, t_scale, seed, n):
    """On held-out trajectories: beta = Cov(Y, G) / Var(G), the share of
    Var(Y) that beta G leaves, and r = the events a prefix run to t_c costs
    as a share of a full run's (both measured on the same full runs)."""
    o = ctx.simulate_snapshot('mixed', seed=seed, traj_begin=0, n_traj=n, t_snap=t_c)
    g = net.predict(ctx.snapshot_features(o['x_snap'], t_c, x_scale, t_scale)).cpu().numpy()
    y = o['verdict'].reshape(-1).cpu().numpy().astype(float)
    dec = o['snap'].reshape(-1).cpu().numpy() == 1
    G = np.where(dec, y, g)
    beta = float(np.cov(y, G)[0, 1] / max(np.var(G, ddof=1), 1e-300))
    resid = float(np.var(y - beta * G) / max(np.var(y), 1e-300))
    r = float(o['e_snap'].double().sum().item() / o['counts'][:, 2].double().sum().item())
    return beta, resid, r, float((~dec).mean())


def _predicted_cost_ratio(resid, r):
    """Cost of the two-phase control variate over the plain estimator's for
    the same variance, at the optimal split: (sqrt(resid (1-r)) +
    sqrt((1-resid) r))^2 when r < 1 - resid, else 1 (no prefix runs)."""
    rho2 = 1.0 - resid
    if r >= rho2:
        return 1.0
    return (math.sqrt(resid * (1 - r)) + math.sqrt(rho2 * r)) ** 2


def _three_arms(smc, torch, inst, prop, net, t_c, x_scale, t_scale, beta, conf, eps, seed, ref=None):
    """One held-out instance to the same Wilson half-width three ways: plain
    FP64 (Fig. 2), plain mixed (Fig. 2), and mixed + control variate (rate
    features centred on the family's reference `ref`, when given)."""
    out = {}
    with smc.Context(0) as ctx:
        ctx.load_model(inst)
        ctx.load_property(prop)
        if ref is not None:
            ctx.set_features(log_rate_ref=ref)
        for prec in ('plain', 'mixed'):
            ctx.estimate(conf, eps, seed=seed + 500, precision=prec, sampling='fixed', fixed_n=1000)  # warm
        torch.cuda.synchronize()
        for prec in ('plain', 'mixed'):
            t0 = time.perf_counter()
            r = ctx.estimate(conf, eps, seed=seed, precision=prec, sampling='iterative')[0]
            out[prec] = dict(s=time.perf_counter() - t0, n=r['launched'], events=r['events'], p=r['p_hat'],
                             half=(r['hi'] - r['lo']) / 2)
        ctx.estimate_cv(net, conf, eps, seed=seed + 2, precision='mixed', t_snap=t_c, x_scale=x_scale,
                        t_scale=t_scale, beta=beta, pilot=1000)  # warm (buffers, tuned shapes)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        cv = ctx.estimate_cv(net, conf, eps, seed=seed + 1, precision='mixed', t_snap=t_c, x_scale=x_scale,
                             t_scale=t_scale, beta=beta, pilot=1000)
        out['cv'] = dict(s=time.perf_counter() - t0, n_eff=cv['n_eff'], n_full=cv['n_full'],
                         n_prefix=cv['n_prefix'], events=cv['events_full'] + cv['events_prefix'],
                         p=cv['p_hat'], half=(cv['hi'] - cv['lo']) / 2)
    return out


MLP_FLOPS_PER_ROW = 3 * 2 * (16 * 128 + 2 * 128 * 128 + 128)  # forward + 2x backward per training row


def _train(ctx, smc, torch, t_c, n_snap, x_scale, t_scale, seed):
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    x, y, used = _collect_snapshots(ctx, torch, t_c, n_snap, 4096, x_scale, t_scale, seed)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = smc.Mlp(x.shape[1], seed=7)
    epochs, batch = 4, 8192
    t1 = time.perf_counter()
    loss = net.train(x, y, epochs=epochs, batch=batch, lr=1e-3, seed=3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    steps = epochs * math.ceil(x.shape[0] / batch)
    flops = steps * batch * MLP_FLOPS_PER_ROW
    return net, dict(snapshots=int(x.shape[0]), trajectories_simulated=int(used * ctx.n_inst), data_seconds=t_data,
                     train_seconds=t_train, epochs=epochs, batch=batch, loss=[float(v) for v in loss],
                     tflops=flops / t_train / 1e12, step_kernels=_train_rate(smc, torch, x, y))


def _train_rate(smc, torch, x, y):
    """The training step's device throughput (step kernel + Adam update,
    CUDA events on the stream the steps run on) on the same rows, per batch
    size: two epochs after one warm-up epoch, on a separate network."""
    out = {}
    for batch in (8192, 65536, 262144):
        net = smc.Mlp(x.shape[1], seed=5)
        net.train(x, y, epochs=1, batch=batch, lr=1e-3, seed=1)
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        net.train(x, y, epochs=2, batch=batch, lr=1e-3, seed=2)
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        steps = 2 * math.ceil(x.shape[0] / batch)
        out[str(batch)] = dict(us_per_step=1e3 * ms / steps, tflops=steps * batch * MLP_FLOPS_PER_ROW / (ms * 1e-3) / 1e12)
        net.close()
    return out


def surrogate(args):
    """Control variate on the Lotka-Volterra family (the configured
    workload): a sweep over the checkpoint t_c, each point training its own
    network on 2M prefixes still undecided at t_c; then the same estimator
    on a linear birth-death survival problem, where a checkpoint settles the
    verdict early."""
    import torch
    import paper_0912_2551_gb300 as smc
    import workloads
    eps, conf = 0.002, 0.95
    x_scale, t_scale = np.array([1000.0, 1000.0], np.float32), 30.0
    fam, p = workloads.lotka_volterra_family(512, seed=1)
    test, _ = workloads.lotka_volterra_family(4, seed=2)
    ref = np.log(np.asarray(fam.rates, np.float64)).mean(axis=0)  # the family's log-rate centre
    sweep = []
    for t_c in (0.5, 1.0, 2.0, 5.0):
        with smc.Context(0) as ctx:
            ctx.load_model(fam)
            ctx.load_property(p)
            ctx.set_features(log_rate_ref=ref)
            net, tr = _train(ctx, smc, torch, t_c, 2_000_000, x_scale, t_scale, seed=11)
            beta, resid, r, alive = _held_out(ctx, net, t_c, x_scale, t_scale, seed=12, n=256)
        rows = [_three_arms(smc, torch, test.instance(i), p, net, t_c, x_scale, t_scale, beta, conf, eps,
                            1000 + 10 * i, ref) for i in range(test.n_inst)]
        T = {k: sum(rw[k]['s'] for rw in rows) for k in ('plain', 'mixed', 'cv')}
        E = {k: sum(rw[k]['events'] for rw in rows) for k in ('plain', 'mixed', 'cv')}
        sweep.append(dict(t_c=t_c, alive_share=alive, prefix_cost_share=r, residual_variance_share=resid,
                          beta=beta, predicted_cost_ratio=_predicted_cost_ratio(resid, r),
                          measured_event_ratio_cv_over_plain=E['cv'] / E['mixed'],
                          wall_s=T, n_eff=sum(rw['cv']['n_eff'] for rw in rows),
                          n_prefix=sum(rw['cv']['n_prefix'] for rw in rows),
                          n_plain=sum(rw['mixed']['n'] for rw in rows), training=tr, per_instance=rows))
    best = min(sweep, key=lambda d: d['wall_s']['cv'])
    # birth-death survival: G[0,20](A > 0), checkpoint t = 8
    bd, bp = workloads.birth_death_survival(1)
    bx, bt = np.array([50.0], np.float32), 20.0
    with smc.Context(0) as ctx:
        ctx.load_model(bd)
        ctx.load_property(bp)
        bnet, btr = _train(ctx, smc, torch, 8.0, 500_000, bx, bt, seed=31)
        bbeta, bresid, br, balive = _held_out(ctx, bnet, 8.0, bx, bt, seed=32, n=100000)
    brows = {h: _three_arms(smc, torch, bd, bp, bnet, 8.0, bx, bt, bbeta, conf, h, 77) for h in (eps, eps / 4)}

    def _bd(brow):
        return {'measured_event_ratio_cv_over_plain': brow['cv']['events'] / (
                    brow['cv']['n_eff'] * brow['mixed']['events'] / brow['mixed']['n']),
                'wall_time_ratio_plain_fp64_over_cv': brow['plain']['s'] / brow['cv']['s'],
                'wall_time_ratio_plain_mixed_over_cv': brow['mixed']['s'] / brow['cv']['s'], 'arms': brow}
    pk, src = bench.peaks()
    T_c = best['wall_s']['cv']
    tf = best['training']['tflops']
    tk = best['training']['step_kernels']['65536']['tflops']
    peak = float(pk.get('bf16_tflops', 1960.8))
    _line(best['n_eff'] / T_c, 'effective trajectories/s', len(best['per_instance']), 1,
          1e3 * T_c / len(best['per_instance']), 'mixed + bf16 surrogate',
          'Lotka-Volterra family (rates x log-uniform [0.7,1.3]), G[0,30](X>0 & Y>0), 95% Wilson half-width '
          '0.002, 4 held-out instances; checkpoint sweep t_c in {0.5, 1, 2, 5}',
          {'best_t_c': best['t_c'],
           'wall_time_ratio_plain_fp64_over_cv': best['wall_s']['plain'] / T_c,
           'wall_time_ratio_plain_mixed_over_cv': best['wall_s']['mixed'] / T_c,
           'sweep': sweep,
           'birth_death_survival': {
               'workload': 'A -> 2A (1.0), A -> 0 (0.8 A), A0 = 5, G[0,20](A > 0), checkpoint t = 8',
               'prefix_cost_share': br, 'residual_variance_share': bresid, 'beta': bbeta,
               'predicted_cost_ratio': _predicted_cost_ratio(bresid, br),
               'half_width_0.002': _bd(brows[eps]), 'half_width_0.0005': _bd(brows[eps / 4]),
               'training': btr},
           'roofline': {'bound': 'tensor',
                        'kernel': 'surrogate training step (fused tcgen05 step kernel + Adam update), batch 65536',
                        'achieved': tk, 'peak': peak, 'unit': 'TFLOP/s', 'frac': tk / peak, 'traffic': None,
                        'peak_source': f'cuBLAS bf16 burst ({src})',
                        'configured_training': {'batch': best['training']['batch'], 'tflops': tf,
                                                'frac': tf / peak}}})


CASCADE_FEATURES = ('KKKs', 'KKP', 'KKPP', 'KP', 'KPP', 'KP_KKPP', 'KPP_KPase')


def cascade(args):
    """The configured cascade: 256 rate-perturbed instances x 100,000
    trajectories per step in one batched launch (mixed path), for the literal
    formula and the KPP<2000 variant; the FP64 path on a 1,000-trajectory
    subsample per instance; and the variant's surrogate-assisted estimate (a
    network trained on prefixes of the batch at t_c = 30, seven counts and
    the time as its inputs) against the plain estimator on four held-out
    instances."""
    import torch
    import oracle
    import paper_0912_2551_gb300 as smc
    import workloads
    out = {}
    n = args.traj or 100_000
    steps, warm = 1, 3
    for variant in (False, True):
        m, p = workloads.mapk_cascade(256, seed=5, variant=variant)
        name = 'variant' if variant else 'literal'
        with smc.Context(0) as ctx:
            ctx.load_model(m)
            ctx.load_property(p)
            ms, c, wil, clk = _timed_simulate(ctx, 'mixed', n, steps, warm, seed=0, label=name,
                                              warm_n=max(1, n // 100))
            kname = bench.kernel_name(ctx, 'mixed')
            n64 = min(n, 1000)
            msp, cp, _, _ = _timed_simulate(ctx, 'plain', n64, 1, warm, seed=0, label=name, warm_n=max(1, n64 // 10))
        ev, evp = float(c[:, 2].sum()), float(cp[:, 2].sum())
        out[name] = dict(
            ms=ms, traj_s=256 * n / (ms / 1e3), events_per_s=ev / (ms / 1e3), events_per_traj=ev / (256 * n),
            yes=int(c[:, 0].sum()), p_per_instance_quartiles=np.percentile(c[:, 0] / np.maximum(c[:, 1], 1),
                                                                          [0, 25, 50, 75, 100]).tolist(),
            plain_fp64=dict(trajectories_per_instance=n64, ms=msp, traj_s=256 * n64 / (msp / 1e3),
                            events_per_s=evp / (msp / 1e3)),
            clocks=clk)
    # surrogate on the variant: train on prefixes at t_c, then four held-out
    # instances to the same 95% half-width (0.01) with and without it
    mv, pv = workloads.mapk_cascade(256, seed=5, variant=True)
    idx = [workloads.MAPK_SPECIES.index(s_) for s_ in CASCADE_FEATURES]
    t_c, xs, ts = 30.0, np.full(len(idx), 2000.0, np.float32), 200.0
    with smc.Context(0) as ctx:
        ctx.load_model(mv)
        ctx.load_property(pv)
        ctx.set_features(species=idx, with_rates=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        o = ctx.simulate_snapshot('mixed', seed=21, traj_begin=0, n_traj=4000, t_snap=t_c)
        feat = ctx.snapshot_features(o['x_snap'], t_c, xs, ts)
        alive = (o['snap'] == 0).reshape(-1)
        x = feat[alive].contiguous()
        y = o['verdict'].reshape(-1)[alive].to(torch.float32).contiguous()
        torch.cuda.synchronize()
        t_data = time.perf_counter() - t0
        net = smc.Mlp(len(idx) + 1, seed=5)
        t1 = time.perf_counter()
        loss = net.train(x, y, epochs=4, batch=8192, lr=1e-3, seed=6)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t1
    held = []
    for i in (1, 3, 5, 7):
        with smc.Context(0) as ctx:
            ctx.load_model(mv.instance(i))
            ctx.load_property(pv)
            ctx.set_features(species=idx, with_rates=False)
            ctx.estimate(0.95, 0.01, seed=5, precision='mixed', sampling='fixed', fixed_n=500)  # warm
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pl = ctx.estimate(0.95, 0.01, seed=60 + i, precision='mixed', sampling='iterative')[0]
            t_pl = time.perf_counter() - t0
            t0 = time.perf_counter()
            cv = ctx.estimate_cv(net, 0.95, 0.01, seed=70 + i, precision='mixed', t_snap=t_c, x_scale=xs,
                                 t_scale=ts, beta=1.0, pilot=1000)
            t_cv = time.perf_counter() - t0
        held.append(dict(instance=i, plain=dict(p=pl['p_hat'], n=pl['launched'], events=pl['events'], s=t_pl),
                         cv=dict(p=cv['p_hat'], n_eff=cv['n_eff'], n_full=cv['n_full'], n_prefix=cv['n_prefix'],
                                 events=cv['events_full'] + cv['events_prefix'], s=t_cv)))
    surrogate = dict(t_c=t_c, features=list(CASCADE_FEATURES) + ['t'], training_rows=int(x.shape[0]),
                     label_mean=float(y.mean()), loss=[float(v) for v in loss], data_seconds=t_data,
                     train_seconds=t_train, held_out=held,
                     wall_ratio_plain_over_cv=sum(h['plain']['s'] for h in held) / sum(h['cv']['s'] for h in held),
                     event_ratio_cv_over_plain=sum(h['cv']['events'] for h in held) /
                     sum(h['plain']['events'] for h in held))
    t0 = time.perf_counter()
    mo, po = workloads.mapk_cascade(4, seed=5, variant=True)
    ro = oracle.run(mo, po, seed=0, instance=0, n_traj=256)
    cpu = time.perf_counter() - t0
    lit, var = out['literal'], out['variant']
    ops = 40 + 4 + 1 + 2 + 31 + 2 + 3 * 5 + 2 * 3 + 2
    _line(lit['traj_s'], 'trajectories/s', steps, warm, lit['ms'],
          'mixed (f32 propensities, f64 clock)',
          f'three-tier cascade, 22 species, 30 reactions, 256 rate-perturbed instances x {n:,} trajectories per '
          'step, one batched launch; (KPP<500) U[0,200] (KPP>=2000 & F[0,50] KPP<500) and the KPP<2000 variant',
          {'events_per_s': lit['events_per_s'], 'configs': out, 'surrogate_variant': surrogate,
           'warmup_trajectories_per_instance': max(1, n // 100),
           'roofline': _issue_roofline(var['events_per_s'], ops, kname),
           'cpu_baseline': {'value': 256 / cpu, 'unit': 'trajectories/s',
                            'events_per_s': float(ro['events'].sum()) / cpu, 'cores': os.cpu_count(),
                            'kind': 'oracle', 'sample': f'256 trajectories of instance 0 (variant), {cpu:.1f} s'}})


# DRAM bytes (read + write) of one launch of the inference kernel on
# 6,000,000 rows (ncu: the FP32 features read once, the outputs written
# once; the weights come from L2)
TRAFFIC_INFER = 144143872 + 13789952


def surrogate_inference(args):
    import torch
    import paper_0912_2551_gb300 as smc
    from oracle import mlp as om
    n = args.traj or 6_000_000
    n_in = 6
    dev = torch.device('cuda', 0)
    g = torch.Generator().manual_seed(0)
    # features as smc_snapshot_features scales them: counts / x_scale in
    # [0, 3), t_c / t_scale, log-rate offsets within +-ln 1.3
    x = torch.empty((n, n_in), dtype=torch.float32)
    x[:, :2] = torch.rand((n, 2), generator=g) * 3.0
    x[:, 2] = 0.5
    x[:, 3:] = (torch.rand((n, 3), generator=g) * 2.0 - 1.0) * math.log(1.3)
    xd = x.to(dev)
    net = smc.Mlp(n_in, seed=1)
    out = torch.empty((n,), dtype=torch.float32, device=dev)
    for _ in range(args.warmup):
        net.predict(xd, out=out)
    torch.cuda.synchronize()
    flush = torch.empty(256 * 2**20 // 4, dtype=torch.int32, device=dev)  # > L2 between steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = bench.Clocks(0)
    clocks.start()
    stream = torch.cuda.current_stream(dev)
    for s in range(args.steps):
        flush.fill_(s)
        ev[s][0].record(stream)
        net.predict(xd, out=out)
        ev[s][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    flop_row = 2.0 * (16 * 128 + 2 * 128 * 128 + 128)  # the padded network's multiply-adds
    tflops = n * flop_row / (ms * 1e-3) / 1e12
    pk, src = bench.peaks()
    peak = float(pk.get('bf16_tflops', 1899.0))
    # sampled rows against the FP64 oracle network (BF16 weights and inputs)
    theta = net.get_params().astype(np.float64)
    for name in ('W1', 'W2', 'W3'):
        o, sz = om.OFF[name]
        theta[o:o + sz] = om.bf16_round(theta[o:o + sz])
    idx = np.random.default_rng(0).choice(n, 4096, replace=False)
    z, _ = om.forward(theta, om.bf16_round(x[idx].numpy()))
    err = float(np.max(np.abs(out.cpu().numpy()[idx] - 1.0 / (1.0 + np.exp(-z)))))
    extra = {'tflops': tflops, 'rows': n,
             'roofline': {'bound': 'tensor', 'kernel': 'mlp_tc_forward (tcgen05, TMEM accumulators)',
                          'achieved': tflops, 'peak': peak, 'unit': 'TFLOP/s', 'frac': tflops / peak,
                          'traffic': TRAFFIC_INFER if n == 6_000_000 else None,
                          'flop_per_row': flop_row,
                          'peak_source': f'bf16_tflops ({src}: cuBLAS bf16 GEMM, burst)'},
             'oracle_max_abs_err': err, 'gpu_launches': args.steps, 'clocks': clk}
    if not args.no_cpu_baseline:
        t0 = time.perf_counter()
        m = 500_000
        om.forward(theta, om.bf16_round(x[:m].numpy()))
        dt = time.perf_counter() - t0
        extra['cpu_baseline'] = {'value': m / dt, 'unit': 'rows/s', 'cores': os.cpu_count(), 'kind': 'oracle',
                                 'sample': f'first {m} rows, FP64 NumPy (BLAS on all host cores), {dt:.1f} s'}
    _line(n / (ms * 1e-3), 'rows/s', args.steps, args.warmup, ms, 'bf16 (fp32 accumulate)',
          f'surrogate network 6 -> 128 x 3 -> 1 on {n:,} rows of Lotka-Volterra-family features', extra)


def surrogate_training(args):
    """The surrogate's training step alone (fused tcgen05 step kernel + Adam
    update, replayed as CUDA graphs): one step of this line is one epoch of
    minibatches of 65,536 rows over 8,388,608 synthetic feature rows (6
    inputs: two counts / 1000 in [0, 3), the time, three log-rate offsets;
    logistic targets), 201 MB of inputs (> L2, no flush needed); the other
    batch sizes are reported beside it."""
    import torch
    import paper_0912_2551_gb300 as smc
    from oracle import mlp as om
    n, n_in, batch = 8 * 2**20, 6, 65536
    dev = torch.device('cuda', 0)
    g = torch.Generator(device=dev).manual_seed(0)
    x = torch.rand((n, n_in), generator=g, device=dev)
    x[:, :2] *= 3.0
    x[:, 3:] = (x[:, 3:] * 2.0 - 1.0) * math.log(1.3)
    logit = 2.0 * (x[:, 0] - x[:, 1]) + 0.5 * x[:, 2] + x[:, 3]
    y = (torch.rand(n, generator=g, device=dev) < torch.sigmoid(logit)).float()
    steps_per_epoch = math.ceil(n / batch)
    flop = MLP_FLOPS_PER_ROW * batch * steps_per_epoch
    net = smc.Mlp(n_in, seed=1)
    stream = torch.cuda.current_stream(dev)
    for w in range(args.warmup):
        net.train(x, y, epochs=1, batch=batch, lr=1e-3, seed=100 + w)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    clocks = bench.Clocks(0)
    clocks.start()
    for k in range(args.steps):
        ev[k][0].record(stream)
        net.train(x, y, epochs=1, batch=batch, lr=1e-3, seed=k)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = sum(a.elapsed_time(b) for a, b in ev) / args.steps
    loss = float(net.train(x[:batch * 8], y[:batch * 8], epochs=1, batch=batch, lr=1e-3, seed=999)[0])
    tflops = flop / (ms * 1e-3) / 1e12
    pk, src = bench.peaks()
    peak = float(pk.get('bf16_tflops', 1960.8))
    sus = float(pk.get('bf16_tflops_sustained', 1754.4))
    others = _train_rate(smc, torch, x[:2**21], y[:2**21])
    extra = {'batch': batch, 'steps_per_epoch': steps_per_epoch, 'tflops': tflops, 'loss_after': loss,
             'batch_sizes': others,
             'roofline': {'bound': 'tensor', 'kernel': 'mlp_train_step_kernel (tcgen05, TMEM) + mlp_update_kernel',
                          'achieved': tflops, 'peak': peak, 'unit': 'TFLOP/s', 'frac': tflops / peak,
                          'frac_of_sustained': tflops / sus, 'traffic': None,
                          'flop_per_row': MLP_FLOPS_PER_ROW,
                          'peak_source': f'bf16_tflops ({src}: cuBLAS bf16 GEMM, burst); sustained {sus}'},
             'gpu_launches': 2 * steps_per_epoch * args.steps, 'clocks': clk}
    if not args.no_cpu_baseline:
        theta = net.get_params().astype(np.float64)
        xs, ys = x[:4096].cpu().numpy().astype(np.float64), y[:4096].cpu().numpy().astype(np.float64)
        t0 = time.perf_counter()
        reps = 0
        while time.perf_counter() - t0 < 10.0:
            om.gradient(theta, xs, ys, bf16=True)
            reps += 1
        dt = time.perf_counter() - t0
        extra['cpu_baseline'] = {'value': reps * 4096 / dt, 'unit': 'training rows/s', 'cores': os.cpu_count(),
                                 'kind': 'oracle',
                                 'sample': f'{reps} gradients of 4096 rows (oracle/mlp.py, FP64 NumPy), {dt:.1f} s'}
    _line(n / (ms * 1e-3), 'training rows/s', args.steps, args.warmup, ms, 'bf16 (fp32 accumulate)',
          f'surrogate network 6 -> 128 x 3 -> 1, Adam, minibatch {batch:,}, one epoch over {n:,} rows', extra)


def _time_batch(smc, b, precision, selection, n, seed=1):
    """Host time of one fixed-size smc_estimate over batch b (after a
    tuning/warm-up estimate) with the given selection mode; events."""
    import torch
    with smc.Context(0) as ctx:
        ctx.set_option('selection', selection)
        ctx.load_batch(b)
        ctx.load_property(b.properties)
        ctx.estimate(0.95, 0.01, seed=99, precision=precision, sampling='fixed', fixed_n=max(1, n // 20))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = ctx.estimate(0.95, 0.01, seed=seed, precision=precision, sampling='fixed', fixed_n=n)
        dt = time.perf_counter() - t0
    return dt, float(sum(r['events'] for r in res))


def large_networks(args):
    """Reaction selection for large networks (65 to 255 reactions): the
    batch of random_networks_large timed with the linear scan and with the
    checkpointed running sums, both precisions; then the crossover, batches
    of 64 networks with exactly R reactions for R from 24 to 255."""
    import oracle
    import paper_0912_2551_gb300 as smc
    import workloads
    b = workloads.random_networks_large(256, seed=8)
    n = args.traj or 2000
    main = {}
    for prec in ('mixed', 'plain'):
        for sel, name in ((1, 'linear'), (2, 'checkpoints')):
            dt, ev = _time_batch(smc, b, prec, sel, n)
            main[f'{prec}_{name}'] = dict(s=dt, traj_s=256 * n / dt, events_per_s=ev / dt)
    sweep = []
    for R in (24, 48, 96, 160, 255):
        bb = workloads.random_networks(64, seed=20 + R, s_range=(16, 48), r_range=(R, R), theta_above_start=True)
        row = dict(R=R)
        for prec in ('mixed', 'plain'):
            for sel, name in ((1, 'linear'), (2, 'checkpoints')):
                dt, ev = _time_batch(smc, bb, prec, sel, 1000)
                row[f'{prec}_{name}_events_per_s'] = ev / dt
            row[f'{prec}_speedup'] = row[f'{prec}_checkpoints_events_per_s'] / row[f'{prec}_linear_events_per_s']
        sweep.append(row)
    t0 = time.perf_counter()
    k = 0
    for i in range(0, 256, 32):
        oracle.run(b.models[i], b.properties[i], seed=1, instance=i, n_traj=8)
        k += 8
    cpu = time.perf_counter() - t0
    best = main['mixed_checkpoints']
    R = np.array([mm.n_reactions for mm in b.models])
    ops = 40 + 4 + 1 + 2 + 2 * (SEL_BLOCK_SCAN + float(np.mean((R + 15) // 16))) + 2.5 + 3 * 8 + 2 + 2
    _line(best['traj_s'], 'trajectories/s', 1, 1, 1e3 * best['s'], 'mixed (f32 propensities, f64 clock)',
          f'256 random mass-action networks (S 16..64, R 65..255) x {n:,} trajectories, F[0,50](X_k>=theta), '
          'selection by running sums checkpointed every 16 reactions vs the linear scan',
          {'events_per_s': best['events_per_s'], 'arms': main, 'crossover': sweep,
           'roofline': _issue_roofline(best['events_per_s'], ops, 'ssa_kernel<mixed>'),
           'cpu_baseline': {'value': k / cpu, 'unit': 'trajectories/s', 'cores': os.cpu_count(),
                            'kind': 'oracle', 'sample': f'8 trajectories of every 32nd instance, {cpu:.1f} s'}})


SEL_BLOCK_SCAN = 8  # expected running sums formed inside the selected block


def run(args):
    {'immigration_death': immigration_death, 'random_networks': random_networks, 'surrogate': surrogate,
     'cascade': cascade, 'surrogate_inference': surrogate_inference, 'surrogate_training': surrogate_training,
     'nested': nested,
     'large_networks': large_networks}[args.config](args)
