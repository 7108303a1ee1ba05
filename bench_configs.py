"""The other measured workloads of bench.py (``--config``), one JSON line each.

* immigration_death: 0 -> A (10), A -> 0 (0.1 A), F[0,100](A >= 130), 10,000
  trajectories per step, FP64 path, Wilson 95%; exact P = 0.0912186.
* random_networks: 4096 random mass-action networks (S in 2..32, R in 4..64)
  x 10,000 trajectories, F[0,50](X_k >= theta), one graph-captured estimate
  per step, mixed path.
* surrogate: Lotka-Volterra family (rates x log-uniform [0.7, 1.3]),
  G[0,30](X>0 & Y>0): 2,000,000 snapshots at t_c = 5 of trajectories still
  undecided there, labelled by their verdicts, train the BF16 network, then
  reach a 95% Wilson half-width of 0.002 on held-out instances with the
  plain estimator (Fig. 2) and with the control-variate estimator; value =
  effective verified trajectories per second of the latter.
* cascade: three-tier phosphorylation cascade, 256 rate-perturbed instances,
  literal and variant properties, mixed path.
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


def _timed_simulate(ctx, precision, n, steps, warmup, seed=0, confidence=0.95):
    import torch
    dev = torch.device('cuda', 0)
    stream = torch.cuda.Stream(dev)
    counts = torch.zeros((ctx.n_inst, 4), dtype=torch.int64, device=dev)
    wil = torch.zeros((ctx.n_inst, 3), dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            ctx.simulate(precision, seed=seed, traj_begin=0, n_traj=n, confidence=confidence, outputs=(),
                         counts=counts, wilson=wil, stream=stream)
    torch.cuda.synchronize()
    counts.zero_()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    clocks = bench.Clocks(0)
    clocks.start()
    with torch.cuda.stream(stream):
        for s in range(steps):
            ev[s][0].record(stream)
            ctx.simulate(precision, seed=seed, traj_begin=0, n_traj=n, confidence=confidence, outputs=(),
                         counts=counts, wilson=wil, stream=stream)
            ev[s][1].record(stream)
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
        it = ctx.estimate(0.95, 0.005, seed=0, precision='plain', sampling='iterative')[0]
    t0 = time.perf_counter()
    r = oracle.run(m, p, seed=0, n_traj=n)
    cpu = time.perf_counter() - t0
    ev = float(c[0, 2])
    _line(n / (ms / 1e3), 'trajectories/s', args.steps, args.warmup, ms, 'f64',
          'immigration-death, F[0,100](A>=130), 10,000 trajectories, Philox seed 0, Wilson 95%',
          {'events_per_s': ev / (ms / 1e3), 'clocks': clk,
           'result': {'p_hat': wil[0, 0], 'lo': wil[0, 1], 'hi': wil[0, 2], 'exact': 0.0912186,
                      'oracle_p_hat': float(r['verdict'].mean()),
                      'iterative_eps_0.005': {'n': it['launched'], 'p_hat': it['p_hat'], 'lo': it['lo'],
                                              'hi': it['hi']}},
           'roofline': _issue_roofline(ev / (ms / 1e3), bench.algorithmic_ops_per_event(m, 1, True),
                                       'ssa_kernel<plain FP64>'),
           'cpu_baseline': {'value': n / cpu, 'unit': 'trajectories/s', 'cores': os.cpu_count(),
                            'kind': 'oracle', 'sample': f'the full {n} trajectories, {cpu:.2f} s'}})


def random_networks(args):
    import oracle
    import paper_0912_2551_gb300 as smc
    import workloads
    b = workloads.random_networks(4096, seed=3)
    n = 10000
    steps = max(1, min(args.steps, 3))
    with smc.Context(0) as ctx:
        ctx.load_batch(b)
        ctx.load_property(b.properties)
        ctx.estimate(0.95, 0.01, seed=99, precision='mixed', sampling='fixed', fixed_n=500)  # tune + warm
        clocks = bench.Clocks(0)
        clocks.start()
        t0 = time.perf_counter()
        tot = None
        for s in range(steps):
            res = ctx.estimate(0.95, 0.01, seed=1 + s, precision='mixed', sampling='fixed', fixed_n=n)
            ev = sum(r['events'] for r in res)
            tot = ev if tot is None else tot + ev
        dt = (time.perf_counter() - t0) / steps
        clk = clocks.stop()
        ev_step = tot / steps
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
          '4096 random mass-action networks (S 2..32, R 4..64) x 10,000 trajectories, F[0,50](X_k>=theta), '
          'one graph-captured estimate per step',
          {'events_per_s': ev_step / dt, 'events_per_trajectory': ev_step / (4096 * n), 'clocks': clk,
           'roofline': _issue_roofline(ev_step / dt, ops, 'ssa_kernel<mixed>'),
           'note': 'host-timed smc_estimate (graph launch, ranges up, counts down); tail-bound: the '
                   'longest trajectories reach ~8e5 events',
           'cpu_baseline': {'value': k / cpu, 'unit': 'trajectories/s', 'cores': os.cpu_count(),
                            'kind': 'oracle', 'sample': f'2 trajectories of every 16th instance, {cpu:.1f} s'}})


def _collect_snapshots(ctx, smc, torch, t_c, want, per_call, x_scale, t_scale, seed):
    """Snapshots at t_c of trajectories still undecided there, with verdicts."""
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


def surrogate(args):
    import torch
    import paper_0912_2551_gb300 as smc
    import workloads
    t_c, eps, conf = 5.0, 0.002, 0.95
    x_scale, t_scale = np.array([1000.0, 1000.0], np.float32), 30.0
    fam, p = workloads.lotka_volterra_family(512, seed=1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with smc.Context(0) as ctx:
        ctx.load_model(fam)
        ctx.load_property(p)
        x, y, used = _collect_snapshots(ctx, smc, torch, t_c, 2_000_000, 4096, x_scale, t_scale, seed=11)
        torch.cuda.synchronize()
        t_data = time.perf_counter() - t0
        net = smc.Mlp(x.shape[1], seed=7)
        epochs, batch = 4, 8192
        t1 = time.perf_counter()
        loss = net.train(x, y, epochs=epochs, batch=batch, lr=1e-3, seed=3)
        torch.cuda.synchronize()
        t_train = time.perf_counter() - t1
        steps = epochs * math.ceil(x.shape[0] / batch)
        flops = steps * batch * 3 * 2 * (16 * 128 + 2 * 128 * 128 + 128)  # forward + 2x backward
        # beta from held-out trajectories of the family (another seed)
        h = ctx.simulate_snapshot('mixed', seed=12, traj_begin=0, n_traj=256, t_snap=t_c)
        gh = net.predict(ctx.snapshot_features(h['x_snap'], t_c, x_scale, t_scale)).cpu().numpy()
        yh = h['verdict'].reshape(-1).cpu().numpy().astype(float)
        dec = h['snap'].reshape(-1).cpu().numpy() == 1
        G = np.where(dec, yh, gh)
        beta = float(np.cov(yh, G)[0, 1] / np.var(G, ddof=1))
        resid = float(np.var(yh - beta * G) / np.var(yh))
    # held-out instances: plain Fig. 2 vs control variate, same target width
    test, _ = workloads.lotka_volterra_family(8, seed=2)
    rows = []
    for i in range(test.n_inst):
        inst = test.instance(i)
        with smc.Context(0) as ctx:
            ctx.load_model(inst)
            ctx.load_property(p)
            ctx.estimate(conf, eps, seed=500 + i, precision='mixed', sampling='fixed', fixed_n=1000)  # warm
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            pl = ctx.estimate(conf, eps, seed=1000 + i, precision='mixed', sampling='iterative')[0]
            tp = time.perf_counter() - t0
            t0 = time.perf_counter()
            cv = ctx.estimate_cv(net, conf, eps, seed=2000 + i, precision='mixed', t_snap=t_c, x_scale=x_scale,
                                 t_scale=t_scale, beta=beta, pilot=2000)
            tc = time.perf_counter() - t0
        rows.append(dict(plain_s=tp, cv_s=tc, plain_n=pl['launched'], plain_events=pl['events'],
                         plain_p=pl['p_hat'], plain_half=(pl['hi'] - pl['lo']) / 2, cv_p=cv['p_hat'],
                         cv_half=(cv['hi'] - cv['lo']) / 2, cv_neff=cv['n_eff'], cv_full=cv['n_full'],
                         cv_prefix=cv['n_prefix'], cv_events=cv['events_full'] + cv['events_prefix']))
    T_p = sum(r['plain_s'] for r in rows)
    T_c = sum(r['cv_s'] for r in rows)
    E_p = sum(r['plain_events'] for r in rows)
    E_c = sum(r['cv_events'] for r in rows)
    n_eff = sum(r['cv_neff'] for r in rows)
    n_plain = sum(r['plain_n'] for r in rows)
    pk, src = bench.peaks()
    _line(n_eff / T_c, 'effective trajectories/s', len(rows), 1, 1e3 * T_c / len(rows), 'mixed + bf16 surrogate',
          'Lotka-Volterra family (rates x log-uniform [0.7,1.3]), G[0,30](X>0 & Y>0), checkpoint t=5, '
          '95% Wilson half-width 0.002, 8 held-out instances',
          {'plain': {'value': n_plain / T_p, 'unit': 'trajectories/s', 'seconds': T_p, 'events': E_p},
           'control_variate': {'seconds': T_c, 'events': E_c, 'n_eff': n_eff,
                               'wall_time_ratio_plain_over_cv': T_p / T_c,
                               'event_ratio_plain_over_cv': E_p / E_c, 'beta': beta,
                               'residual_variance_share': resid},
           'training': {'snapshots': int(x.shape[0]), 'trajectories_simulated': int(used * fam.n_inst),
                        'data_seconds': t_data, 'train_seconds': t_train, 'epochs': epochs, 'batch': batch,
                        'loss': [float(v) for v in loss]},
           'roofline': {'bound': 'tensor', 'kernel': 'surrogate training (mma.sync bf16)',
                        'achieved': flops / t_train / 1e12, 'peak': float(pk.get('bf16_tflops', 1899.0)),
                        'unit': 'TFLOP/s', 'frac': flops / t_train / 1e12 / float(pk.get('bf16_tflops', 1899.0)),
                        'traffic': None, 'peak_source': f'cuBLAS bf16 burst ({src})'},
           'per_instance': rows})


def cascade(args):
    import oracle
    import paper_0912_2551_gb300 as smc
    import workloads
    out = {}
    n = 2000
    for variant in (False, True):
        m, p = workloads.mapk_cascade(256, seed=5, variant=variant)
        with smc.Context(0) as ctx:
            ctx.load_model(m)
            ctx.load_property(p)
            ms, c, wil, clk = _timed_simulate(ctx, 'mixed', n, max(1, min(args.steps, 3)), 1, seed=0)
            msp, cp, _, _ = _timed_simulate(ctx, 'plain', 200, 1, 1, seed=0)
        ev = float(c[:, 2].sum())
        out['variant' if variant else 'literal'] = dict(
            ms=ms, traj_s=256 * n / (ms / 1e3), events_per_s=ev / (ms / 1e3), events_per_traj=ev / (256 * n),
            yes=int(c[:, 0].sum()), plain_traj_s=256 * 200 / (msp / 1e3), clocks=clk)
    t0 = time.perf_counter()
    m, p = workloads.mapk_cascade(4, seed=5, variant=False)
    oracle.run(m, p, seed=0, instance=0, n_traj=64)
    cpu = time.perf_counter() - t0
    lit = out['literal']
    ops = 40 + 4 + 1 + 2 + 31 + 2 + 3 * 5 + 2 * 3 + 2
    _line(lit['traj_s'], 'trajectories/s', max(1, min(args.steps, 3)), 1, lit['ms'],
          'mixed (f32 propensities, f64 clock)',
          'three-tier cascade, 22 species, 30 reactions, 256 rate-perturbed instances x 2,000 trajectories, '
          '(KPP<500) U[0,200] (KPP>=2000 & F[0,50] KPP<500) and the KPP<2000 variant',
          {'events_per_s': lit['events_per_s'], 'configs': out,
           'roofline': _issue_roofline(lit['events_per_s'], ops, 'ssa_kernel<mixed>'),
           'cpu_baseline': {'value': 64 / cpu, 'unit': 'trajectories/s', 'cores': os.cpu_count(),
                            'kind': 'oracle', 'sample': f'64 trajectories of instance 0 (literal), {cpu:.1f} s'}})


def run(args):
    {'immigration_death': immigration_death, 'random_networks': random_networks, 'surrogate': surrogate,
     'cascade': cascade}[args.config](args)
