"""Benchmark: verified trajectories/s and SSA events/s of the statistical model
checking hot path on GB300.

Workload (one step): 1,000,000 Lotka-Volterra trajectories (X -> 2X 1.0,
X + Y -> 2Y 0.005, Y -> 0 0.6, X0 = Y0 = 1000), each checked on the fly
against G[0,30](X > 0 & Y > 0) and stopped when its verdict is fixed, the
verdicts reduced on the device into the Wilson interval at 99%.  The FP64
path ("plain", the configuration's arithmetic) gives ``value``; the mixed
path ("chosen": FP32 propensities and selection, FP64 clock) is timed on the
same workload beside it.  The iterative Wilson sample size for half-width
0.001 at 99% (Fig. 2) is reported separately.

Launch: python bench.py [--gpus N --steps K --warmup W] [--impl reference]
(for N > 1 under torch.distributed.run: each rank runs its own 1,000,000
trajectories, a disjoint index range, weak scaling).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_TRAJ = 1_000_000
CONFIDENCE = 0.99
HALF_WIDTH = 0.001
SEED = 0
METRIC = 'verified trajectories/s & SSA events/s at fixed 95% Wilson width, plain vs chosen'
# DRAM bytes (read + write) of one launch of the FP64 kernel on this workload
# (ncu, 262,144-trajectory launch: the tables read once per block; the figure
# does not grow with the trajectories); None when not taken for the kernel
# as it stands.
TRAFFIC_PLAIN = 1820160
WORKLOAD = ('Lotka-Volterra X->2X 1.0, X+Y->2Y 0.005, Y->0 0.6, X0=Y0=1000; G[0,30](X>0 & Y>0); '
            '1,000,000 trajectories per step; 99% Wilson half-width 0.001')


def nvtx_push(name):
    """Opens an NVTX range (lets a profiler select one loop's launches)."""
    try:
        import torch
        torch.cuda.nvtx.range_push(name)
    except Exception:  # NVTX not available in this torch build
        pass


def nvtx_pop():
    try:
        import torch
        torch.cuda.nvtx.range_pop()
    except Exception:
        pass


def kernel_name(ctx, precision):
    """The SSA kernel serving ctx's model for a precision ('plain' / 'mixed')."""
    spec = all(sh['specialized'] for sh in ctx.launch_shapes(precision))
    if spec:
        return f'smc_jit_ssa_{precision} (model-specialized)'
    return 'ssa_kernel<plain FP64>' if precision == 'plain' else 'ssa_kernel<mixed>'


def peaks():
    try:
        with open(os.path.join(ROOT, 'MEASURED_PEAKS.json')) as f:
            return json.load(f), 'measured'
    except OSError:
        return {'sm_max_mhz': 2070.0}, 'fallback'


def algorithmic_ops_per_event(model, n_atoms: int, plain: bool) -> float:
    """Thread-level operations the method needs per SSA event (the issue
    roofline's work count): Philox4x32-10 (10 rounds x 4), two uniform maps (2 x 2), ln
    (1), clock (divide, add: 2), selection (add + compare per scanned
    reaction, (R+1)/2 expected), x += v_j (nnz), propensities (plain: R
    multiplies, R conversions and R adds for a_0; mixed: 3 per dependent
    propensity), atoms (2 each) and the horizon compare (2)."""
    import numpy as np
    R = model.n_reactions
    nnz = float((model.stoich != 0).sum(axis=1).mean())
    changes = model.stoich != 0
    dep = []
    for j in range(R):
        k_dep = 0
        for k in range(R):
            ra, rb = model.reactants[k]
            if (ra >= 0 and changes[j, ra]) or (rb >= 0 and changes[j, rb]):
                k_dep += 1
        dep.append(k_dep)
    prop = 3.0 * R if plain else 3.0 * float(np.mean(dep))
    return 40 + 4 + 1 + 2 + 2 * (R + 1) / 2.0 + nnz + prop + 2 * n_atoms + 2


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""
    Q = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
         'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
         'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.f = None

    def start(self):
        try:
            self.f = tempfile.NamedTemporaryFile('w+', suffix='.csv', delete=False)
            self.proc = subprocess.Popen(['nvidia-smi', '-i', str(self.index), f'--query-gpu={self.Q}',
                                          '--format=csv,noheader,nounits', '-lms', '200'],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(',') for r in self.f.read().strip().splitlines() if r.strip()]
        self.f.close()
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == 'active':
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {'sm_mhz': statistics.median(sm), 'sm_max_mhz': mx, 'reasons': sorted(reasons),
                'samples': len(sm)}


def oracle_baseline(model, prop, seconds_target=12.0, n_max=200_000):
    """Times the CPU oracle, as it stands, on all host cores on a bounded
    sample of the workload's trajectories (test infrastructure leg)."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.run(model, prop, seed=SEED, traj_begin=0, n_traj=min(2000, n_max), threads=cores)  # warm
    n = 4000
    while True:
        t0 = time.perf_counter()
        r = oracle.run(model, prop, seed=SEED, traj_begin=0, n_traj=n, threads=cores)
        dt = time.perf_counter() - t0
        if dt * 2 > seconds_target or n >= n_max:
            break
        n = min(n_max, int(n * max(2.0, seconds_target / max(dt, 1e-3) * 0.6)))
    ev = float(r['events'].astype('float64').sum())
    return {'value': n / dt, 'unit': 'trajectories/s', 'events_per_s': ev / dt, 'cores': cores,
            'kind': 'oracle', 'sample': f'first {n} trajectories of the workload (seed {SEED}), {dt:.1f} s'}


def run_reference(args):
    import workloads
    rank = int(os.environ.get('RANK', '0'))
    if rank != 0:
        return
    model, prop = workloads.lotka_volterra()
    import oracle
    cores = os.cpu_count() or 1
    per_step = 40_000
    for w in range(args.warmup):
        oracle.run(model, prop, seed=SEED, traj_begin=w * per_step, n_traj=per_step // 4, threads=cores)
    t0 = time.perf_counter()
    ev = 0.0
    for s in range(args.steps):
        r = oracle.run(model, prop, seed=SEED, traj_begin=s * per_step, n_traj=per_step, threads=cores)
        ev += float(r['events'].astype('float64').sum())
    dt = time.perf_counter() - t0
    value = args.steps * per_step / dt
    line = {
        'impl': 'reference', 'metric': METRIC, 'value': value, 'unit': 'trajectories/s',
        'events_per_s': ev / dt, 'n_gpus': 0, 'steps': args.steps, 'warmup': args.warmup,
        'ms_per_step': 1e3 * dt / args.steps, 'higher_is_better': True, 'scaling': 'weak',
        'vs_baseline': None, 'dtype': 'f64', 'data': 'synthetic',
        'config': {'workload': WORKLOAD, 'per_step': f'{per_step} trajectories (bounded sample)'},
        'cpu_baseline': {'value': value, 'unit': 'trajectories/s', 'cores': cores, 'kind': 'oracle',
                         'sample': f'{args.steps} x {per_step} trajectories of the workload'},
        'e2e': {'value': value, 'unit': 'trajectories/s', 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0},
    }
    print(json.dumps(line), flush=True)


def make_parser() -> argparse.ArgumentParser:
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=10)
    ap.add_argument('--warmup', type=int, default=3)
    ap.add_argument('--impl', default='native', choices=['native', 'reference'])
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--trace-cap', type=int, default=None,
                    help='nested: positions recorded per lane (SMC_OPT_TRACE_CAP)')
    ap.add_argument('--no-e2e', action='store_true')
    ap.add_argument('--traj', type=int, default=None,
                    help='trajectories per step (per instance for --config workloads; profiling runs)')
    ap.add_argument('--config', default='lotka_volterra',
                    choices=['lotka_volterra', 'immigration_death', 'random_networks', 'surrogate', 'cascade',
                             'surrogate_inference', 'surrogate_training', 'large_networks', 'nested'])
    return ap


def main():
    global N_TRAJ
    ap = make_parser()
    args = ap.parse_args()
    if args.traj is not None and args.config == 'lotka_volterra':
        N_TRAJ = args.traj
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == 'reference':
        run_reference(args)
        return
    if args.config != 'lotka_volterra':
        import bench_configs
        bench_configs.run(args)
        return

    import numpy as np
    import torch
    import workloads
    import paper_0912_2551_gb300 as smc

    world = int(os.environ.get('WORLD_SIZE', '1'))
    rank = int(os.environ.get('RANK', '0'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl')
    torch.cuda.set_device(local)
    dev = torch.device('cuda', local)

    model, prop = workloads.lotka_volterra()
    ctx = smc.Context(local)
    ctx.load_model(model)
    ctx.load_property(prop)
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)  # > 129 MB L2
    base = rank * N_TRAJ

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    def timed(precision):
        counts = torch.zeros((1, 4), dtype=torch.int64, device=dev)
        wil = torch.zeros((1, 3), dtype=torch.float64, device=dev)
        with torch.cuda.stream(stream):
            for w in range(args.warmup):
                ctx.simulate(precision, seed=SEED, traj_begin=base, n_traj=N_TRAJ, confidence=CONFIDENCE,
                             outputs=(), counts=counts, wilson=wil, stream=stream)
        barrier()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        counts.zero_()
        clocks = Clocks(local)
        clocks.start()
        barrier()
        t0 = time.perf_counter()
        nvtx_push(f'{precision}_steps')  # lets a profiler select this loop's launches
        with torch.cuda.stream(stream):
            for s in range(args.steps):
                flush.fill_(s)  # L2 flush between steps, outside the step's events
                evs[s][0].record(stream)
                ctx.simulate(precision, seed=SEED, traj_begin=base, n_traj=N_TRAJ, confidence=CONFIDENCE,
                             outputs=(), counts=counts, wilson=wil, stream=stream)
                evs[s][1].record(stream)
        nvtx_pop()
        barrier()
        wall = time.perf_counter() - t0
        clk = clocks.stop()
        step_ms = [a.elapsed_time(b) for a, b in evs]
        c = counts.cpu().numpy()[0]
        return dict(step_ms=step_ms, wall=wall, counts=c, clocks=clk)

    plain = timed('plain')
    mixed = timed('mixed')

    def reduce_max(x):
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def reduce_sum(arr):
        if dist is None:
            return arr
        t = torch.tensor(arr, dtype=torch.int64, device=dev)
        dist.all_reduce(t)
        return t.cpu().numpy()

    res = {}
    for name, r in (('plain', plain), ('mixed', mixed)):
        tot_ms = reduce_max(sum(r['step_ms']))
        cnt = reduce_sum(r['counts'])
        ev = float(cnt[2]) / args.steps  # events per step, all ranks
        n_all = N_TRAJ * world
        res[name] = dict(ms=tot_ms / args.steps, traj_s=n_all * args.steps / (tot_ms / 1e3),
                         events_s=ev * args.steps / (tot_ms / 1e3), yes=int(cnt[0]) // args.steps,
                         n=int(cnt[1]) // args.steps, budget=int(cnt[3]), events_per_traj=ev / n_all,
                         clocks=r['clocks'], per_rank_ms=sum(r['step_ms']) / args.steps)

    # iterative Wilson sample size at the configured width (Fig. 2), untimed
    it = ctx.estimate(CONFIDENCE, HALF_WIDTH, seed=SEED, precision='plain', sampling='iterative')[0]
    # Wilson interval of one step's counts (computed on the device)
    one = ctx.simulate('plain', seed=SEED, traj_begin=base, n_traj=N_TRAJ, confidence=CONFIDENCE, outputs=())
    torch.cuda.synchronize(dev)
    wil = one['wilson'].cpu().numpy()[0].tolist()

    # e2e: through the public API with host buffers, every step loading the
    # model and property from host memory and reading the result back
    e2e_steps = max(3, min(args.steps, 5))
    e2e_value = None
    if not args.no_e2e:
        ctx2 = smc.Context(local)
        for w in range(args.warmup):  # the same calls, untimed (first one runs the autotuner)
            ctx2.load_model(model)
            ctx2.load_property(prop)
            ctx2.estimate(CONFIDENCE, HALF_WIDTH, seed=SEED + 1000 + w, precision='plain', sampling='fixed',
                          fixed_n=N_TRAJ)
        barrier()
        t0 = time.perf_counter()
        for s in range(e2e_steps):
            ctx2.load_model(model)
            ctx2.load_property(prop)
            # each rank its own trajectories (a seed of its own: the estimate numbers them from 0)
            ctx2.estimate(CONFIDENCE, HALF_WIDTH, seed=SEED + s + 7919 * rank, precision='plain',
                          sampling='fixed', fixed_n=N_TRAJ)
        barrier()
        e2e_dt = reduce_max(time.perf_counter() - t0)
        ctx2.close()
        e2e_value = world * N_TRAJ * e2e_steps / e2e_dt
    # bytes: the instance table and monitor program up, ranges up, counts and
    # interval down (counted from the library's layouts)
    h2d = 4 * 64 + 352 + 16
    d2h = 4 * 8 + 3 * 8

    pk, pk_src = peaks()
    f_clk = float(pk.get('sm_max_mhz', 2070.0)) * 1e6
    props = torch.cuda.get_device_properties(dev)
    n_sm = props.multi_processor_count
    peak_ops = n_sm * 4 * 32 * f_clk  # thread instructions per second at the issue limit
    w_plain = algorithmic_ops_per_event(model, 2, True)
    w_mixed = algorithmic_ops_per_event(model, 2, False)
    ach_plain = w_plain * res['plain']['events_s'] / max(world, 1)
    ach_mixed = w_mixed * res['mixed']['events_s'] / max(world, 1)
    # FP64 pipe: GB300 issues 2 FP64 operations per clock per SM (1/64 of
    # FP32).  Per event the kernel leaves R products and R - 1 sums (Eq. 1),
    # the clock add and u_sel * a_0 on it; ln u and the division by a_0 run
    # on the integer pipes.  Had they stayed FP64 (15 operations for the
    # table-driven logarithm, 9.75 for the correctly rounded division, as
    # counted by ncu), the FP64 pipe alone would cap the path at
    # fp64_only_bound_events_per_s.
    R = model.n_reactions
    fp64_per_event = 2 * R - 1 + 2
    fp64_naive = fp64_per_event + 15 + 9.75
    fp64_peak = n_sm * 2 * f_clk
    fp64_ach = fp64_per_event * res['plain']['events_s'] / max(world, 1)

    line = {
        'metric': METRIC,
        'value': res['plain']['traj_s'],
        'unit': 'trajectories/s',
        'events_per_s': res['plain']['events_s'],
        'n_gpus': world,
        'steps': args.steps,
        'warmup': args.warmup,
        'ms_per_step': res['plain']['ms'],
        'higher_is_better': True,
        'scaling': 'weak',
        'vs_baseline': None,
        'dtype': 'f64',
        'data': 'synthetic',
        'config': {'workload': WORKLOAD, 'trajectories_per_step': N_TRAJ * world,
                   'parallelism': f'{world} independent trajectory ranges' if world > 1 else 'single GPU',
                   'l2': 'flushed between steps (512 MiB write), outside the step events',
                   'events_per_trajectory': res['plain']['events_per_traj'],
                   'launch': {'plain': ctx.launch_shapes('plain'), 'mixed': ctx.launch_shapes('mixed')}},
        'chosen': {'precision': 'mixed (FP32 propensities and selection, int32 counts, FP64 clock)',
                   'value': res['mixed']['traj_s'], 'unit': 'trajectories/s',
                   'events_per_s': res['mixed']['events_s'], 'ms_per_step': res['mixed']['ms'],
                   'p_hat': res['mixed']['yes'] / max(res['mixed']['n'], 1),
                   'speedup_vs_plain': res['mixed']['traj_s'] / res['plain']['traj_s'],
                   'roofline_frac': ach_mixed / peak_ops},
        'result': {'p_hat': wil[0], 'lo': wil[1], 'hi': wil[2], 'n': res['plain']['n'],
                   'budget_hits': res['plain']['budget'],
                   'iterative_wilson': {'half_width': HALF_WIDTH, 'confidence': CONFIDENCE,
                                        'n': it['launched'], 'p_hat': it['p_hat'], 'lo': it['lo'],
                                        'hi': it['hi'], 'iterations': it['iterations']}},
        'roofline': {'bound': 'alu', 'kernel': kernel_name(ctx, 'plain'),
                     'achieved': ach_plain / 1e9, 'peak': peak_ops / 1e9, 'unit': 'G thread-op/s',
                     'frac': ach_plain / peak_ops, 'traffic': TRAFFIC_PLAIN,
                     'ops_per_event': w_plain,
                     'peak_source': f'{n_sm} SMs x 4 issue slots x 32 lanes x {f_clk / 1e6:.0f} MHz '
                                    f'({pk_src} max SM clock)'},
        'fp64_pipe': {'kernel': kernel_name(ctx, 'plain'), 'fp64_ops_per_event': fp64_per_event,
                      'achieved': fp64_ach / 1e9, 'peak': fp64_peak / 1e9, 'unit': 'G FP64 op/s',
                      'frac': fp64_ach / fp64_peak,
                      'fp64_only_bound_events_per_s': fp64_peak / fp64_naive,
                      'peak_source': f'{n_sm} SMs x 2 FP64 ops/clk x {f_clk / 1e6:.0f} MHz'},
        'e2e': {'value': e2e_value, 'unit': 'trajectories/s', 'h2d_bytes_per_step': h2d,
                'd2h_bytes_per_step': d2h},
        'gpu_launches': 2 * args.steps,
        'clocks': res['plain']['clocks'],
        'clocks_chosen': res['mixed']['clocks'],
    }
    if rank == 0 and not args.no_cpu_baseline and world == 1:
        line['cpu_baseline'] = oracle_baseline(model, prop)
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == '__main__':
    main()
