"""The multi-rank Fig. 2 driver (paper_0912_2551_gb300.distributed.fig2) on
two gloo ranks on the CPU: every rank runs its slice of each batch with the
CPU oracle, counts are all-reduced, and the result must equal the
single-process procedure on the same trajectory indices."""
import os

import numpy as np
import pytest


def _worker(rank, world, port, q):
    os.environ['MASTER_ADDR'] = '127.0.0.1'
    os.environ['MASTER_PORT'] = str(port)
    import torch.distributed as dist
    dist.init_process_group('gloo', rank=rank, world_size=world)
    try:
        import oracle
        import workloads
        from paper_0912_2551_gb300 import distributed
        m, p = workloads.lotka_volterra()
        seen = []

        def run(begin, count):
            seen.append((begin, count))
            r = oracle.run(m, p, seed=3, traj_begin=begin, n_traj=count, threads=2)
            return np.array([int(r['verdict'].sum()), int((r['status'] == 0).sum()),
                             int(r['events'].sum()), int((r['status'] == 1).sum())], np.int64)

        res = distributed.fig2(run, 0.02, 0.95)
        q.put((rank, res, seen))
    finally:
        dist.destroy_process_group()


def test_two_rank_fig2_equals_single_process():
    import multiprocessing as mp
    pytest.importorskip('torch')
    from oracle import wilson
    import oracle
    import workloads
    import socket
    s = socket.socket()
    s.bind(('127.0.0.1', 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context('spawn')
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = [q.get(timeout=300) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    out.sort(key=lambda t: t[0])
    r0, r1 = out[0][1], out[1][1]
    assert r0 == r1  # every rank takes the same decision
    # the ranks covered disjoint slices of the same batches
    s0, s1 = out[0][2], out[1][2]
    assert len(s0) == len(s1) == r0['iterations']
    for (b0, c0), (b1, c1) in zip(s0, s1):
        assert b0 + c0 == b1
    m, p = workloads.lotka_volterra()

    def run(begin, count):
        r = oracle.run(m, p, seed=3, traj_begin=begin, n_traj=count)
        return int(r['verdict'].sum()), int((r['status'] == 0).sum())

    ref = wilson.iterative(run, 0.02, 0.95)
    assert r0['launched'] == ref['n_tot'] and r0['yes'] == ref['yes']
    assert r0['iterations'] == ref['iterations']
    assert abs(r0['lo'] - ref['lo']) <= 1e-12 * max(ref['lo'], 1e-300) + 1e-300
    assert abs(r0['hi'] - ref['hi']) <= 1e-12 * ref['hi']
