"""The multi-rank Fig. 2 driver (paper_0912_2551_gb300.distributed.fig2) on
two and three gloo ranks on the CPU (three: batches that do not split
evenly): every rank runs its slice of each batch with the CPU oracle,
counts are all-reduced, and the result must equal the single-process
procedure on the same trajectory indices."""
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


@pytest.mark.parametrize('world', [2, 3])
def test_multi_rank_fig2_equals_single_process(world):
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
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    out = [q.get(timeout=300) for _ in procs]
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    out.sort(key=lambda t: t[0])
    r0 = out[0][1]
    assert all(o[1] == r0 for o in out)  # every rank takes the same decision
    # the ranks covered contiguous, disjoint slices of the same batches
    slices = [o[2] for o in out]
    assert all(len(sl) == r0['iterations'] for sl in slices)
    for it in range(r0['iterations']):
        for r in range(world - 1):
            b, c = slices[r][it]
            assert b + c == slices[r + 1][it][0]
        counts = [slices[r][it][1] for r in range(world)]
        assert max(counts) - min(counts) <= 1  # balanced to within one trajectory
    m, p = workloads.lotka_volterra()

    def run(begin, count):
        r = oracle.run(m, p, seed=3, traj_begin=begin, n_traj=count)
        return int(r['verdict'].sum()), int((r['status'] == 0).sum())

    ref = wilson.iterative(run, 0.02, 0.95)
    assert r0['launched'] == ref['n_tot'] and r0['yes'] == ref['yes']
    assert r0['iterations'] == ref['iterations']
    assert abs(r0['lo'] - ref['lo']) <= 1e-12 * max(ref['lo'], 1e-300) + 1e-300
    assert abs(r0['hi'] - ref['hi']) <= 1e-12 * ref['hi']


def test_slices_partition_every_batch():
    from paper_0912_2551_gb300.distributed import _slice
    for world in (1, 2, 3, 4, 7, 8):
        for count in (0, 1, 2, 5, 7, 8, 127, 2648, 10**6 + 3):
            begin = 12345
            parts = [_slice(begin, count, r, world) for r in range(world)]
            assert parts[0][0] == begin
            for (b, c), (b2, _) in zip(parts, parts[1:]):
                assert b + c == b2
            assert sum(c for _, c in parts) == count
            assert max(c for _, c in parts) - min(c for _, c in parts) <= 1
