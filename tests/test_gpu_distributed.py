"""The multi-rank estimate (paper_0912_2551_gb300.distributed) on the GPU:
a one-rank NCCL process group runs the same Fig. 2 batches, the counts go
through an NCCL all_reduce on the device, and the result equals smc_estimate
on the same context bit for bit (counts, events, iterations and interval)."""
import socket

import pytest

import workloads

pytestmark = pytest.mark.gpu


def _free_port():
    s = socket.socket()
    s.bind(('127.0.0.1', 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.mark.parametrize('sampling,precision', [('iterative', 'plain'), ('iterative', 'mixed'),
                                                ('conservative', 'plain'), ('fixed', 'mixed')])
def test_one_rank_nccl_estimate_equals_smc_estimate(sampling, precision):
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no GPU')
    import torch.distributed as dist
    import paper_0912_2551_gb300 as smc
    from paper_0912_2551_gb300 import distributed
    torch.cuda.set_device(0)
    dist.init_process_group('nccl', init_method=f'tcp://127.0.0.1:{_free_port()}', rank=0, world_size=1)
    try:
        assert dist.get_backend() == 'nccl'
        m, p = workloads.immigration_death()
        with smc.Context(0) as ctx:
            ctx.load_model(m)
            ctx.load_property(p)
            got = distributed.estimate(ctx, 0.99, 0.01, seed=21, precision=precision, sampling=sampling,
                                       fixed_n=5000)
            ref = ctx.estimate(0.99, 0.01, seed=21, precision=precision, sampling=sampling, fixed_n=5000)[0]
        for k in ('yes', 'n', 'events', 'budget_hits', 'launched', 'iterations'):
            assert got[k] == ref[k], (k, got[k], ref[k])
        assert got['p_hat'] == ref['p_hat'] and got['lo'] == ref['lo'] and got['hi'] == ref['hi'], (got, ref)
        if sampling == 'iterative':
            assert got['iterations'] >= 2
    finally:
        dist.destroy_process_group()
