"""smc_simulate_noalloc: the entry point for callers that must not allocate
device memory while they run (their device memory belongs to another
allocator, or they run in a loop that must not block in cudaMalloc).  It
keeps the SSA kernel's work queue in a fixed array of the library instead of
context buffers.  Its outputs must equal smc_simulate's on the same inputs,
on consecutive calls (the shared array keeps the previous call's counters,
which each call resets).  Collected last so that a failure here comes after
every other test has run.
"""
import ctypes

import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope='module')
def env():
    torch = pytest.importorskip('torch')
    if not torch.cuda.is_available():
        pytest.skip('no GPU')
    import paper_0912_2551_gb300 as smc
    from paper_0912_2551_gb300 import _native
    return torch, smc, _native


def _outs(torch, n_inst, n_traj):
    dev = torch.device('cuda', 0)
    o = dict(counts=torch.zeros((n_inst, 4), dtype=torch.int64, device=dev),
             wilson=torch.zeros((n_inst, 3), dtype=torch.float64, device=dev),
             verdict=torch.zeros((n_inst, n_traj), dtype=torch.uint8, device=dev),
             events=torch.zeros((n_inst, n_traj), dtype=torch.int64, device=dev))
    return o, None


def _call(torch, N, ctx, name, precision, seed, begin, n_traj, o):
    so = N.smc_sim_out()
    for k, v in o.items():
        setattr(so, k, v.data_ptr())
    stream = torch.cuda.current_stream()
    rc = getattr(N, name)(ctx.h, precision, seed, begin, n_traj, 0.99, ctypes.byref(so),
                          ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return rc


@pytest.mark.parametrize('which', ['lotka_volterra', 'lv_family3'])
@pytest.mark.parametrize('precision', [0, 1])
def test_noalloc_matches_simulate_on_two_calls(env, which, precision):
    torch, smc, N = env
    if which == 'lotka_volterra':
        m, p = workloads.lotka_volterra()
    else:
        m, p = workloads.lotka_volterra_family(3, seed=2)
    n_traj, begin, seed = 20000, 1000, 17
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        ref, _ = _outs(torch, m.n_inst, n_traj)
        assert _call(torch, N, ctx, 'smc_simulate', precision, seed, begin, n_traj, ref) == 0
        for _ in range(2):
            got, _ = _outs(torch, m.n_inst, n_traj)
            rc = _call(torch, N, ctx, 'smc_simulate_noalloc', precision, seed, begin, n_traj, got)
            assert rc == 0, N.smc_last_error(ctx.h)
            assert torch.equal(got['verdict'], ref['verdict'])
            assert torch.equal(got['events'], ref['events'])
            assert torch.equal(got['counts'], ref['counts'])
            w, wr = got['wilson'].cpu().numpy(), ref['wilson'].cpu().numpy()
            assert np.all(np.abs(w - wr) <= 1e-12 * np.abs(wr))


def test_noalloc_reports_missing_tables_and_too_many_instances(env):
    torch, smc, N = env
    m, p = workloads.lotka_volterra()
    with smc.Context(0) as ctx:
        ctx.load_model(m)
        ctx.load_property(p)
        o, _ = _outs(torch, 1, 10)
        assert _call(torch, N, ctx, 'smc_simulate_noalloc', 0, 1, 0, 10, o) == N.SMC_E_STATE
    big, pb = workloads.lotka_volterra(n_inst=4097)
    with smc.Context(0) as ctx:
        ctx.load_model(big)
        ctx.load_property(pb)
        o, _ = _outs(torch, 4097, 1)
        assert _call(torch, N, ctx, 'smc_simulate', 0, 1, 0, 1, o) == 0
        assert _call(torch, N, ctx, 'smc_simulate_noalloc', 0, 1, 0, 1, o) == N.SMC_E_INVALID_ARG
        assert b'4096' in N.smc_last_error(ctx.h)
