"""Fig. 2 across the ranks of a torch.distributed process group.

The trajectories of an estimate are independent, so ranks share them by
index: each batch [N_tot, N_tot + N) of the iterative Wilson procedure
(Fig. 2) is cut into one contiguous slice per rank.  The counts (yes, n,
events, budget hits) are summed with one all_reduce per iteration -- the
only exchange, the counterpart of the paper's MPI_Gather of verdicts
(Sec. 4.1) without the traces -- and every rank then takes the same
decision.  Because random numbers are keyed by trajectory index, the result
equals a single-GPU run bit for bit.

``fig2`` is the host loop over any ``run(begin, count) -> counts``;
``estimate`` wires it to a Context on this rank's GPU (single-instance
contexts).
"""
from __future__ import annotations

import ctypes
from typing import Callable, Optional

import numpy as np

from . import _native as N

SAMPLING = {'fixed': N.SMC_FIXED_N, 'iterative': N.SMC_ITERATIVE, 'conservative': N.SMC_CONSERVATIVE}


def _slice(total_begin: int, count: int, rank: int, world: int):
    """This rank's contiguous part of trajectories [total_begin,
    total_begin + count): the first count % world ranks take one more."""
    q, r = divmod(count, world)
    return total_begin + rank * q + min(rank, r), q + (1 if rank < r else 0)


def _next_batch(sampling: int, fixed_n: int, confidence: float, half_width: float, tot, n_tot: int) -> int:
    """Fig. 2's decision between batches, taken by the library
    (smc_fig2_next_batch): the next batch size, 0 = stop."""
    nxt = ctypes.c_uint64()
    rc = N.smc_fig2_next_batch(sampling, int(fixed_n), float(confidence), float(half_width), int(tot[0]),
                               int(tot[1]), int(n_tot), ctypes.byref(nxt))
    if rc != N.SMC_OK:
        raise ValueError(f'smc_fig2_next_batch failed ({rc})')
    return int(nxt.value)


def fig2(run: Callable[[int, int], np.ndarray], half_width: float, confidence: float, group=None,
         sampling: str = 'iterative', fixed_n: Optional[int] = None, max_iter: int = 1000,
         reduce_device=None):
    """The iterative Wilson procedure over ranks.  ``run(begin, count)`` runs
    this rank's trajectories and returns int64 counts [yes, n, events,
    budget].  ``sampling``: 'iterative' (Fig. 2), 'conservative' (one batch
    of Eq. 5 at p = 1/2) or 'fixed' (one batch of ``fixed_n``).  The batch
    sizes come from the library's smc_fig2_next_batch; this loop only cuts
    each batch into the ranks' slices and sums the counts.  Returns a dict
    like smc_estimate's result."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    mode = SAMPLING[sampling]
    fixed = int(fixed_n) if sampling == 'fixed' else 0
    tot = np.zeros(4, np.int64)
    n_tot = 0
    it = 0
    batch = _next_batch(mode, fixed, confidence, half_width, tot, n_tot)
    while batch > 0 and it < max_iter:
        it += 1
        b, c = _slice(n_tot, batch, rank, world)
        local = np.asarray(run(b, c) if c > 0 else np.zeros(4, np.int64), np.int64)
        t = torch.tensor(local, dtype=torch.int64, device=reduce_device or 'cpu')
        if dist.is_initialized():
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        tot += t.cpu().numpy()
        n_tot += batch
        batch = _next_batch(mode, fixed, confidence, half_width, tot, n_tot)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    yes, n = int(tot[0]), int(tot[1])
    N.smc_wilson_interval(yes, n, confidence, ctypes.byref(lo), ctypes.byref(hi))
    return dict(p_hat=yes / n if n else float('nan'), lo=lo.value, hi=hi.value, n=n, yes=yes,
                events=int(tot[2]), budget_hits=int(tot[3]), launched=n_tot, iterations=it)


def estimate(ctx, confidence: float, half_width: float, seed: int = 0, precision: str = 'plain',
             sampling: str = 'iterative', fixed_n: int = 0, group=None):
    """smc_estimate's procedure across ranks for a single-instance context:
    each rank simulates its slice on its own GPU (smc_simulate), the counts
    are all-reduced (NCCL when the group's backend is nccl)."""
    import torch
    import torch.distributed as dist
    if ctx.n_inst != 1:
        raise ValueError('distributed estimate needs a single-instance context')
    dev = torch.device('cuda', ctx.device)
    backend = dist.get_backend(group) if dist.is_initialized() else 'gloo'

    def run(begin, count):
        out = ctx.simulate(precision, seed=seed, traj_begin=begin, n_traj=count, confidence=confidence,
                           outputs=())
        torch.cuda.synchronize(dev)
        return out['counts'].cpu().numpy()[0]

    return fig2(run, half_width, confidence, group, sampling=sampling,
                fixed_n=fixed_n if sampling == 'fixed' else None,
                reduce_device=dev if backend == 'nccl' else None)
