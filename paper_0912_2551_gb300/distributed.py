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

import math
from typing import Callable, Optional

import numpy as np

from . import _native as N


def _slice(total_begin: int, count: int, rank: int, world: int):
    """This rank's contiguous part of trajectories [total_begin,
    total_begin + count): the first count % world ranks take one more."""
    q, r = divmod(count, world)
    return total_begin + rank * q + min(rank, r), q + (1 if rank < r else 0)


def fig2(run: Callable[[int, int], np.ndarray], half_width: float, confidence: float, group=None,
         start_p: float = 1.0, fixed_n: Optional[int] = None, max_iter: int = 1000,
         reduce_device=None):
    """Iterative Wilson procedure over ranks.  ``run(begin, count)`` runs this
    rank's trajectories and returns int64 counts [yes, n, events, budget].
    start_p = 1: iterative; 0.5: conservative (one batch); fixed_n: one batch
    of that size.  Returns a dict like smc_estimate's result."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    if fixed_n is not None:
        N_batch = int(fixed_n)
    else:
        N_batch = int(math.ceil(N.smc_wilson_sample(start_p, half_width, confidence)))
    tot = np.zeros(4, np.int64)
    n_tot = 0
    it = 0
    while True:
        it += 1
        b, c = _slice(n_tot, N_batch, rank, world)
        local = np.asarray(run(b, c) if c > 0 else np.zeros(4, np.int64), np.int64)
        t = torch.tensor(local, dtype=torch.int64, device=reduce_device or 'cpu')
        if world > 1:
            dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
        tot += t.cpu().numpy()
        n_tot += N_batch
        if fixed_n is not None or start_p == 0.5 or it >= max_iter:
            break
        p = tot[0] / tot[1] if tot[1] else 0.0
        pp = p + half_width if p <= 0.5 else p - half_width
        n_prime = int(math.ceil(N.smc_wilson_sample(pp, half_width, confidence)))
        if n_prime - n_tot > 0:
            N_batch = n_prime - n_tot
            continue
        break
    import ctypes
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

    start_p = {'iterative': 1.0, 'conservative': 0.5, 'fixed': 1.0}[sampling]
    return fig2(run, half_width, confidence, group, start_p=start_p,
                fixed_n=fixed_n if sampling == 'fixed' else None,
                reduce_device=dev if backend == 'nccl' else None)
