"""Test helpers for per-trajectory parity between the CUDA path and the oracle.

``first_divergence`` locates, for one trajectory whose GPU and oracle results
differ, the first event after which the two states differ: both sides are
re-run with an event budget b (the trajectory stops after b events with its
state and clock), and b is bisected.  Both sides draw the same random numbers
(Philox keyed by event, trajectory and instance), so the reaction sequence is
the same until the first reaction whose selection differs; a clock that
differs only in its last bits (the logarithm of Eq. 2a is faithful, not
correctly rounded on both sides) changes no selection, only where a time
window closes.
"""
from __future__ import annotations

import numpy as np


def _gpu_state(ctx, precision, seed, traj, budget, instance):
    import torch
    ctx.set_option('event_budget', budget)
    o = ctx.simulate(precision, seed=seed, traj_begin=traj, n_traj=1,
                     outputs=('verdict', 'status', 'events', 't_final', 'x_final'))
    torch.cuda.synchronize()
    return (int(o['events'][instance, 0]), float(o['t_final'][instance, 0]),
            o['x_final'][instance, 0].cpu().numpy().copy(), int(o['status'][instance, 0]))


DEFAULT_BUDGET = 1 << 24  # the library's default event budget


def first_divergence(ctx, orc, model, prop, seed, traj, instance=0, precision='plain', max_events=DEFAULT_BUDGET):
    """Bisects the event budget for the first event after which the GPU and
    oracle states (event count, counts, clock bits) differ.  Returns a dict:
    event (the first differing event count, or None if the two agree at
    every budget up to max_events), and the two sides' states there.  The
    context's model and property must be loaded; its event budget is reset
    to the library's default afterwards."""
    S = model.n_species

    def same(b):
        ge, gt, gx, gs = _gpu_state(ctx, precision, seed, traj, b, instance)
        r = orc.run(model, prop, seed=seed, instance=instance, traj_begin=traj, n_traj=1, budget=b, want_x=True)
        re_, rt, rx = int(r['events'][0]), float(r['t_final'][0]), r['x_final'][0]
        ok = ge == re_ and gt == rt and np.array_equal(gx[:S], rx)
        return ok, dict(gpu=dict(events=ge, t=gt, x=gx[:S].tolist(), status=gs),
                        oracle=dict(events=re_, t=rt, x=rx.tolist(), status=int(r['status'][0])))

    try:
        ok, info = same(max_events)
        if ok:
            return dict(event=None, **info)
        lo, hi = 0, max_events  # same(lo) holds, same(hi) fails
        bad = info
        while hi - lo > 1:
            mid = (lo + hi) // 2
            ok, info = same(mid)
            if ok:
                lo = mid
            else:
                hi, bad = mid, info
        return dict(event=hi, **bad)
    finally:
        ctx.set_option('event_budget', DEFAULT_BUDGET)


def ulps_apart(a: float, b: float) -> int:
    """Distance of two positive doubles in units in the last place."""
    ia = np.array([a], np.float64).view(np.int64)[0]
    ib = np.array([b], np.float64).view(np.int64)[0]
    return int(abs(int(ia) - int(ib)))
