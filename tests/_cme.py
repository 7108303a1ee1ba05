"""Exact transient probabilities of tiny reaction networks, used to pin the
oracle's SSA and monitor (a test helper, independent of both paths).

The chemical master equation of a network with a finite reachable state set
is a CTMC; P(F[0,T] goal) is the probability that the chain, with the goal
states made absorbing, sits in a goal state at T: the matching row of
expm(Q T) (SciPy).  This is the exact-numerical-model-checking comparison of
Sec. 5 (there done with PRISM) on models small enough to solve directly.
"""
from collections import deque

import numpy as np
from scipy.linalg import expm


def _rate(c, reac, x):
    a, b = reac
    if a < 0 and b < 0:
        return c
    if b < 0:
        return c * x[a]
    if a < 0:
        return c * x[b]
    if a == b:
        return c * x[a] * (x[a] - 1) / 2.0
    return c * x[a] * x[b]


def _factor(x, m, n, a0, a1, b0, b1):
    v = float(x[m]) ** n
    return (a0 + a1 * v) / (b0 + b1 * v)


def eventually_probability(model, goal, T, cap=None, inst=0):
    """P(exists t <= T with goal(x(t))) for x(0) = model.x0[inst]; states
    with any count above ``cap`` are made absorbing and counted as failure
    (truncation; choose cap so their probability is negligible)."""
    x0 = tuple(int(v) for v in model.x0[inst])
    rates = model.rates[inst]
    index = {x0: 0}
    states = [x0]
    q = deque([x0])
    edges = []
    while q:
        x = q.popleft()
        i = index[x]
        if goal(x) or (cap is not None and max(x) > cap):
            continue
        for j in range(model.n_reactions):
            r = _rate(rates[j], model.reactants[j], x)
            for f in getattr(model, 'factors', None) or []:
                if f[0] == j:
                    r *= _factor(x, *f[1:])
            if r <= 0:
                continue
            y = tuple(int(v) for v in np.asarray(x) + model.stoich[j])
            if y not in index:
                index[y] = len(states)
                states.append(y)
                q.append(y)
            edges.append((i, index[y], r))
    n = len(states)
    Q = np.zeros((n, n))
    for i, k, r in edges:
        Q[i, k] += r
        Q[i, i] -= r
    P = expm(Q * T)[0]
    return float(sum(P[index[s]] for s in states if goal(s)))


def until_probability(model, stay, goal, T, cap=None, inst=0):
    """P(stay U[0,T] goal): goal states absorbing (success), states where
    neither holds absorbing (failure), states above ``cap`` absorbing
    (failure, truncation)."""
    x0 = tuple(int(v) for v in model.x0[inst])
    rates = model.rates[inst]
    index = {x0: 0}
    states = [x0]
    q = deque([x0])
    edges = []
    while q:
        x = q.popleft()
        i = index[x]
        if goal(x) or not stay(x) or (cap is not None and max(x) > cap):
            continue
        for j in range(model.n_reactions):
            r = _rate(rates[j], model.reactants[j], x)
            for f in getattr(model, 'factors', None) or []:
                if f[0] == j:
                    r *= _factor(x, *f[1:])
            if r <= 0:
                continue
            y = tuple(int(v) for v in np.asarray(x) + model.stoich[j])
            if y not in index:
                index[y] = len(states)
                states.append(y)
                q.append(y)
            edges.append((i, index[y], r))
    n = len(states)
    Q = np.zeros((n, n))
    for i, k, r in edges:
        Q[i, k] += r
        Q[i, i] -= r
    P = expm(Q * T)[0]
    return float(sum(P[index[s]] for s in states if goal(s)))
