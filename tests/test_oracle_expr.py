"""Arithmetic atoms (Sec. 3.1: val <| val with + - * /, sqrt, pow) in the
oracle: the evaluation on hand-made states (exact cases, IEEE division by
zero and NaN), and the paper's example formula (X1 < sqrt(X2)) U (X2 >= 10 +
X3) on a small network against the exact CME solution of the same chain."""
import math

import numpy as np
import pytest

import oracle
import workloads
from tests import _cme

SP = ['X1', 'X2', 'X3']


def holds(atom, state):
    p = workloads.Property([atom], ('atom', 0))
    return oracle.eval_prefix(p, 3, np.asarray([state]), np.asarray([0.0]), 0.0, True) == 1


def test_sqrt_comparisons_are_exact_at_squares():
    a = workloads.expr_atom(SP, [('x', 'X1')], '<', [('x', 'X2'), ('sqrt',)])
    assert holds(a, [2, 9, 0]) and not holds(a, [3, 9, 0]) and holds(a, [3, 10, 0])
    b = workloads.expr_atom(SP, [('x', 'X2')], '>=', [('c', 10.0), ('x', 'X3'), ('+',)])
    assert holds(b, [0, 15, 5]) and not holds(b, [0, 14, 5])


def test_powers_products_and_quotients():
    a = workloads.expr_atom(SP, [('x', 'X1'), ('pow', 2)], '==', [('c', 9.0)])
    assert holds(a, [3, 0, 0]) and not holds(a, [4, 0, 0])
    z = workloads.expr_atom(SP, [('x', 'X1'), ('pow', 0)], '==', [('c', 1.0)])
    assert holds(z, [0, 0, 0])
    q = workloads.expr_atom(SP, [('x', 'X1'), ('x', 'X2'), ('/',)], '>', [('c', 1.5)])
    assert holds(q, [4, 2, 0]) and not holds(q, [3, 2, 0])
    # a linear combination written as a program equals the linear atom
    lin = workloads.atom(SP, {'X1': 2, 'X3': -1}, '<=', 7)
    ex = workloads.expr_atom(SP, [('c', 2.0), ('x', 'X1'), ('*',), ('x', 'X3'), ('-',)], '<=', [('c', 7.0)])
    for s in ([3, 0, 0], [4, 0, 0], [4, 0, 1], [5, 0, 2], [5, 0, 4]):
        assert holds(lin, s) == holds(ex, s)


def test_ieee_division_by_zero_and_nan():
    q = workloads.expr_atom(SP, [('x', 'X1'), ('x', 'X2'), ('/',)], '>', [('c', 1e300)])
    assert holds(q, [1, 0, 0])            # 1 / 0 = +inf
    assert not holds(q, [0, 0, 0])        # 0 / 0 = NaN: comparison false
    ne = workloads.expr_atom(SP, [('x', 'X1'), ('x', 'X2'), ('/',)], '!=', [('c', 0.0)])
    assert holds(ne, [0, 0, 0])           # NaN != 0 is true
    neg = workloads.expr_atom(SP, [('c', -1.0), ('sqrt',)], '<', [('c', 0.0)])
    assert not holds(neg, [0, 0, 0])      # sqrt(-1) = NaN


def test_paper_example_formula_against_cme():
    m, p = workloads.sqrt_race()
    stay = lambda x: x[0] < math.sqrt(x[1])  # noqa: E731
    goal = lambda x: x[1] >= 10 + x[2]  # noqa: E731
    exact = _cme.until_probability(m, stay, goal, p.formula[2], cap=20)
    assert 0.2 < exact < 0.9
    y = oracle.run(m, p, seed=7, n_traj=20000)['verdict'].astype(float)
    assert abs(y.mean() - exact) < 4.5 * math.sqrt(exact * (1 - exact) / y.size), (y.mean(), exact)
    # the same formula with sqrt dropped (X1 < X2) has a different answer
    alt = workloads.Property([workloads.expr_atom(SP, [('x', 'X1')], '<', [('x', 'X2')]), p.atoms[1]], p.formula)
    wrong = _cme.until_probability(m, lambda x: x[0] < x[1], goal, p.formula[2], cap=20)
    assert abs(wrong - exact) > 0.05
    y2 = oracle.run(m, alt, seed=7, n_traj=8000)['verdict'].astype(float)
    assert abs(y2.mean() - wrong) < 4.5 * math.sqrt(wrong * (1 - wrong) / y2.size)
