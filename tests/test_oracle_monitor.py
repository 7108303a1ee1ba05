"""Pins of the oracle's BLTLc evaluator (Sec. 3.1 semantics) against a
brute-force evaluation written independently below:

* on complete (closed) paths, a literal transcription of the quantifiers
  (exists i / for all j < i) with Python's any/all over every position;
* on prefixes, the three-valued verdict is checked against all extensions
  of the prefix by up to two further states on a grid of entry times that
  includes ties with every interval end: a defined (true/false) verdict must
  agree with every extension (soundness); for single-operator formulas an
  undetermined verdict must have two extensions that disagree (completeness).
"""
import itertools
import random

import numpy as np
import pytest

import workloads

SP = ['A']


def _atoms():
    return [workloads.atom(SP, 'A', '>=', 2), workloads.atom(SP, 'A', '<=', 0),
            workloads.atom(SP, 'A', '==', 1), workloads.atom(SP, {'A': 2}, '>', 3.5),
            workloads.atom(SP, 'A', '!=', 3), workloads.atom(SP, 'A', '<', 1.5)]


A = lambda k: ('atom', k)
FORMULAS = [
    ('F', 0.0, 2.0, A(0)),
    ('F', 1.0, 2.0, A(0)),
    ('G', 0.0, 2.0, A(4)),
    ('G', 0.5, 1.5, A(5)),
    ('U', 0.0, 2.0, A(4), A(0)),
    ('U', 1.0, 3.0, ('not', A(1)), A(2)),
    ('U', 0.0, 2.0, A(5), ('and', A(0), ('F', 0.0, 1.0, A(1)))),
    ('U', 0.0, 2.0, ('true',), ('and', A(3), ('G', 0.0, 1.0, A(4)))),
    ('F', 0.0, 3.0, ('and', A(0), ('F', 0.0, 1.0, A(2)))),
    ('G', 0.0, 2.0, ('implies', A(0), ('F', 0.0, 1.0, A(1)))),
    ('and', ('F', 0.0, 2.0, A(0)), ('G', 0.0, 1.0, A(4))),
    ('or', ('F', 0.0, 1.0, A(2)), ('not', ('F', 0.0, 2.0, A(1)))),
    ('or', A(2), ('U', 0.0, 1.0, A(5), A(0))),
    ('implies', A(0), ('G', 0.0, 1.0, A(0))),
    ('X', 0.0, 1.0, A(0)),
    ('X', 0.5, 1.5, ('not', A(1))),
    ('and', ('X', 0.0, 2.0, A(2)), ('F', 0.0, 2.0, A(0))),
    ('or', ('X', 0.25, 1.0, A(5)), A(2)),
    # nesting beyond the unit monitor's shapes (the trace monitor's formulas)
    ('U', 0.0, 2.0, ('U', 0.0, 1.0, A(4), A(0)), A(2)),
    ('F', 0.0, 2.0, ('X', 0.0, 0.5, A(0))),
    ('G', 0.5, 2.0, ('X', 0.0, 1.0, ('not', A(1)))),
    ('U', 0.0, 2.5, ('X', 0.0, 1.0, A(4)), A(2)),
    ('F', 0.5, 1.5, ('G', 0.5, 1.0, A(0))),
    ('G', 0.0, 1.5, ('F', 0.0, 1.0, ('G', 0.0, 0.5, A(0)))),
    ('X', 0.0, 1.0, ('X', 0.0, 1.0, A(2))),
    ('U', 0.5, 2.0, ('F', 0.0, 0.5, A(5)), ('G', 0.0, 1.0, A(4))),
    ('or', ('G', 0.0, 1.0, ('F', 0.5, 1.0, A(0))), ('X', 0.0, 0.25, A(1))),
    ('implies', ('F', 0.0, 1.0, A(2)), ('U', 0.0, 2.0, ('not', A(1)), ('X', 0.25, 0.75, A(0)))),
]
NESTED = set(range(18, len(FORMULAS)))  # outside the unit monitor's fragment
SINGLE = {0, 1, 2, 3, 4, 5, 14, 15}  # single-operator formulas: Kleene is complete


def _atom_val(a, x):
    v = float(int(a.coef[0]) * x)
    return {'<': v < a.bound, '<=': v <= a.bound, '>=': v >= a.bound, '>': v > a.bound,
            '==': v == a.bound, '!=': v != a.bound}[a.op]


def sat(f, xs, ts, i, atoms):
    """sigma^i |= f on the complete finite path (xs, ts), literally."""
    k = f[0]
    if k == 'true':
        return True
    if k == 'false':
        return False
    if k == 'atom':
        return _atom_val(atoms[f[1]], xs[i])
    if k == 'not':
        return not sat(f[1], xs, ts, i, atoms)
    if k == 'and':
        return sat(f[1], xs, ts, i, atoms) and sat(f[2], xs, ts, i, atoms)
    if k == 'or':
        return sat(f[1], xs, ts, i, atoms) or sat(f[2], xs, ts, i, atoms)
    if k == 'implies':
        return (not sat(f[1], xs, ts, i, atoms)) or sat(f[2], xs, ts, i, atoms)
    if k == 'U':
        _, a, b, l, r = f
        return any(a <= ts[j] - ts[i] <= b and sat(r, xs, ts, j, atoms)
                   and all(sat(l, xs, ts, m, atoms) for m in range(i, j))
                   for j in range(i, len(xs)))
    if k == 'F':
        return sat(('U', f[1], f[2], ('true',), f[3]), xs, ts, i, atoms)
    if k == 'G':
        return not sat(('F', f[1], f[2], ('not', f[3])), xs, ts, i, atoms)
    if k == 'X':
        _, a, b, g = f
        return i + 1 < len(xs) and a <= ts[i + 1] - ts[i] <= b and sat(g, xs, ts, i + 1, atoms)
    raise ValueError(k)


def _paths(rng, n_paths):
    grid = [0.0, 0.5, 1.0, 1.5, 2.0, 2.5, 3.0, 3.5]
    out = []
    for L in range(1, 6):
        for xs in itertools.product(range(4), repeat=L):
            for _ in range(2):
                ts = [0.0]
                for _ in range(L - 1):
                    step = rng.choice([0.0, 0.25, 0.5, 1.0, rng.random()])
                    ts.append(ts[-1] + step)
                if rng.random() < 0.5:  # snap to the grid for exact ties
                    ts = [min(grid, key=lambda g: abs(g - t)) if abs(min(grid, key=lambda g: abs(g - t)) - t) < 0.3 else t for t in ts]
                    ts = list(np.maximum.accumulate(ts))
                out.append((list(xs), ts))
    rng.shuffle(out)
    return out[:n_paths]


@pytest.mark.parametrize('fi', range(len(FORMULAS)))
def test_closed_paths_match_literal_semantics(orc, fi):
    rng = random.Random(fi)
    f = FORMULAS[fi]
    prop = workloads.Property(_atoms(), f)
    for xs, ts in _paths(rng, 1500):
        want = sat(f, xs, ts, 0, prop.atoms)
        got = orc.eval_prefix(prop, 1, np.asarray(xs), np.asarray(ts), float('inf'), True)
        assert got == int(want), (f, xs, ts, got, want)


@pytest.mark.parametrize('fi', range(len(FORMULAS)))
def test_prefix_verdicts_are_sound_and_complete(orc, fi):
    rng = random.Random(100 + fi)
    f = FORMULAS[fi]
    prop = workloads.Property(_atoms(), f)
    checked = 0
    for xs, ts in _paths(rng, 160):
        tmin = ts[-1] + rng.choice([0.0, 0.0, 0.5, 1.0, 1.75])
        got = orc.eval_prefix(prop, 1, np.asarray(xs), np.asarray(ts), tmin, False)
        grid = sorted({tmin, tmin + 0.25, tmin + 0.5, 1.0, 1.5, 2.0, 3.0, 4.0, 5.0, 7.0} - {t for t in [] })
        grid = [g for g in grid if g >= tmin]
        verdicts = set()
        # extensions: absorb now, or one or two more states
        verdicts.add(sat(f, xs, ts, 0, prop.atoms))
        for y in range(4):
            for t1 in grid:
                verdicts.add(sat(f, xs + [y], ts + [t1], 0, prop.atoms))
                for y2 in range(4):
                    for t2 in grid:
                        if t2 >= t1:
                            verdicts.add(sat(f, xs + [y, y2], ts + [t1, t2], 0, prop.atoms))
        if got != 2:
            assert verdicts == {bool(got)}, (f, xs, ts, tmin, got, verdicts)
        elif fi in SINGLE:
            assert len(verdicts) == 2, (f, xs, ts, tmin, verdicts)
        checked += 1
    assert checked > 100


def test_nested_until_on_a_handmade_path(orc):
    # (A<=0 | A==1) U[0,200] (A>=2 & F[0,50] A<=0) with the nested window:
    # the candidate at t=10 needs a zero by t=60; the zero at t=60 is in
    # (closed interval), the zero at t=60.5 is not.
    sp = ['A']
    atoms = [workloads.atom(sp, 'A', '<', 2), workloads.atom(sp, 'A', '>=', 2),
             workloads.atom(sp, 'A', '<=', 0)]
    f = ('U', 0.0, 200.0, A(0), ('and', A(1), ('F', 0.0, 50.0, A(2))))
    prop = workloads.Property(atoms, f)
    xs, ts = [0, 1, 2, 1, 0], [0.0, 5.0, 10.0, 30.0, 60.0]
    assert orc.eval_prefix(prop, 1, np.asarray(xs), np.asarray(ts), 60.0, False) == 1
    ts2 = [0.0, 5.0, 10.0, 30.0, 60.5]
    assert orc.eval_prefix(prop, 1, np.asarray(xs), np.asarray(ts2), 60.5, False) == 0
    # before the zero: undetermined until the next entry time passes 60
    assert orc.eval_prefix(prop, 1, np.asarray(xs[:4]), np.asarray(ts[:4]), 59.0, False) == 2
    assert orc.eval_prefix(prop, 1, np.asarray(xs[:4]), np.asarray(ts[:4]), 60.0, False) == 2
    assert orc.eval_prefix(prop, 1, np.asarray(xs[:4]), np.asarray(ts[:4]), 60.01, False) == 0


@pytest.mark.parametrize('fi', range(len(FORMULAS)))
def test_prefix_verdicts_with_a_drawn_next_time_are_sound(orc, fi):
    # after the next entry time is drawn (tmin exact), a defined verdict must
    # agree with every extension whose next state is entered exactly then
    rng = random.Random(300 + fi)
    f = FORMULAS[fi]
    prop = workloads.Property(_atoms(), f)
    for xs, ts in _paths(rng, 160):
        t1 = ts[-1] + rng.choice([0.0, 0.25, 0.5, 1.0, 1.5])
        got = orc.eval_prefix(prop, 1, np.asarray(xs), np.asarray(ts), t1, False, tmin_exact=True)
        if got == 2:
            continue
        grid = [g for g in (t1, t1 + 0.25, t1 + 0.5, 1.0, 2.0, 3.0, 5.0) if g >= t1]
        verdicts = set()
        for y in range(4):
            verdicts.add(sat(f, xs + [y], ts + [t1], 0, prop.atoms))
            for y2 in range(4):
                for t2 in grid:
                    verdicts.add(sat(f, xs + [y, y2], ts + [t1, t2], 0, prop.atoms))
        assert verdicts == {bool(got)}, (f, xs, ts, t1, got, verdicts)
