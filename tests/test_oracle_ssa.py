"""Pins of the oracle's SSA (Sec. 2.2, Eq. 1-2) against closed forms and exact
CME solutions.  Every check is statistical with a fixed seed; bounds are set
at >= 4 sigma so a correct implementation passes and a dropped term, wrong
sign, wrong propensity or wrong selection fails by a wide margin."""
import math

import numpy as np
import pytest
from scipy import stats

import workloads
from tests import _cme


def _chi2_ok(obs, expected_p, alpha=1e-4):
    """Pearson chi-square with bins of expected count < 5 merged."""
    n = obs.sum()
    e = expected_p * n
    o_b, e_b = [], []
    acc_o = acc_e = 0.0
    for oi, ei in zip(obs, e):
        acc_o += oi
        acc_e += ei
        if acc_e >= 5:
            o_b.append(acc_o); e_b.append(acc_e)
            acc_o = acc_e = 0.0
    if acc_e > 0:
        o_b[-1] += acc_o; e_b[-1] += acc_e
    o_b, e_b = np.asarray(o_b), np.asarray(e_b)
    chi2 = ((o_b - e_b) ** 2 / e_b).sum()
    return chi2 < stats.chi2.ppf(1 - alpha, len(o_b) - 1), chi2


def test_pure_decay_binomial(orc):
    # A -> 0 at rate k A: A(T) ~ Binomial(A0, exp(-k T)).
    A0, k, T = 1000, 1.0, 1.0
    m, p = workloads.pure_decay(A0, k, T)
    r = orc.run(m, p, seed=11, n_traj=4000, want_x=True)
    assert (r['status'] == 0).all() and (r['verdict'] == 1).all()
    a = r['x_final'][:, 0]
    q = math.exp(-k * T)
    mean, var = A0 * q, A0 * q * (1 - q)
    assert abs(a.mean() - mean) < 4.5 * math.sqrt(var / a.size)
    assert abs(a.var() / var - 1) < 0.12
    ks = np.arange(A0 + 1)
    hist = np.bincount(a, minlength=A0 + 1)
    ok, chi2 = _chi2_ok(hist, stats.binom.pmf(ks, A0, q))
    assert ok, chi2
    # the final state is the state occupied at T: entered at or before T
    assert (r['t_final'] <= T).all()


def test_immigration_death_poisson(orc):
    # 0 -> A (k1), A -> 0 (k2 A) from A0 = 0: A(T) ~ Poisson(k1/k2 (1 - e^{-k2 T})).
    m, _ = workloads.immigration_death()
    T = 60.0
    p = workloads.Property([workloads.atom(['A'], 'A', '>=', 0)], ('G', 0.0, T, ('atom', 0)))
    r = orc.run(m, p, seed=5, n_traj=3000, want_x=True)
    a = r['x_final'][:, 0]
    lam = 10.0 / 0.1 * (1 - math.exp(-0.1 * T))
    assert abs(a.mean() - lam) < 4.5 * math.sqrt(lam / a.size)
    assert abs(a.var() / lam - 1) < 0.12
    ks = np.arange(a.max() + 40)
    ok, chi2 = _chi2_ok(np.bincount(a, minlength=ks.size), stats.poisson.pmf(ks, lam))
    assert ok, chi2


def test_immigration_event_count_poisson(orc):
    # 0 -> A at rate k: the number of events with entry time <= T is Poisson(kT).
    k, T = 5.0, 10.0
    m, p = workloads.immigration_only(k, T)
    r = orc.run(m, p, seed=9, n_traj=4000)
    ev = r['events'].astype(np.int64)
    lam = k * T
    assert abs(ev.mean() - lam) < 4.5 * math.sqrt(lam / ev.size)
    ok, chi2 = _chi2_ok(np.bincount(ev, minlength=120), stats.poisson.pmf(np.arange(120), lam))
    assert ok, chi2


def test_homodimer_two_molecules(orc):
    # 2A -> B from A0 = 2: exactly one pair, so h = 1 and the reaction
    # happens by time t with probability 1 - exp(-c t).
    sp = ['A', 'B']
    c, t = 0.7, 1.3
    m = workloads.Model('dimer2', sp, [[0, 0]], [[-2, 1]], [[c]], [[2, 0]])
    p = workloads.Property([workloads.atom(sp, 'B', '>=', 1)], ('F', 0.0, t, ('atom', 0)))
    r = orc.run(m, p, seed=3, n_traj=20000)
    exact = 1 - math.exp(-c * t)
    assert abs(r['verdict'].mean() - exact) < 4.5 * math.sqrt(exact * (1 - exact) / 20000)


def test_heterodimer_and_selection_against_cme(orc):
    # A + B -> C (c1) competing with A -> 0 (c2); P(F[0,T] C >= 2) by CME.
    sp = ['A', 'B', 'C']
    m = workloads.Model('hetero', sp, [[0, 1], [0, -1]], [[-1, -1, 1], [-1, 0, 0]],
                        [[0.05, 0.4]], [[6, 4, 0]])
    T = 1.5
    p = workloads.Property([workloads.atom(sp, 'C', '>=', 2)], ('F', 0.0, T, ('atom', 0)))
    exact = _cme.eventually_probability(m, lambda x: x[2] >= 2, T)
    n = 20000
    r = orc.run(m, p, seed=21, n_traj=n)
    assert abs(r['verdict'].mean() - exact) < 4.5 * math.sqrt(exact * (1 - exact) / n)


def test_c1_matches_exact_cme(orc):
    # Immigration-death, F[0,100](A >= 130): exact value from the CME with
    # A = 130 absorbing (a 131-state chain), compared with 10,000 oracle
    # trajectories at Philox seed 0.
    m, p = workloads.immigration_death()
    exact = _cme.eventually_probability(m, lambda x: x[0] >= 130, 100.0)
    assert abs(exact - 0.0912186) < 5e-7
    r = orc.run(m, p, seed=0, n_traj=10000)
    from oracle import wilson
    _, lo, hi = wilson.wilson_interval(int(r['verdict'].sum()), 10000, 0.9999)
    assert lo <= exact <= hi
    # on-the-fly stopping: every true verdict stops at the first state with A = 130
    # and every false one at the first draw past t = 100
    assert (r['t_final'][r['verdict'] == 1] <= 100.0).all()


def test_instances_and_trajectories_are_independent_streams(orc):
    # different trajectory ids / instances give different paths; the same id
    # gives the same path whatever range it is run in.
    m, p = workloads.immigration_death(n_inst=2)
    a = orc.run(m, p, seed=1, instance=0, traj_begin=0, n_traj=50)
    b = orc.run(m, p, seed=1, instance=0, traj_begin=20, n_traj=10)
    assert (a['events'][20:30] == b['events']).all()
    assert (a['t_final'][20:30] == b['t_final']).all()
    c = orc.run(m, p, seed=1, instance=1, traj_begin=0, n_traj=50)
    assert (a['events'] != c['events']).sum() > 40
    d = orc.run(m, p, seed=2, instance=0, traj_begin=0, n_traj=50)
    assert (a['events'] != d['events']).sum() > 40


def test_event_budget_is_reported(orc):
    m, p = workloads.immigration_death()
    r = orc.run(m, p, seed=0, n_traj=200, budget=100)
    assert (r['status'] == 1).sum() > 150
    assert (r['events'][r['status'] == 1] == 100).all()


def test_absorbing_state_closes_the_path(orc):
    # A -> 0 from A0 = 3 with F[0,100](A >= 5): the path absorbs at A = 0
    # after exactly 3 events and the verdict is false.
    m, _ = workloads.pure_decay(3, 1.0, 1.0)
    p = workloads.Property([workloads.atom(['A'], 'A', '>=', 5)], ('F', 0.0, 100.0, ('atom', 0)))
    r = orc.run(m, p, seed=0, n_traj=100)
    assert (r['status'] == 0).all() and (r['verdict'] == 0).all() and (r['events'] == 3).all()


def birth_death_survival_exact(b, d, A0, T):
    """P(a linear birth-death lineage from A0 is alive at T) = 1 - P0(T),
    P0(T) = (d (e^{(b-d)T} - 1) / (b e^{(b-d)T} - d))^A0 (Kendall 1948)."""
    g = math.exp((b - d) * T)
    return 1.0 - (d * (g - 1.0) / (b * g - d)) ** A0


def test_birth_death_survival_closed_form(orc):
    # G[0,T](A > 0) on A -> 2A (b), A -> 0 (d A): the verdict is survival to T.
    m, p = workloads.birth_death_survival(1, b=1.0, d=0.8, A0=5, T=20.0)
    exact = birth_death_survival_exact(1.0, 0.8, 5, 20.0)
    r = orc.run(m, p, seed=21, n_traj=4000)
    y = r['verdict'].astype(float)
    assert abs(y.mean() - exact) < 4.5 * math.sqrt(exact * (1 - exact) / y.size), (y.mean(), exact)
    # a shorter horizon, where extinction is still under way
    m2, p2 = workloads.birth_death_survival(1, b=1.0, d=0.8, A0=2, T=3.0)
    exact2 = birth_death_survival_exact(1.0, 0.8, 2, 3.0)
    y2 = orc.run(m2, p2, seed=22, n_traj=8000)['verdict'].astype(float)
    assert abs(y2.mean() - exact2) < 4.5 * math.sqrt(exact2 * (1 - exact2) / y2.size), (y2.mean(), exact2)


@pytest.mark.parametrize('name', ['mm_degradation', 'autorepressor'])
def test_rate_law_factors_against_cme(orc, name):
    # Propensities with rational rate-law factors (Michaelis-Menten
    # degradation vmax A/(K + A); Hill-repressed production k K^2/(K^2 + A^2)):
    # the oracle's P(F[0,T] goal) against the exact CME solve of the same
    # chain (tests/_cme.py applies the factors independently).
    m, p = getattr(workloads, name)()
    atom = p.atoms[0]
    T = p.formula[2]
    if atom.op == '<=':
        goal = lambda x: x[0] <= atom.bound  # noqa: E731
    else:
        goal = lambda x: x[0] >= atom.bound  # noqa: E731
    exact = _cme.eventually_probability(m, goal, T, cap=300)
    assert 0.2 < exact < 0.8
    r = orc.run(m, p, seed=41, n_traj=20000)
    y = r['verdict'].astype(float)
    assert abs(y.mean() - exact) < 4.5 * math.sqrt(exact * (1 - exact) / y.size), (y.mean(), exact)


def test_rate_law_factor_dropped_is_detected(orc):
    # the same Hill-repressed gene without its factor is a plain
    # immigration-death chain with a different answer: the pin above fails
    # for an oracle that ignores factors
    m, p = workloads.autorepressor()
    exact = _cme.eventually_probability(m, lambda x: x[0] >= 48, 40.0, cap=300)
    plain = workloads.Model(m.name, m.species, m.reactants, m.stoich, m.rates, m.x0)
    wrong = _cme.eventually_probability(plain, lambda x: x[0] >= 48, 40.0, cap=300)
    assert abs(exact - wrong) > 0.2
    y = orc.run(plain, p, seed=41, n_traj=4000)['verdict'].astype(float)
    assert abs(y.mean() - wrong) < 4.5 * math.sqrt(wrong * (1 - wrong) / y.size)


def test_next_operator_closed_form(orc):
    # immigration-death from A = 0: the first event is an immigration at an
    # Exp(10) time, so X[0.05,0.2](A >= 1) holds with e^-0.5 - e^-2
    m, _ = workloads.immigration_death()
    p = workloads.Property([workloads.atom(['A'], 'A', '>=', 1)], ('X', 0.05, 0.2, ('atom', 0)))
    exact = math.exp(-0.5) - math.exp(-2.0)
    r = orc.run(m, p, seed=17, n_traj=20000)
    y = r['verdict'].astype(float)
    assert abs(y.mean() - exact) < 4.5 * math.sqrt(exact * (1 - exact) / y.size), (y.mean(), exact)
    # decided by the first event: when its time falls outside the window, at
    # the draw (no reaction applied); otherwise at the first state
    assert set(np.unique(r['events'])) <= {0, 1}


# Totals of the three-tier cascade that no reaction changes: each enzyme is
# free or in one of its complexes, and each tier's protein is in one of its
# phosphorylation states, free or bound.
MAPK_TOTALS = [
    ['E1', 'KKK_E1'],
    ['E2', 'KKKs_E2'],
    ['KKK', 'KKKs', 'KKK_E1', 'KKKs_E2', 'KK_KKKs', 'KKP_KKKs'],
    ['KKPase', 'KKPP_KKPase', 'KKP_KKPase'],
    ['KK', 'KKP', 'KKPP', 'KK_KKKs', 'KKP_KKKs', 'KKPP_KKPase', 'KKP_KKPase', 'K_KKPP', 'KP_KKPP'],
    ['KPase', 'KPP_KPase', 'KP_KPase'],
    ['K', 'KP', 'KPP', 'K_KKPP', 'KP_KKPP', 'KPP_KPase', 'KP_KPase'],
]


def test_state_updates_keep_the_cascade_totals(orc):
    """x += v_j on a 22-species, 30-reaction network: the seven totals of
    the cascade (the whole left null space of its stoichiometry, rank 15)
    stay at their initial values and no count goes negative, over
    trajectories of about 2.5e4 events each (the literal formula stops at
    the first KPP = 500)."""
    m, p = workloads.mapk_cascade(n_inst=2)
    W = np.zeros((len(MAPK_TOTALS), m.n_species), np.int64)
    for i, names in enumerate(MAPK_TOTALS):
        for nm in names:
            W[i, m.species.index(nm)] = 1
    st = m.stoich.astype(np.int64)
    assert not (st @ W.T).any()                                  # no reaction changes a total
    assert np.linalg.matrix_rank(W) == m.n_species - np.linalg.matrix_rank(st) == 7
    r = orc.run(m, p, seed=3, instance=1, n_traj=6, want_x=True)
    assert (r['events'] > 10_000).all()
    xf = r['x_final'].astype(np.int64)
    assert (xf >= 0).all()
    assert np.array_equal(xf @ W.T, np.tile(m.x0[1].astype(np.int64) @ W.T, (len(xf), 1)))
    assert not np.array_equal(xf[0], m.x0[1])                   # the state did move
