"""The seeded inputs follow their stated recipes (the generators hold none
of the method's arithmetic; these checks pin the shapes, ranges and
structure the benchmarks and parity tests rely on)."""
import math

import numpy as np

import workloads


def test_random_networks_recipe():
    batch = workloads.random_networks(n_inst=512)
    assert batch.n_inst == 512
    Ss, Rs, orders = [], [], []
    for model, prop in zip(batch.models, batch.properties):
        S, R = model.n_species, model.n_reactions
        Ss.append(S)
        Rs.append(R)
        assert 2 <= S <= 32 and 4 <= R <= 64 and model.n_inst == 1
        rates = model.rates[0]
        assert np.all(rates >= 1e-3) and np.all(rates <= 1.0)
        assert np.all((model.x0 >= 0) & (model.x0 <= 200))
        for j in range(R):
            ra, rb = model.reactants[j]
            assert ra >= 0 or rb < 0  # a single reactant sits in the first slot
            order = int(ra >= 0) + int(rb >= 0)
            orders.append(order)
            consumed = np.zeros(S, np.int64)
            for s in (ra, rb):
                if s >= 0:
                    consumed[s] += 1
            produced = model.stoich[j].astype(np.int64) + consumed
            assert np.all(produced >= 0)
            n_prod = int(produced.sum())
            assert n_prod <= (2 if order == 0 else order)  # mass is created only by order-0 reactions
        # F[0,50](X_k >= theta), theta = max(1, ceil(1.5 mean x0))
        assert prop.formula == ('F', 0.0, 50.0, ('atom', 0)) and len(prop.atoms) == 1
        a = prop.atoms[0]
        assert a.op == '>=' and np.count_nonzero(a.coef) == 1 and a.coef.max() == 1
        assert a.bound == max(1, math.ceil(1.5 * float(model.x0[0].mean())))
    # the draws cover their ranges
    assert min(Ss) == 2 and max(Ss) == 32 and min(Rs) <= 6 and max(Rs) >= 62
    counts = np.bincount(orders, minlength=3) / len(orders)
    assert np.all(np.abs(counts - 1 / 3) < 0.02)


def test_random_networks_are_seeded():
    a = workloads.random_networks(n_inst=8, seed=3)
    b = workloads.random_networks(n_inst=8, seed=3)
    c = workloads.random_networks(n_inst=8, seed=4)
    for x, y in zip(a.models, b.models):
        assert np.array_equal(x.stoich, y.stoich) and np.array_equal(x.rates, y.rates)
    assert any(x.n_species != y.n_species or not np.array_equal(x.x0, y.x0) for x, y in zip(a.models, c.models))


def test_cascade_recipe():
    m, p = workloads.mapk_cascade(n_inst=256)
    assert (m.n_species, m.n_reactions, m.n_inst) == (22, 30, 256)
    # ten enzymatic steps E + S <-> ES -> E + P: binding (order 2), unbinding
    # and catalysis (order 1) in that order
    for step in range(10):
        bind, unbind, cat = m.stoich[3 * step:3 * step + 3].astype(np.int64)
        assert np.array_equal(unbind, -bind)
        assert (m.reactants[3 * step] >= 0).all() and (m.reactants[3 * step + 1:3 * step + 3, 1] < 0).all()
        assert np.count_nonzero(cat) == 3 and cat.sum() == 1  # ES -> E + P
    # per-instance rate factors log-uniform in [0.8, 1.25] around shared base values
    ratio = m.rates / m.rates[0]
    assert np.all(ratio >= 0.8 / 1.25 - 1e-12) and np.all(ratio <= 1.25 / 0.8 + 1e-12)
    assert p.text.startswith('(KPP<500) U[0,200]')
    _, pv = workloads.mapk_cascade(n_inst=1, variant=True)
    assert pv.text.startswith('(KPP<2000) U[0,200]')


def test_lotka_volterra_family_recipe():
    m, p = workloads.lotka_volterra_family(1000, seed=1)
    base, _ = workloads.lotka_volterra()
    f = m.rates / base.rates[0]
    assert np.all(f >= 0.7 - 1e-12) and np.all(f <= 1.3 + 1e-12)
    # log-uniform: ln f is uniform on [ln 0.7, ln 1.3]
    lf = np.log(f).ravel()
    q = (lf - math.log(0.7)) / (math.log(1.3) - math.log(0.7))
    assert abs(q.mean() - 0.5) < 0.02 and abs(q.var() - 1 / 12) < 0.01
    assert np.all(m.x0 == 1000)


def test_large_random_networks_recipe():
    b = workloads.random_networks_large(64, seed=8)
    S = np.array([m.n_species for m in b.models])
    R = np.array([m.n_reactions for m in b.models])
    assert S.min() >= 16 and S.max() <= 64 and R.min() >= 65 and R.max() <= 255
    for m, p in zip(b.models, b.properties):
        a = p.atoms[0]
        k = int(np.nonzero(a.coef)[0][0])
        assert a.op == '>=' and a.bound > m.x0[0, k]  # not satisfied at t = 0
